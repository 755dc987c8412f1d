// snp_raster_ts32.cu -- forward and backward rasterizers for 32 x 32 tiles.
#include "snp_raster_launch.cuh"

namespace snp {

snp_status launch_fwd_ts32(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_fwd<32, false>(a, nc, form, bf16, st);
}

snp_status launch_bwd_ts32(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_bwd<32, false>(a, nc, form, bf16, st);
}

}  // namespace snp
