// snp_raster_ts16.cu -- forward and backward rasterizers for 16 x 16 tiles.
#include "snp_raster_launch.cuh"

namespace snp {

snp_status launch_fwd_ts16(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_fwd<16, true>(a, nc, form, bf16, st);
}

snp_status launch_bwd_ts16(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_bwd<16, true>(a, nc, form, bf16, st);
}

}  // namespace snp
