// snp_raster_ts8.cu -- forward and backward rasterizers for 8 x 8 tiles.
#include "snp_raster_launch.cuh"

namespace snp {

snp_status launch_fwd_ts8(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_fwd<8, false>(a, nc, form, bf16, st);
}

snp_status launch_bwd_ts8(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    return dispatch_bwd<8, false>(a, nc, form, bf16, st);
}

}  // namespace snp
