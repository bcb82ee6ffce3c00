// fuse.cu — single-stream launch of the per-voxel map update; the device
// body is in fuse_dev.cuh.
#include "fuse_dev.cuh"
#include "kernels.h"

namespace prism {

template <bool BF16>
__global__ void __launch_bounds__(256) k_fuse(KParams P, MapPlanes M, const float* __restrict__ w2c,
                                              const float* __restrict__ depth, const float* __restrict__ rgb,
                                              const uint8_t* __restrict__ mask, DevStats* __restrict__ stats) {
    pdl_enter();
    fuse_tile<BF16>(P, M, w2c, depth, rgb, mask, stats, blockIdx.x);
}

cudaError_t launch_fuse(const KParams& P, const MapPlanes& M, const float* w2c, const float* depth,
                        const float* rgb, const uint8_t* mask, DevStats* stats, cudaStream_t s) {
    const unsigned int tiles = (unsigned int)(P.nbx * P.nby * P.nbz);
    if (P.bf16)
        launch_pdl(k_fuse<true>, tiles, 256, s, P, M, w2c, depth, rgb, mask, stats);
    else
        launch_pdl(k_fuse<false>, tiles, 256, s, P, M, w2c, depth, rgb, mask, stats);
    return cudaGetLastError();
}

}  // namespace prism
