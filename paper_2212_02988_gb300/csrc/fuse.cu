// fuse.cu — single-stream launch of the per-voxel map update; the device
// body is in fuse_dev.cuh.
#include <cuda/atomic>

#include "fuse_dev.cuh"
#include "kernels.h"

namespace prism {

template <bool BF16>
__global__ void __launch_bounds__(256) k_fuse(KParams P, MapPlanes M, const float* __restrict__ w2c,
                                              const float* __restrict__ depth, const float* __restrict__ rgb,
                                              const uint8_t* __restrict__ mask, DevStats* __restrict__ stats) {
    pdl_enter();
    __shared__ float sM[9], sb[3];
    load_w2c(w2c, sM, sb);
    __syncthreads();
    fuse_tile<BF16>(P, M, sM, sb, depth, rgb, mask, stats, blockIdx.x);
}

// The tiles in the frustum, appended to `list` (ctr[0] counts them; the
// order is irrelevant: every tile's update is independent of the others).
// rejected (nullable): a nonzero value lists no tile (the localisation of
// this step was rejected, so its frame is not fused).
__global__ void __launch_bounds__(256) k_fuse_cull(KParams P, const float* __restrict__ w2c, int* __restrict__ list,
                                                   unsigned int* __restrict__ ctr, const int* __restrict__ rejected) {
    pdl_enter();
    __shared__ float sM[9], sb[3];
    load_w2c(w2c, sM, sb);
    __syncthreads();
    const int n = P.nbx * P.nby * P.nbz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (t < n && !(rejected && *rejected)) keep = !tile_outside_frustum(P, sM, sb, t % P.nbx, (t / P.nbx) % P.nby, t / (P.nbx * P.nby));
    const unsigned int ballot = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31;
    unsigned int base = 0;
    if (lane == 0 && ballot) base = atomicAdd(&ctr[0], (unsigned int)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) list[base + __popc(ballot & ((1u << lane) - 1u))] = t;
}

// Persistent over the listed tiles; the last block to finish (ticket in
// ctr[1]) resets both counters for the next frame.
template <bool BF16>
__global__ void __launch_bounds__(256, 4) k_fuse_list(KParams P, MapPlanes M, const float* __restrict__ w2c,
                                                   const float* __restrict__ depth, const float* __restrict__ rgb,
                                                   const uint8_t* __restrict__ mask, DevStats* __restrict__ stats,
                                                   const int* __restrict__ list, unsigned int* __restrict__ ctr) {
    pdl_enter();
    __shared__ float sM[9], sb[3];
    load_w2c(w2c, sM, sb);
    __syncthreads();
    const unsigned int count = ctr[0];
    for (unsigned int i = blockIdx.x; i < count; i += gridDim.x) {
        fuse_tile<BF16, false>(P, M, sM, sb, depth, rgb, mask, stats, (uint32_t)list[i]);
        __syncthreads();   // the tile's shared reduction scratch is reused by the next item
    }
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> ticket(ctr[1]);
        s_last = ticket.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        ctr[0] = 0u;
        ctr[1] = 0u;
    }
}

template <bool BF16>
static int fuse_grid() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fuse_list<BF16>, 256, 0);
        cached = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
    }
    return cached;
}

cudaError_t launch_fuse_listed(const KParams& P, const MapPlanes& M, const float* w2c, const float* depth,
                               const float* rgb, const uint8_t* mask, DevStats* stats, int* list, unsigned int* ctr,
                               const int* rejected, cudaStream_t s) {
    const int n = P.nbx * P.nby * P.nbz;
    cudaError_t e = launch_pdl(k_fuse_cull, (n + 255) / 256, 256, s, P, w2c, list, ctr, rejected);
    if (e != cudaSuccess) return e;
    if (P.bf16) return launch_pdl(k_fuse_list<true>, fuse_grid<true>(), 256, s, P, M, w2c, depth, rgb, mask, stats,
                                  (const int*)list, ctr);
    return launch_pdl(k_fuse_list<false>, fuse_grid<false>(), 256, s, P, M, w2c, depth, rgb, mask, stats,
                      (const int*)list, ctr);
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
