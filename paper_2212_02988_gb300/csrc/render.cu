// render.cu — single-stream launches of the render (App. B) and of the anchor
// masks and packing; the device bodies are in render_dev.cuh.
#include "kernels.h"
#include "render_dev.cuh"

namespace prism {

// Without DETAIL counters the march takes two samples a step (render_tile's
// NS): 8 blocks an SM (64 registers) with two samples' loads in flight beat
// 10 blocks with one, on the rays that march longest.  One block per 16x8
// tile, block b rendering tile plan.order[b] (row-major without an order);
// with plan.cost the block records the tile's cost for the next plan.
template <bool BF16, bool DETAIL, int PX>
__global__ void __launch_bounds__(128, DETAIL ? 10 : 8) k_render(KParams P, const float* __restrict__ mats, MapPlanes M,
                                                float* __restrict__ depth, float* __restrict__ rgb,
                                                uint8_t* __restrict__ mask, int32_t* __restrict__ hitk,
                                                DevStats* __restrict__ stats, const double* __restrict__ anchor_src,
                                                double* __restrict__ anchor_dst, RenderPlan plan) {
    pdl_enter();
    __shared__ float sR[9], sc[3];
    __shared__ uint32_t s_cost;
    if (threadIdx.x < 12) {
        if (threadIdx.x < 9) sR[threadIdx.x] = mats[threadIdx.x];
        else sc[threadIdx.x - 9] = mats[threadIdx.x];
    }
    if (threadIdx.x == 0) s_cost = 0u;
    if (blockIdx.x == 0) {
        if (anchor_dst && threadIdx.x < 7) anchor_dst[threadIdx.x] = anchor_src[threadIdx.x];
        if (plan.rot && threadIdx.x < 12) plan.rot[threadIdx.x] = mats[threadIdx.x];
    }
    __syncthreads();
    const int gx = (P.W + 15) >> 4, nt = gx * ((P.H + 7) >> 3);
    int tile = plan.order ? plan.order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)tile >= (unsigned)nt) {   // (never taken: the order is a permutation)
        PRISM_IN_RANGE(P, CHK_PLAN, tile, nt);
        tile = (int)blockIdx.x;
    }
    const int ns = render_tile<BF16, DETAIL, PX, DETAIL ? 1 : 2>(P, sR, sc, M, depth, rgb, mask, hitk, stats,
                                                                   tile % gx, tile / gx);
    if (plan.cost) {
        const unsigned int wmax = __reduce_max_sync(0xffffffffu, (unsigned int)ns);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_cost, wmax);
        __syncthreads();
        if (threadIdx.x == 0) plan.cost[tile] = s_cost;
    }
}

__global__ void __launch_bounds__(1024) k_render_plan(KParams P, RenderPlanIn in) {
    pdl_enter();
    render_plan_block(P, in);
}

__global__ void k_depth_mask(KParams P, const float* __restrict__ depth, uint8_t* __restrict__ mask) {
    pdl_enter();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P.W * P.H) depth_mask_px(P, depth, mask, p);
}

__global__ void __launch_bounds__(256) k_anchor_pack(KParams P, const float* __restrict__ depth,
                                                     const float* __restrict__ rgb, float4* __restrict__ a0,
                                                     float4* __restrict__ a1) {
    pdl_enter();
    anchor_pack_tile(P, depth, rgb, a0, a1, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------- launchers
// The compile-time padded stride for cubic grids of 64, 128 and 256 voxels a
// side, else 0 (runtime strides).
int render_px_specialisation(const KParams& P) {
    if (P.nx != P.ny || P.px != P.py) return 0;
    return (P.nx == 64 || P.nx == 128 || P.nx == 256) ? (int)P.px : 0;
}

template <bool BF16, bool DETAIL>
static void render_px(const KParams& P, unsigned int grid, const float* mats, const MapPlanes& M, float* depth,
                      float* rgb, uint8_t* mask, int32_t* hitk, DevStats* stats, const double* anchor_src,
                      double* anchor_dst, const RenderPlan& plan, cudaStream_t s) {
    switch (render_px_specialisation(P)) {
        case 66: launch_pdl(k_render<BF16, DETAIL, 66>, grid, 128, s, P, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan); break;
        case 130: launch_pdl(k_render<BF16, DETAIL, 130>, grid, 128, s, P, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan); break;
        case 258: launch_pdl(k_render<BF16, DETAIL, 258>, grid, 128, s, P, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan); break;
        default: launch_pdl(k_render<BF16, DETAIL, 0>, grid, 128, s, P, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan);
    }
}

cudaError_t launch_render(const KParams& P, const float* mats, const MapPlanes& M, float* depth, float* rgb,
                          uint8_t* mask, int32_t* hitk, DevStats* stats, const double* anchor_src,
                          double* anchor_dst, bool detail, cudaStream_t s, const RenderPlan& plan) {
    const unsigned int grid = (unsigned int)(((P.W + 15) / 16) * ((P.H + 7) / 8));
    if (P.bf16) {
        if (detail) render_px<true, true>(P, grid, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan, s);
        else render_px<true, false>(P, grid, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan, s);
    } else {
        if (detail) render_px<false, true>(P, grid, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan, s);
        else render_px<false, false>(P, grid, mats, M, depth, rgb, mask, hitk, stats, anchor_src, anchor_dst, plan, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_render_plan(const KParams& P, const RenderPlanIn& in, cudaStream_t s) {
    return launch_pdl(k_render_plan, 1, 1024, s, P, in);
}

cudaError_t launch_depth_mask(const KParams& P, const float* depth, uint8_t* mask, cudaStream_t s) {
    int n = P.W * P.H;
    launch_pdl(k_depth_mask, (n + 255) / 256, 256, s, P, depth, mask);
    return cudaGetLastError();
}

cudaError_t launch_anchor_pack(const KParams& P, const float* depth, const float* rgb, float4* a0, float4* a1,
                               cudaStream_t s) {
    const dim3 grid((P.W + kPackTW - 1) / kPackTW, (P.H + kPackTH - 1) / kPackTH);
    return launch_pdl(k_anchor_pack, grid, kPackTW * kPackTH, s, P, depth, rgb, a0, a1);
}

}  // namespace prism
