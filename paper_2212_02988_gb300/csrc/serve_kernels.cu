// serve_kernels.cu — the batched filter step of the serving runtime: one
// persistent launch per kernel of the step over the work of every stream in
// the batch (see serve.h).  Items of unequal cost (render tiles,
// localisation blocks) are taken dynamically from a per-launch counter;
// uniform ones (pixel blocks, voxel tiles) by a grid stride.
#include "fuse_dev.cuh"
#include "render_dev.cuh"
#include "serve.h"
#include "state_dev.cuh"
#include "track_dev.cuh"

namespace prism {

namespace {

// Member whose item range [off[i], off[i + 1]) holds `item` (off[0] = 0).
__device__ __forceinline__ int find_member(const int* off, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The block's next work item from a launch-wide counter.  The first barrier
// keeps every thread's use of the previous item (and of the block's shared
// memory) ahead of the next item's.
__device__ __forceinline__ int next_item(unsigned int* ctr) {
    __shared__ int s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    return s_item;
}

}  // namespace

// Prediction and the Gauss-Newton start pose matrices; block k runs the k-th
// localising member.
__global__ void __launch_bounds__(256) kb_predict(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b,
                                                  const double* __restrict__ imu) {
    pdl_enter();
    const int k = blockIdx.x;
    if (k >= b->n_loc) return;
    const BatchMember& m = b->m[b->loc[k]];
    const SlotDesc& S = slots[m.slot];
    predict_block(S.P, S.dev, imu + 7 * m.imu_off, m.n_imu, m.dt);
    __syncthreads();
    if (threadIdx.x < 32) {
        PoseArg pa{};
        prep_mats_warp(S.dev, PREP_REL, pa);
    }
}

// Depth validity of the observed frames.
__global__ void __launch_bounds__(256) kb_mask(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b) {
    pdl_enter();
    const int total = b->pix_off[b->n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_member(b->pix_off, b->n, item);
        const SlotDesc& S = slots[b->m[i].slot];
        const int p = (item - b->pix_off[i]) * 256 + threadIdx.x;
        if (p < S.P.W * S.P.H) depth_mask_px(S.P, S.depth, S.o_mask, p);
    }
}

__global__ void __launch_bounds__(256) kb_pack(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b) {
    pdl_enter();
    const int total = b->pix_off[b->n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_member(b->pix_off, b->n, item);
        const SlotDesc& S = slots[b->m[i].slot];
        const int p = (item - b->pix_off[i]) * 256 + threadIdx.x;
        if (p < S.P.W * S.P.H) anchor_pack_px(S.P, S.a_depth, S.a_rgb, S.a0, S.a1, p);
    }
}

// One localisation pass of every localising member; item = one virtual block.
template <int MODE>
__global__ void __launch_bounds__(Block<MODE>::threads, 1) kb_track(const SlotDesc* __restrict__ slots, BatchDesc* __restrict__ b,
                                                int ctr) {
    pdl_enter();
    const int* off = MODE == TRACK_GN ? b->gn_off : b->lap_off;
    const int total = off[b->n_loc];
    for (;;) {
        const int item = next_item(&b->ctr[ctr]);
        if (item >= total) break;
        const int k = find_member(off, b->n_loc, item);
        const SlotDesc& S = slots[b->m[b->loc[k]].slot];
        const int nvb = MODE == TRACK_GN ? S.grid_gn : S.grid_lap;
        track_item<MODE>(S.P, S.depth, S.rgb, S.o_mask, S.a0, S.a1, S.dev, S.partials, S.pstride, S.counter, S.stats,
                         item - off[k], nvb);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256, 4) kb_fuse(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b) {
    pdl_enter();
    __shared__ float sM[9], sb[3];
    const int total = b->fuse_off[b->n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_member(b->fuse_off, b->n, item);
        const SlotDesc& S = slots[b->m[i].slot];
        if (S.dev->rejected) continue;   // the member's localisation was rejected: its frame is not fused
        load_w2c(S.dev->w2c, sM, sb);
        __syncthreads();
        fuse_tile<BF16>(S.P, S.M, sM, sb, S.depth, S.rgb, S.o_mask, S.stats, (uint32_t)(item - b->fuse_off[i]));
        __syncthreads();   // the shared matrices, cull flag and reduction scratch are reused by the next item
    }
}

// The brick bounds of every member after its fuse; item = one top-level
// brick (render_dev.cuh).
__global__ void __launch_bounds__(512) kb_bricks(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b) {
    pdl_enter();
    const int total = b->brick_off[b->n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_member(b->brick_off, b->n, item);
        const SlotDesc& S = slots[b->m[i].slot];
        render_detail::brick_pyramid_block(S.P, S.M, item - b->brick_off[i]);
    }
}

// The anchor render at each member's new state mean; item = one 16x8 tile.
template <bool BF16>
__global__ void __launch_bounds__(128) kb_render(const SlotDesc* __restrict__ slots, BatchDesc* __restrict__ b,
                                                 int ctr) {
    pdl_enter();
    __shared__ float sR[9], sc[3];
    const int total = b->tiles_off[b->n];
    for (;;) {
        const int item = next_item(&b->ctr[ctr]);
        if (item >= total) break;
        const int i = find_member(b->tiles_off, b->n, item);
        const SlotDesc& S = slots[b->m[i].slot];
        const int t = item - b->tiles_off[i];
        DevState* dev = S.dev;
        if (threadIdx.x < 12) {
            if (threadIdx.x < 9) sR[threadIdx.x] = dev->c2w[threadIdx.x];
            else sc[threadIdx.x - 9] = dev->c2w[threadIdx.x];
        }
        // the state mean (t[3], q[4], contiguous) becomes the anchor's pose
        if (t == 0 && threadIdx.x < 7) dev->anchor_pose[threadIdx.x] = dev->t[threadIdx.x];
        __syncthreads();
        const int tx = t % S.tiles_x, ty = t / S.tiles_x;
        switch (S.px_spec) {
            case 66: render_tile<BF16, false, 66>(S.P, sR, sc, S.M, S.a_depth, S.a_rgb, nullptr, nullptr, S.stats, tx, ty); break;
            case 130: render_tile<BF16, false, 130>(S.P, sR, sc, S.M, S.a_depth, S.a_rgb, nullptr, nullptr, S.stats, tx, ty); break;
            case 258: render_tile<BF16, false, 258>(S.P, sR, sc, S.M, S.a_depth, S.a_rgb, nullptr, nullptr, S.stats, tx, ty); break;
            default: render_tile<BF16, false, 0>(S.P, sR, sc, S.M, S.a_depth, S.a_rgb, nullptr, nullptr, S.stats, tx, ty);
        }
    }
}

// Each member's posterior (and device flags, which are cleared) to `out`.
__global__ void __launch_bounds__(256) kb_out(const SlotDesc* __restrict__ slots, const BatchDesc* __restrict__ b,
                                              ServeOut* __restrict__ out) {
    pdl_enter();
    const int i = blockIdx.x;
    if (i >= b->n) return;
    DevState* d = slots[b->m[i].slot].dev;
    ServeOut& o = out[i];
    for (int e = threadIdx.x; e < 144; e += blockDim.x) o.cov[e] = d->cov[e];
    if (threadIdx.x < 3) {
        o.t[threadIdx.x] = d->t[threadIdx.x];
        o.v[threadIdx.x] = d->v[threadIdx.x];
        o.w[threadIdx.x] = d->w[threadIdx.x];
    }
    if (threadIdx.x < 4) o.q[threadIdx.x] = d->q[threadIdx.x];
    if (threadIdx.x == 0) {
        o.n_localised = d->n_localised;
        o.flags = d->flags;
        d->flags = 0;
    }
}

// ----------------------------------------------------------------- host side
namespace {

template <typename K>
int grid_of(K kern, int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
    return (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
}

}  // namespace

cudaError_t batch_grids(bool bf16, BatchGrids* g) {
    g->pix = grid_of(kb_mask, 256);
    g->bricks = grid_of(kb_bricks, 512);
    g->track_gn = grid_of(kb_track<TRACK_GN>, Block<TRACK_GN>::threads);
    g->track_lap = grid_of(kb_track<TRACK_LAPLACE>, Block<TRACK_LAPLACE>::threads);
    g->fuse = bf16 ? grid_of(kb_fuse<true>, 256) : grid_of(kb_fuse<false>, 256);
    g->render = bf16 ? grid_of(kb_render<true>, 128) : grid_of(kb_render<false>, 128);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const SlotDesc* slots, BatchDesc* batch, const double* imu, ServeOut* out, int n_gn,
                              bool bf16, const BatchGrids& g, cudaStream_t s) {
    cudaError_t e;
#define PRISM_BK(call)                        \
    do {                                      \
        if ((e = (call)) != cudaSuccess) return e; \
    } while (0)
    PRISM_BK(launch_pdl(kb_predict, kServeMaxSlots, 256, s, slots, batch, imu));
    PRISM_BK(launch_pdl(kb_mask, g.pix, 256, s, slots, batch));
    for (int it = 0; it < n_gn; ++it) PRISM_BK(launch_pdl(kb_track<TRACK_GN>, g.track_gn, Block<TRACK_GN>::threads, s, slots, batch, it));
    PRISM_BK(launch_pdl(kb_track<TRACK_LAPLACE>, g.track_lap, Block<TRACK_LAPLACE>::threads, s, slots, batch, n_gn));
    if (bf16) PRISM_BK(launch_pdl(kb_fuse<true>, g.fuse, 256, s, slots, batch));
    else PRISM_BK(launch_pdl(kb_fuse<false>, g.fuse, 256, s, slots, batch));
    PRISM_BK(launch_pdl(kb_bricks, g.bricks, 512, s, slots, batch));
    if (bf16) PRISM_BK(launch_pdl(kb_render<true>, g.render, 128, s, slots, batch, n_gn + 1));
    else PRISM_BK(launch_pdl(kb_render<false>, g.render, 128, s, slots, batch, n_gn + 1));
    PRISM_BK(launch_pdl(kb_pack, g.pix, 256, s, slots, batch));
    PRISM_BK(launch_pdl(kb_out, kServeMaxSlots, 256, s, slots, batch, out));
#undef PRISM_BK
    return cudaSuccess;
}

}  // namespace prism
