// rollout.cu — predictive rollouts from the filter belief (App. I,
// "Prediction and Control"; Fig. 1).  A candidate control sequence
// propagates q(s_t) with the transition of App. E.1/E.2 and no observation:
// each frame's prior (mean, velocities and the full 12x12 covariance) is the
// next frame's state.  The map mean is then rendered at every predicted pose
// mean, all frames in one launch, with the render's tile body (App. B).
#include <cstddef>

#include "kernels.h"
#include "prism_dev.cuh"
#include "render_dev.cuh"
#include "state_dev.cuh"

namespace prism {

// The posterior (t, q, v, w, cov) and the prior (pt, pq, pv, pw, pcov) are
// each 157 contiguous doubles, and RollOut starts with the same 157.
constexpr int kBelief = 3 + 4 + 3 + 3 + 144;
static_assert(offsetof(DevState, cov) == offsetof(DevState, t) + 13 * sizeof(double), "posterior layout");
static_assert(offsetof(DevState, pcov) == offsetof(DevState, pt) + 13 * sizeof(double), "prior layout");
static_assert(offsetof(RollOut, cov) == 13 * sizeof(double) && offsetof(RollOut, n_localised) == kBelief * 8,
              "rollout record layout");

__device__ __forceinline__ double* belief_of(DevState* d) {
    return reinterpret_cast<double*>(reinterpret_cast<char*>(d) + offsetof(DevState, t));
}
__device__ __forceinline__ const double* prior_of(const DevState* d) {
    return reinterpret_cast<const double*>(reinterpret_cast<const char*>(d) + offsetof(DevState, pt));
}

// One block of 256 threads per candidate sequence (block index = sequence).
__global__ void __launch_bounds__(256) k_rollout_states(KParams P, const DevState* __restrict__ src,
                                                        DevState* scratch, int k, const double* __restrict__ imu,
                                                        const long long* __restrict__ row0,
                                                        const int* __restrict__ counts,
                                                        const double* __restrict__ dts, RollOut* __restrict__ out,
                                                        float* __restrict__ mats) {
    pdl_enter();
    const int seq = blockIdx.x, tid = threadIdx.x;
    DevState* dev = scratch + seq;
    {
        const double* s = reinterpret_cast<const double*>(reinterpret_cast<const char*>(src) + offsetof(DevState, t));
        double* d = belief_of(dev);
        for (int e = tid; e < kBelief; e += blockDim.x) d[e] = s[e];
        if (tid == 0) {
            dev->n_localised = src->n_localised;
            dev->flags = 0;
        }
    }
    __syncthreads();
    for (int i = 0; i < k; ++i) {
        const int f = seq * k + i;
        predict_block(P, dev, imu + 7 * row0[f], counts[f], dts[f]);
        __syncthreads();
        // the prior becomes the state, and the frame's record
        const double* pr = prior_of(dev);
        double* d = belief_of(dev);
        double* o = out[f].t;
        for (int e = tid; e < kBelief; e += blockDim.x) {
            const double v = pr[e];
            d[e] = v;
            o[e] = v;
        }
        __syncthreads();
        if (tid < 32) {
            if (tid == 0) {
                out[f].n_localised = dev->n_localised;
                out[f].flags = dev->flags;
                dev->flags = 0;
            }
            // the pose normalised as a host-given render pose is (IEEE FP64,
            // same operation order), then its decision matrices
            const double* q = dev->q;
            const double n = __dsqrt_rn(__dadd_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])),
                __dmul_rn(q[3], q[3])));
            const double pn[7] = {dev->t[0], dev->t[1], dev->t[2], __ddiv_rn(q[0], n), __ddiv_rn(q[1], n),
                                  __ddiv_rn(q[2], n), __ddiv_rn(q[3], n)};
            warp_mats_c2w(pn, mats + 12 * (size_t)f);
        }
        __syncthreads();
    }
}

cudaError_t launch_rollout_states(const KParams& P, const DevState* src, DevState* scratch, int n_seq, int k,
                                  const double* imu, const long long* row0, const int* counts, const double* dts,
                                  RollOut* out, float* mats, cudaStream_t s) {
    return launch_pdl(k_rollout_states, n_seq, 256, s, P, src, scratch, k, imu, row0, counts, dts, out, mats);
}

// The render of many poses in one launch: grid z indexes the frame.
template <bool BF16, int PX>
__global__ void __launch_bounds__(128, 10) k_render_frames(KParams P, const float* __restrict__ mats, MapPlanes M,
                                                       float* __restrict__ depth, float* __restrict__ rgb,
                                                       int32_t* __restrict__ hitk, DevStats* __restrict__ stats) {
    pdl_enter();
    __shared__ float sR[9], sc[3];
    const size_t f = blockIdx.z, npix = (size_t)P.W * P.H;
    if (threadIdx.x < 12) {
        const float v = mats[12 * f + threadIdx.x];
        if (threadIdx.x < 9) sR[threadIdx.x] = v;
        else sc[threadIdx.x - 9] = v;
    }
    __syncthreads();
    render_tile<BF16, false, PX>(P, sR, sc, M, depth ? depth + f * npix : nullptr,
                                 rgb ? rgb + 3 * f * npix : nullptr, nullptr, hitk ? hitk + f * npix : nullptr,
                                 stats, blockIdx.x, blockIdx.y);
}

template <bool BF16>
static cudaError_t render_frames_px(const KParams& P, dim3 grid, const float* mats, const MapPlanes& M, float* depth,
                                   float* rgb, int32_t* hitk, DevStats* stats, cudaStream_t s) {
    switch (render_px_specialisation(P)) {
        case 66: return launch_pdl(k_render_frames<BF16, 66>, grid, 128, s, P, mats, M, depth, rgb, hitk, stats);
        case 130: return launch_pdl(k_render_frames<BF16, 130>, grid, 128, s, P, mats, M, depth, rgb, hitk, stats);
        case 258: return launch_pdl(k_render_frames<BF16, 258>, grid, 128, s, P, mats, M, depth, rgb, hitk, stats);
        default: return launch_pdl(k_render_frames<BF16, 0>, grid, 128, s, P, mats, M, depth, rgb, hitk, stats);
    }
}

cudaError_t launch_render_frames(const KParams& P, const float* mats, int frames, const MapPlanes& M, float* depth,
                                 float* rgb, int32_t* hitk, DevStats* stats, cudaStream_t s) {
    if (frames < 1 || frames > 65535) return cudaErrorInvalidValue;
    const dim3 grid((P.W + 15) / 16, (P.H + 7) / 8, frames);
    return P.bf16 ? render_frames_px<true>(P, grid, mats, M, depth, rgb, hitk, stats, s)
                  : render_frames_px<false>(P, grid, mats, M, depth, rgb, hitk, stats, s);
}

}  // namespace prism
