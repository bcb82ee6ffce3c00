// adam.cu — the paper's pose optimiser (App. F.2, "Pose optimisation"): Adam
// with its momentum disabled, on the objective of App. E.3
// (Eq. pointtoplanelaplace), as an alternative to the Gauss-Newton passes.
//
// One block runs every step.  Per step: warp 0 derives the pose of the
// iterate xi (tangent coordinates at the prior mean, the retraction of the
// Gauss-Newton passes) and its FP32 matrices into the anchor camera (the
// decision recipe), warp 1 the tangent map C = diag(Ra^T, Ra^T J_l(xi_theta));
// thread k < pixels draws pixel floor(n u), u the high 32 bits of SplitMix64
// output (n_localised steps + s - 1) pixels + k from `seed` over 2^32, and
// evaluates it with the localisation passes' device code (the L1 subgradient
// sign(r) J / b of its kept residuals); a fixed-order block sum gives the
// anchor-frame gradient g'.  Warp 0 then forms the tangent gradient
// g = (n_pixels / pixels) C^T g' + L xi (the data term estimates the
// full-image objective; L = prior pose precision) and takes the Adam step,
// one component a lane: v = beta2 v + (1 - beta2) g^2, v_hat = v / (1 - beta2^s),
// xi -= lr g / (sqrt(v_hat) + eps), lr = lr_t on translation, lr_r on rotation.
// The unstated constants (beta2, eps) take Adam's defaults in the caller's
// configuration.
#include "kernels.h"
#include "linalg64.cuh"
#include "prism_dev.cuh"
#include "track_dev.cuh"

namespace prism {

namespace {

// Output i of SplitMix64 started at state `seed` (Steele, Lea and Flood 2014:
// the golden gamma increment and the variant-13 finaliser).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The pose of xi on every lane of the calling warp: t = pt + xi_t,
// q = normalise(Exp(xi_theta) (x) pq).
__device__ __forceinline__ void warp_pose_of(const double* xi, const double* pq, const double* pt, double pose[7]) {
    const int lane = threadIdx.x & 31;
    const double qn = warp_quat_exp_mul(xi + 3, pq);
    pose[3] = __shfl_sync(0xffffffffu, qn, 0);
    pose[4] = __shfl_sync(0xffffffffu, qn, 1);
    pose[5] = __shfl_sync(0xffffffffu, qn, 2);
    pose[6] = __shfl_sync(0xffffffffu, qn, 3);
    const int ta = lane < 3 ? lane : 0;
    const double tv = pt[ta] + xi[ta];
    pose[0] = __shfl_sync(0xffffffffu, tv, 0);
    pose[1] = __shfl_sync(0xffffffffu, tv, 1);
    pose[2] = __shfl_sync(0xffffffffu, tv, 2);
}

constexpr int kAdamThreads = 256;

__global__ void __launch_bounds__(kAdamThreads, 1)
    k_adam(KParams P, const float* __restrict__ od, const float* __restrict__ orgb, const uint8_t* __restrict__ om,
           const float4* __restrict__ a0, const float4* __restrict__ a1, DevState* dev, AdamArgs A) {
    pdl_enter();
    constexpr int N = NV<TRACK_ADAM>::value;   // g' (6), cost, count
    __shared__ float sMb[12];
    __shared__ double s_xi[6], s_C[18], s_anchor[7], s_pq[4], s_pt[3], s_prec[36];
    __shared__ float swarp[kAdamThreads / 32][N];
    __shared__ unsigned long long s_c0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 7) s_anchor[tid] = dev->anchor_pose[tid];
    else if (tid < 11) s_pq[tid - 7] = dev->pq[tid - 7];
    else if (tid < 14) s_pt[tid - 11] = dev->pt[tid - 11];
    else if (tid < 20) s_xi[tid - 14] = 0.0;
    else if (tid >= 32 && tid < 68) s_prec[tid - 32] = dev->prec_pp[tid - 32];
    if (tid == 0) s_c0 = (unsigned long long)dev->n_localised * (unsigned long long)A.steps * (unsigned long long)A.pixels;
    __syncthreads();
    const float* sM = sMb;
    const float* sb = sMb + 9;
    const int W = P.W, Hh = P.H, NP = W * Hh;
    const float fW1 = (float)(W - 1), fH1 = (float)(Hh - 1), fW2 = (float)(W - 2), fH2 = (float)(Hh - 2);
    const EvalConst kc{1.0f / P.b_geo32, 1.0f / P.b_rgb32};
    const double scale = (double)NP / (double)A.pixels;
    // warp 1: the anchor rotation's entries (lanes 0..8), fixed over the steps
    double ra = 0.0;
    if (warp == 1) ra = quat_R_entry_rn(s_anchor[3], s_anchor[4], s_anchor[5], s_anchor[6], lane < 9 ? lane : 0);
    double v2 = 0.0, b2t = 1.0;   // warp 0, lane i < 6: second moment of component i
    for (int s = 1; s <= A.steps; ++s) {
        if (warp == 0) {
            double pose[7];
            warp_pose_of(s_xi, s_pq, s_pt, pose);
            warp_mats_rel(pose, s_anchor, sMb);
        } else if (warp == 1) {
            // C0 = Ra^T, C1 = Ra^T J_l(xi_theta): lanes 0..8 hold Ra entries, J_l entries
            const int e = lane < 9 ? lane : 0, i = e / 3, j = e % 3;
            const double jl = so3_exp_jl_entry(s_xi + 3, false, i, j);
            const double ra_i0 = __shfl_sync(0xffffffffu, ra, i), ra_i1 = __shfl_sync(0xffffffffu, ra, 3 + i),
                         ra_i2 = __shfl_sync(0xffffffffu, ra, 6 + i);
            const double jl_0j = __shfl_sync(0xffffffffu, jl, j), jl_1j = __shfl_sync(0xffffffffu, jl, 3 + j),
                         jl_2j = __shfl_sync(0xffffffffu, jl, 6 + j);
            const double c0 = __shfl_sync(0xffffffffu, ra, 3 * j + i);
            if (lane < 9) {
                s_C[lane] = c0;
                s_C[9 + lane] = fdot3(ra_i0, jl_0j, ra_i1, jl_1j, ra_i2, jl_2j);
            }
        }
        __syncthreads();
        float acc[N];
#pragma unroll
        for (int v = 0; v < N; ++v) acc[v] = 0.0f;
        if (tid < A.pixels) {
            const unsigned long long u = splitmix64(A.seed, s_c0 + (unsigned long long)(s - 1) * A.pixels + tid);
            const int p = (int)(((u >> 32) * (unsigned long long)NP) >> 32);
            TrackPix q;
            track_fetch<false>(P, sM, sb, od, orgb, om, nullptr, a0, a1, p, W, fW1, fH1, fW2, fH2, q);
            track_eval<TRACK_ADAM>(P, kc, sb, q, acc);
        }
        // fixed-order block sum: a shuffle tree per warp, then warps 0, 1, ...
#pragma unroll
        for (int v = 0; v < N; ++v) {
            float x = acc[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) swarp[warp][v] = x;
        }
        __syncthreads();
        if (warp == 0) {
            float sv = 0.0f;
            if (lane < N) {
                sv = swarp[0][lane];
                for (int w = 1; w < kAdamThreads / 32; ++w) sv += swarp[w][lane];
            }
            // lane i < 6: g_i = scale (C^T g')_i + (L xi)_i, then the Adam step
            const int i = lane < 6 ? lane : 0, bi = i / 3, ii = i % 3;
            const double* Cb = s_C + 9 * bi;
            const double g0 = (double)__shfl_sync(0xffffffffu, sv, 3 * bi),
                         g1 = (double)__shfl_sync(0xffffffffu, sv, 3 * bi + 1),
                         g2 = (double)__shfl_sync(0xffffffffu, sv, 3 * bi + 2);
            const double mg = fdot3(Cb[ii], g0, Cb[3 + ii], g1, Cb[6 + ii], g2);
            double lx = 0.0;
            for (int k = 0; k < 6; ++k) lx = fma(s_prec[6 * i + k], s_xi[k], lx);
            const double g = scale * mg + lx;
            b2t *= A.beta2;
            v2 = A.beta2 * v2 + (1.0 - A.beta2) * g * g;
            const double vhat = v2 / (1.0 - b2t), lr = i < 3 ? A.lr_t : A.lr_r;
            const double xn = s_xi[i] - lr * g / (sqrt(vhat) + A.eps);
            __syncwarp();
            if (lane < 6) s_xi[lane] = xn;
        }
        __syncthreads();
    }
    if (warp == 0) {   // the optimum's pose and matrices for the Laplace pass
        double pose[7];
        warp_pose_of(s_xi, s_pq, s_pt, pose);
        warp_mats_rel(pose, s_anchor, dev->rel);
        if (lane < 6) dev->xi[lane] = s_xi[lane];
        if (lane < 7) dev->cur_pose[lane] = pose[lane];
    }
}

}  // namespace

cudaError_t launch_adam(const KParams& P, const float* o_depth, const float* o_rgb, const uint8_t* o_mask,
                        const float4* a0, const float4* a1, DevState* dev, const AdamArgs& A, cudaStream_t s) {
    if (A.pixels < 1 || A.pixels > kAdamThreads || A.steps < 1) return cudaErrorInvalidValue;
    return launch_pdl(k_adam, 1, kAdamThreads, s, P, o_depth, o_rgb, o_mask, a0, a1, dev, A);
}

}  // namespace prism
