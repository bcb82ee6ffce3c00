// track_dev.cuh — device body of the localisation passes (App. E.3,
// Eq. pointtoplanelaplace) and their FP64 finish, shared by the
// single-stream kernel (track.cu) and the batched serving kernels
// (serve_kernels.cu).
//
// One launch = one evaluation at the current pose.  Every thread walks a
// grid-stride set of observed pixels and, for each kept pixel, forms four
// residuals — point-to-plane against the nearest anchor pixel and three
// photometric against the bilinear anchor colour — with their 6-D Jacobians
// in the anchor camera frame, J' = [a_X, y_a x a_X] (a_X: gradient with
// respect to the point in the anchor frame, y_a = R_a^T (R P)).  Sums of
// w J'^T J', w J'^T r (IRLS weights w = 1/(b max(|r|, floor))), J'^T J'/b^2,
// |r|/b and the pixel count are reduced in FP32 within a warp, in FP64
// across warps, and written as one FP64 partial per block.  The last block
// to finish (ticket counter, no waiting) adds the partials in a fixed order
// — the result does not depend on block scheduling — rotates them to the
// world frame (H = T H' T^T, T = diag(R_a, R_a)) and runs the mode's finish:
//   TRACK_GN       one Gauss-Newton step in the prior's tangent coordinates:
//                  (M^T H M + L) dxi = -(M^T g + L xi), M = diag(I, J_l(xi_theta)),
//                  FP64 Cholesky; xi += dxi; pose = retract(xi)            (R15)
//   TRACK_LAPLACE  Sigma = (2 Ht + M^-T L M^-1)^-1 (Sec. 4.1, R16), EMA (App.
//                  F.2, R17), recombination with the velocity conditional
//                  (Sec. 3.3.2, R23) into the new state
//   TRACK_EXPORT   H, g, Ht, cost, count to dev->ne_out
// Integer decisions (validity, nearest pixel, bilinear cell, gates) follow
// the FP32 recipe with explicitly rounded intrinsics.
#pragma once

#include <cuda/atomic>

#include "kernels.h"
#include "linalg64.cuh"
#include "prism_dev.cuh"

namespace prism {

namespace track_detail {

// Threads a block: one block of 512 an SM for the Gauss-Newton and Laplace
// passes (half the partials of two blocks of 256 for the last block to add),
// 256 for the export of the normal equations (50 sums a thread).
template <int MODE>
struct Block {
    static constexpr int threads = MODE == TRACK_EXPORT ? 256 : 512;
    static constexpr int warps = threads / 32;
};
constexpr int kMaxPerLane = 16;   // partials per lane in the last block: grid <= 512
// The cooperative passes' grid barrier polls at most this often (each poll
// an L2 round trip of ~0.5 us: about a second) before it gives up.
constexpr unsigned int kCoopSpinLimit = 1u << 21;

template <int MODE>
struct NV {
    static constexpr int value = MODE == TRACK_GN ? 29 : (MODE == TRACK_LAPLACE ? 23 : (MODE == TRACK_ADAM ? 8 : 50));
};

// offsets into the per-thread accumulator
template <int MODE>
struct Layout {
    static constexpr bool H = MODE == TRACK_GN || MODE == TRACK_EXPORT;
    static constexpr bool G = MODE != TRACK_LAPLACE;
    static constexpr bool HT = MODE == TRACK_LAPLACE || MODE == TRACK_EXPORT;
    static constexpr int oH = 0;
    static constexpr int oG = H ? 21 : 0;
    static constexpr int oHT = oG + (G ? 6 : 0);
    static constexpr int oCost = oHT + (HT ? 21 : 0);
    static constexpr int oCount = oCost + 1;
};

// One residual r with Jacobian J: H += w J J^T, g += w r J, Ht += J J^T / b^2,
// with sw = sqrt(w) (the IRLS weight) and ib = 1 / b (the Laplace scale)
// folded into J first, so that every matrix entry is one FMA; for the
// paper's Adam (TRACK_ADAM) g += sign(r) J / b, the L1 subgradient.
template <int MODE>
__device__ __forceinline__ void accumulate(float* acc, const float J[6], float r, float sw, float ib, float cost) {
    using L = Layout<MODE>;
    float Js[6], Jt[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Js[i] = J[i] * sw;
        Jt[i] = J[i] * ib;
    }
    int e = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j, ++e) {
            if (L::H) acc[L::oH + e] = fmaf(Js[i], Js[j], acc[L::oH + e]);
            if (L::HT) acc[L::oHT + e] = fmaf(Jt[i], Jt[j], acc[L::oHT + e]);
        }
    if constexpr (MODE == TRACK_ADAM) {   // the L1 subgradient sign(r) / b J
        const float sg = r > 0.0f ? ib : (r < 0.0f ? -ib : 0.0f);
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[L::oG + i] = fmaf(sg, J[i], acc[L::oG + i]);
    } else if (L::G) {
        const float swr = sw * r;
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[L::oG + i] = fmaf(swr, Js[i], acc[L::oG + i]);
    }
    acc[L::oCost] += cost;
}

// The FP64 state the finish reads, slot e of the staging array: prec_pp
// 0..35, xi 36..41, anchor 42..48, pq 49..52, pt 53..55; Gauss-Newton also
// the prior's anchor-frame terms Ci 56..73, L' 74..109, m 110..115, and q0
// 116..119, b0 120..122; Laplace also D 56..91, the pose
// block of the previous covariance 92..127, cov_vel 128..163, pv 164..166,
// pw 167..169, and of the final iterate L' 170..205, J_l^-1 206..214 and
// Ra 215..223.  nullptr past the mode's last slot.
template <int MODE>
__device__ __forceinline__ const double* stage_src(const DevState* dev, int e) {
    if (e < 36) return dev->prec_pp + e;
    if (e < 42) return dev->xi + (e - 36);
    if (e < 49) return dev->anchor_pose + (e - 42);
    if (e < 53) return dev->pq + (e - 49);
    if (e < 56) return dev->pt + (e - 53);
    if (MODE == TRACK_GN) {
        if (e < 74) return dev->gn_Ci + (e - 56);
        if (e < 110) return dev->gn_Lp + (e - 74);
        if (e < 116) return dev->gn_m + (e - 110);
        if (e < 120) return dev->gn_q0 + (e - 116);
        if (e < 123) return dev->gn_b0 + (e - 120);
    }
    if (MODE == TRACK_LAPLACE) {
        if (e < 92) return dev->D + (e - 56);
        if (e < 128) return dev->cov + 12 * ((e - 92) / 6) + (e - 92) % 6;
        if (e < 164) return dev->cov_vel + (e - 128);
        if (e < 167) return dev->pv + (e - 164);
        if (e < 170) return dev->pw + (e - 167);
        if (e < 206) return dev->gn_Lp + (e - 170);
        if (e < 215) return dev->gn_Ji + (e - 206);
        if (e < 224) return dev->gn_Ci + (e - 215);
    }
    return nullptr;
}
constexpr int kStage = 224;

// Asynchronous global -> shared copies (no registers held, no stall until
// the wait).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const size_t g = __cvta_generic_to_global(gmem);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Reciprocals of the Laplace scales, computed once per thread.
struct EvalConst {
    float ib_geo, ib_rgb;
};

// A_world = T A' T^T with T = diag(Ra, Ra), one element per thread
__device__ inline void rotate_to_world(const double* Ra, const double* Ap, double* Aw) {
    for (int e = threadIdx.x; e < 36; e += blockDim.x) {
        int i = e / 6, j = e % 6, bi = i / 3, bj = j / 3, ii = i % 3, jj = j % 3;
        double s = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) s = fma(Ra[3 * ii + k] * Ap[6 * (3 * bi + k) + 3 * bj + l], Ra[3 * jj + l], s);
        Aw[e] = s;
    }
}

// One observed pixel between its loads and its residuals.
struct TrackPix {
    float X0, X1, X2, iz, up, vp, aa, cc;
    float4 A, I00, I10, I01, I11;
    float c0, c1, c2;   // observed colour
    int iu, iv;
    bool ok;
};

// Decisions up to the anchor gathers of pixel p, and the gathers themselves,
// issued together (nearest normal/depth and the four bilinear colour taps)
// as soon as the projection is known.  ok = the pixel passed the mask,
// z > 0 and both image-range tests; the remaining gates are in track_eval.
// MASKGEN: the pixel's depth validity is evaluated here (depth_valid) and
// stored to om_out instead of read from om.
template <bool MASKGEN>
__device__ __forceinline__ void track_fetch(const KParams& P, const float* sM, const float* sb,
                                            const float* __restrict__ od, const float* __restrict__ orgb,
                                            const uint8_t* __restrict__ om, uint8_t* __restrict__ om_out,
                                            const float4* __restrict__ a0, const float4* __restrict__ a1, int p,
                                            int W, float fW1, float fH1, float fW2, float fH2, TrackPix& q) {
    bool m;
    if constexpr (MASKGEN) {
        m = depth_valid(P, od, p % W, p / W);
        om_out[p] = (uint8_t)m;
    } else {
        m = om[p] != 0;
    }
    const float z = od[p];
    q.c0 = orgb[3 * p];
    q.c1 = orgb[3 * p + 1];
    q.c2 = orgb[3 * p + 2];
    const int u = p % W, v = p / W;
    // ---- decisions (FP32 recipe) ----
    float Pc[3], X[3];
    backproject_rn(P, u, v, z, Pc);
    affine_rn(sM, sb, Pc, X);
    q.X0 = X[0]; q.X1 = X[1]; q.X2 = X[2];
    q.iz = __fdiv_rn(1.0f, X[2]);
    q.up = __fmaf_rn(__fmul_rn(P.fx32, X[0]), q.iz, P.cx32);
    q.vp = __fmaf_rn(__fmul_rn(P.fy32, X[1]), q.iz, P.cy32);
    const float nu = floorf(__fadd_rn(q.up, 0.5f)), nv = floorf(__fadd_rn(q.vp, 0.5f));
    const float bu = floorf(q.up), bv = floorf(q.vp);
    q.ok = m && X[2] > 0.0f && nu >= 0.0f && nu <= fW1 && nv >= 0.0f && nv <= fH1 && bu >= 0.0f &&
           bu <= fW2 && bv >= 0.0f && bv <= fH2;
    q.iu = q.ok ? (int)nu : 0;
    q.iv = q.ok ? (int)nv : 0;
    q.aa = __fsub_rn(q.up, bu);
    q.cc = __fsub_rn(q.vp, bv);
    if (q.ok) {
        const int b00 = (int)bv * W + (int)bu;
        q.ok = PRISM_IN_RANGE(P, CHK_TRACK_ANCHOR, q.iv * W + q.iu, (long long)W * P.H) &&
               PRISM_IN_RANGE(P, CHK_TRACK_ANCHOR, b00, (long long)W * P.H) &&
               PRISM_IN_RANGE(P, CHK_TRACK_ANCHOR, b00 + W + 1, (long long)W * P.H);
        (void)b00;   // (unused where the checks compile to true)
    }
    if (q.ok) {
        const int b00 = (int)bv * W + (int)bu;
        q.A = a0[q.iv * W + q.iu];
        q.I00 = a1[b00];
        q.I10 = a1[b00 + 1];
        q.I01 = a1[b00 + W];
        q.I11 = a1[b00 + W + 1];
    }
}

// The remaining gates of a fetched pixel (valid anchor depth and colour taps,
// |r_geo|, |r_rgb|) and, if kept, its four residuals and Jacobians into acc.
template <int MODE>
__device__ __forceinline__ void track_eval(const KParams& P, const EvalConst& k, const float* sb, const TrackPix& q,
                                           float* acc) {
    using L = Layout<MODE>;
    if (!q.ok) return;
    const float4 A = q.A, I00 = q.I00, I10 = q.I10, I01 = q.I01, I11 = q.I11;
    if (!(A.w > 0.0f)) return;
    if (!(I00.w > 0.0f && I10.w > 0.0f && I01.w > 0.0f && I11.w > 0.0f)) return;
    const float aa = q.aa, cc = q.cc;
    float ph[3];
    backproject_rn(P, q.iu, q.iv, A.w, ph);
    const float e0 = __fsub_rn(ph[0], q.X0), e1 = __fsub_rn(ph[1], q.X1), e2 = __fsub_rn(ph[2], q.X2);
    const float rgeo = __fmaf_rn(A.x, e0, __fmaf_rn(A.y, e1, __fmul_rn(A.z, e2)));
    if (!(fabsf(rgeo) <= P.gate_geo32)) return;
    float rr[3];
    {
        float t = lerp_rn(I00.x, I10.x, aa), b = lerp_rn(I01.x, I11.x, aa);
        rr[0] = __fsub_rn(lerp_rn(t, b, cc), q.c0);
        t = lerp_rn(I00.y, I10.y, aa); b = lerp_rn(I01.y, I11.y, aa);
        rr[1] = __fsub_rn(lerp_rn(t, b, cc), q.c1);
        t = lerp_rn(I00.z, I10.z, aa); b = lerp_rn(I01.z, I11.z, aa);
        rr[2] = __fsub_rn(lerp_rn(t, b, cc), q.c2);
    }
    if (!(fabsf(rr[0]) <= P.gate_rgb32 && fabsf(rr[1]) <= P.gate_rgb32 && fabsf(rr[2]) <= P.gate_rgb32)) return;
    // ---- values (FP32) ----
    const float ya0 = q.X0 - sb[0], ya1 = q.X1 - sb[1], ya2 = q.X2 - sb[2];
    float J[6];
    {   // point-to-plane: a_X = -n
        const float ax = -A.x, ay = -A.y, az = -A.z;
        J[0] = ax; J[1] = ay; J[2] = az;
        J[3] = fmaf(ya1, az, -(ya2 * ay)); J[4] = fmaf(ya2, ax, -(ya0 * az)); J[5] = fmaf(ya0, ay, -(ya1 * ax));
        const float ar = fabsf(rgeo);
        const float sw = rsqrtf(P.b_geo32 * fmaxf(ar, P.floor_geo32));
        accumulate<MODE>(acc, J, rgeo, sw, k.ib_geo, ar * k.ib_geo);
    }
    const float iz = q.iz, izz = iz * iz;
    const float du0 = P.fx32 * iz, du2 = -P.fx32 * q.X0 * izz;
    const float dv1 = P.fy32 * iz, dv2 = -P.fy32 * q.X1 * izz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float i00 = c == 0 ? I00.x : (c == 1 ? I00.y : I00.z);
        const float i10 = c == 0 ? I10.x : (c == 1 ? I10.y : I10.z);
        const float i01 = c == 0 ? I01.x : (c == 1 ? I01.y : I01.z);
        const float i11 = c == 0 ? I11.x : (c == 1 ? I11.y : I11.z);
        const float gu = fmaf(1.0f - cc, i10 - i00, cc * (i11 - i01));
        const float gv = fmaf(1.0f - aa, i01 - i00, aa * (i11 - i10));
        const float ax = gu * du0, ay = gv * dv1, az = fmaf(gu, du2, gv * dv2);
        J[0] = ax; J[1] = ay; J[2] = az;
        J[3] = fmaf(ya1, az, -(ya2 * ay)); J[4] = fmaf(ya2, ax, -(ya0 * az)); J[5] = fmaf(ya0, ay, -(ya1 * ax));
        const float ar = fabsf(rr[c]);
        const float sw = rsqrtf(P.b_rgb32 * fmaxf(ar, P.floor_rgb32));
        accumulate<MODE>(acc, J, rr[c], sw, k.ib_rgb, ar * k.ib_rgb);
    }
    acc[L::oCount] += 1.0f;
}

}  // namespace track_detail

using namespace track_detail;

// One block's share of one evaluation: virtual block vb of nvb (pixels
// vb * threads + t, stepping by nvb * threads), its partial, the ticket, and — in
// the block that takes the last ticket — the fixed-order sum and the mode's
// finish.  A launch of nvb blocks (vb = vb) and a persistent grid
// that takes the virtual blocks one by one give the same bits.  MASKGEN:
// the observed pixels' depth validity is evaluated from od and written to
// om_out (the pass then needs no mask pass before it).
//
// COOP (Gauss-Newton only): pass `pass` of a cooperative launch whose nvb
// blocks are all resident.  In place of the ticket every block waits at a
// grid barrier (*counter reaching nvb (pass + 1), a bounded spin), sums all
// partials in the same fixed order and runs the same FP64 finish, so every
// block holds the identical next iterate and its matrices in shared memory
// and goes on to the next pass without a launch; block 0 also writes them
// to the device state.  Partials alternate between two buffers by pass.
// Returns false when the launch's passes must stop (a system that is not
// positive definite, or a barrier that timed out; both raise a flag).
template <int MODE, bool MASKGEN = false, bool COOP = false>
__device__ __forceinline__ bool track_item(const KParams& P, const float* __restrict__ od,
                                           const float* __restrict__ orgb, const uint8_t* __restrict__ om,
                                           const float4* __restrict__ a0, const float4* __restrict__ a1,
                                           DevState* dev, float* __restrict__ partials, int pstride,
                                           unsigned int* __restrict__ counter, DevStats* __restrict__ stats,
                                           int vb, int nvb, uint8_t* __restrict__ om_out = nullptr, int pass = 0) {
    static_assert(!COOP || MODE == TRACK_GN, "the cooperative passes are Gauss-Newton passes");
    constexpr int N = NV<MODE>::value;
    constexpr int kThreads = Block<MODE>::threads, kWarps = Block<MODE>::warps;
    using L = Layout<MODE>;
    __shared__ float sM[9], sb[3];
    __shared__ float swarp[kWarps][N];
    __shared__ double S[64];
    __shared__ double sm[8][36];
    __shared__ double sx[8][36];
    __shared__ int s_last, s_ok;
    __shared__ double st[kStage];
    __shared__ int s_nloc, s_flags;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Every block starts copying the state the last block's finish will need
    // (written by earlier kernels), so that it is in shared memory when the
    // last ticket is drawn.  (A cooperative launch's later passes find it,
    // and the pass's matrices, in shared memory from the pass before.)
    if (!COOP || pass == 0) {
        if (tid < kStage) {
            const double* src = stage_src<MODE>(dev, tid);
            if (src) cp_async(&st[tid], src, 8);
        } else if (MODE == TRACK_LAPLACE && tid == kStage) {
            cp_async(&s_nloc, &dev->n_localised, 4);
        } else if (MODE == TRACK_LAPLACE && tid == kStage + 1) {
            cp_async(&s_flags, &dev->flags, 4);
        }
        if (tid < 12) {
            const float* mats = MODE == TRACK_EXPORT ? dev->aux : dev->rel;
            if (tid < 9) sM[tid] = mats[tid];
            else sb[tid - 9] = mats[tid];
        }
    }
    __syncthreads();
    float* const pbuf = COOP ? partials + (size_t)(pass & 1) * N * pstride : partials;

    float acc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = 0.0f;
    const EvalConst kc{1.0f / P.b_geo32, 1.0f / P.b_rgb32};
    const int W = P.W, Hh = P.H, NP = W * Hh;
    const float fW1 = (float)(W - 1), fH1 = (float)(Hh - 1), fW2 = (float)(W - 2), fH2 = (float)(Hh - 2);
    // Two pixels per iteration: both are fetched (all their loads in flight)
    // before either is evaluated; the sums see the pixels in the order of a
    // plain stride loop.
    const int stride = nvb * kThreads;
    for (int p = vb * kThreads + tid; p < NP; p += 2 * stride) {
        TrackPix q0, q1;
        track_fetch<MASKGEN>(P, sM, sb, od, orgb, om, om_out, a0, a1, p, W, fW1, fH1, fW2, fH2, q0);
        const bool two = p + stride < NP;
        if (two) track_fetch<MASKGEN>(P, sM, sb, od, orgb, om, om_out, a0, a1, p + stride, W, fW1, fH1, fW2, fH2, q1);
        else q1.ok = false;
        track_eval<MODE>(P, kc, sb, q0, acc);
        track_eval<MODE>(P, kc, sb, q1, acc);
    }
    cp_async_wait_all();   // this thread's staging copies (visible to the block after the barriers below)

    // ---- block reduction: FP32, in a fixed order (warp reduce-scatter, then warps 0..7) ----
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = c0 + i < N ? acc[c0 + i] : 0.0f;
        warp_reduce_scatter32(v);
        if (c0 + lane < N) swarp[warp][c0 + lane] = v[0];
    }
    __syncthreads();
    if (tid < N) {   // partials are stored value-major: partials[v * pstride + block]
        float s = swarp[0][tid];
        for (int w = 1; w < kWarps; ++w) s += swarp[w][tid];
        if (PRISM_IN_RANGE(P, CHK_TRACK_PARTIAL, vb, pstride)) pbuf[(size_t)tid * pstride + vb] = s;
    }
    __syncthreads();
    if constexpr (COOP) {
        // Grid barrier: the release add publishes this block's partials; the
        // acquire load that sees all nvb arrivals of this pass makes everyone's
        // visible.  Bounded: past the limit the block raises FLAG_SYNC_TIMEOUT
        // and the launch's passes stop (the step is then rejected).
        if (tid == 0) {
            cuda::atomic_ref<unsigned int, cuda::thread_scope_device> bar(*counter);
            bar.fetch_add(1u, cuda::memory_order_release);
            const unsigned int target = (unsigned int)nvb * (unsigned int)(pass + 1);
            unsigned int spins = 0;
            int ok = 1;
            while (bar.load(cuda::memory_order_acquire) < target) {
                if (++spins > kCoopSpinLimit) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            s_last = ok;
        }
        __syncthreads();
        if (!s_last) {
            if (tid == 0) atomicOr(&dev->flags, FLAG_SYNC_TIMEOUT);
            return false;
        }
    } else {
        // Ticket: the acq_rel atomic releases this block's partials (ordered
        // before it by the barrier) and, for the last block, acquires everyone's.
        if (tid == 0) {
            cuda::atomic_ref<unsigned int, cuda::thread_scope_device> ticket(*counter);
            s_last = ticket.fetch_add(1u, cuda::memory_order_acq_rel) == nvb - 1;
        }
        __syncthreads();
        if (!s_last) return true;
    }

    // ---- last block ----
    // The staged FP64 state (st, s_nloc) arrived during the pixel loop: GB300's
    // FP64 pipe has ~64-cycle latency, so the tail is a latency chain and
    // every global round trip on it costs ~600 cycles.
    // Fixed-order sum of the partials: warp w sums rows v = w, w + 8, ...
    // (at most kRows); lane l adds blocks 4l .. 4l + 3, then 4 (l + 32) .., in
    // order, then a fixed shuffle tree; the order never depends on scheduling.
    // All of a warp's (float4) loads are issued before the first add (the
    // loops are fully unrolled; G <= 32 * kMaxPerLane is checked at launch).
    // The sums stay FP32 (a GB300 SM retires about two FP64 adds per clock,
    // so ~9,000 of them would dominate this block's tail; FP32 keeps the
    // sums to ~1e-6 relative, far inside what a Gauss-Newton step or the
    // Laplace covariance needs) and are widened to FP64 for the finish.
    const int G = nvb;
    constexpr int kRows = (N + kWarps - 1) / kWarps;
    constexpr int kQuads = kMaxPerLane / 4;   // float4 loads per row and lane (rows are 16-byte aligned)
    float4 x[kRows][kQuads];
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
        const int v = warp + kWarps * q;
        const float4* row = reinterpret_cast<const float4*>(pbuf + (size_t)(v < N ? v : 0) * pstride);
#pragma unroll
        for (int j = 0; j < kQuads; ++j) {
            const int b = 4 * (lane + 32 * j);
            float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (v < N && b < G) {
                t = __ldcg(row + lane + 32 * j);
                if (b + 1 >= G) t.y = 0.0f;
                if (b + 2 >= G) t.z = 0.0f;
                if (b + 3 >= G) t.w = 0.0f;
            }
            x[q][j] = t;
        }
    }
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < kQuads; ++j) s = (((s + x[q][j].x) + x[q][j].y) + x[q][j].z) + x[q][j].w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int v = warp + kWarps * q;
        if (lane == 0 && v < N) S[v] = (double)s;
    }
    __syncthreads();
    if (tid == 0 && !COOP) *counter = 0u;
    // the first Gauss-Newton pass of a localisation (the one that evaluates the
    // depth validity) also clears counter[1], the barrier of the cooperative
    // launch of the passes that follow it (launch_track_coop)
    if (tid == 0 && MODE == TRACK_GN && MASKGEN && !COOP) counter[1] = 0u;
    if (tid == 0 && (!COOP || vb == 0) && stats) atomicAdd(&stats->track_pixels, (unsigned long long)S[L::oCount]);

    // sm[0]: Ra; sm[1]: H' (sym); sm[2]: Ht' (sym); sm[3], sm[4]: world-frame H, Ht
    double* Ra = sm[0];
    if (MODE == TRACK_EXPORT && tid < 32) {   // the anchor rotation, one entry a lane
        const double* qa = st + 45;
        const double re = quat_R_entry_rn(qa[0], qa[1], qa[2], qa[3], tid < 9 ? tid : 0);
        if (tid < 9) Ra[tid] = re;
    }
    if (MODE == TRACK_EXPORT && L::H && tid >= 32 && tid < 53) {   // unpack the upper triangles in parallel
        const int e = tid - 32;
        int i = 0, r = e;
        while (r >= 6 - i) { r -= 6 - i; ++i; }
        const int j = i + r;
        sm[1][6 * i + j] = sm[1][6 * j + i] = S[L::oH + e];
    }
    if (MODE == TRACK_EXPORT && L::HT && tid >= 64 && tid < 85) {
        const int e = tid - 64;
        int i = 0, r = e;
        while (r >= 6 - i) { r -= 6 - i; ++i; }
        const int j = i + r;
        sm[2][6 * i + j] = sm[2][6 * j + i] = S[L::oHT + e];
    }
    if (MODE == TRACK_EXPORT) __syncthreads();   // (the Gauss-Newton and Laplace finishes read S directly)
    double* Hw = sm[3];
    double* Htw = sm[4];
    if (MODE == TRACK_EXPORT) {
        if (L::H) rotate_to_world(Ra, sm[1], Hw);
        if (L::HT) rotate_to_world(Ra, sm[2], Htw);
        __syncthreads();
    }

    if (MODE == TRACK_EXPORT) {
        if (tid < 36) {
            dev->ne_out[tid] = Hw[tid];
            dev->ne_out[42 + tid] = Htw[tid];
        }
        if (tid < 2) {
            double gw[3];
            const double* gp = S + L::oG + 3 * tid;
            mat3vec(Ra, gp, gw);
            for (int a = 0; a < 3; ++a) dev->ne_out[36 + 3 * tid + a] = gw[a];
        }
        if (tid == 0) {
            dev->ne_out[78] = S[L::oCost];
            dev->ne_out[79] = S[L::oCount];
        }
        return true;
    }

    if (MODE == TRACK_GN) {
        // In the anchor frame J' = J T^T... the tangent step dxi maps to the
        // anchor-frame perturbation through C = T M = diag(Ra^T, Ra^T J_l(xi_theta)),
        // so the step solves (C^T H' C + L) dxi = -(C^T g' + L xi).  In y = C dxi
        // this is (H' + L') y = -(g' + m) with L' = Ci^T L Ci, m = Ci^T L xi and
        // Ci = C^-1 = diag(Ra, J_l^-1 Ra), and dxi = Ci y (warp_gn_prior_terms):
        // the sums enter the FP64 solve with one addition each.  Ci, L' and m of
        // the current iterate were prepared by the previous pass's finish (or
        // with the start matrices before the first pass), off this pass's
        // critical path.
        const double* Ci = st + 56;   // 3x3 blocks: Ra, J_l^-1 Ra
        const double* Lp = st + 74;
        const double* mv = st + 110;
        double* xn = sx[4];
        __shared__ int s_pd;
        if (warp == 0) {
            // lane e < 21: entry (li, lm) of the lower triangle of H' + L'; lane
            // 21 + li: -(g' + m)_li (the layout of warp_ldlt6_solve).  H' is stored
            // as its upper triangle, row-major: (r, c), r <= c, at 5 r - r (r - 1) / 2 + c.
            int li = 0, lm = 0;
            if (lane < 21) {
#pragma unroll
                for (int i = 1; i < 6; ++i)
                    if (lane >= tri6(i, 0)) li = i;
                lm = lane - tri6(li, 0);
            }
            const bool rhs = lane >= 21 && lane < 27;
            const int ri = rhs ? lane - 21 : 0;
            // one addition for every lane (operands selected by index), the
            // right-hand side negated by a select
            const double s0 = S[rhs ? L::oG + ri : L::oH + 5 * lm - lm * (lm - 1) / 2 + li];
            const double s1 = rhs ? mv[ri] : Lp[6 * li + lm];
            const double sum = s0 + s1;
            const double a = sel64(rhs, -sum, sum);
            bool pd;
            const double y = warp_ldlt6_solve(a, &pd);
            // dxi = Ci y on lanes 21..26: row ri of block bi of Ci against y's block bi
            const int bi = ri / 3, ii = ri % 3;
            const double y0 = __shfl_sync(0xffffffffu, y, 21 + 3 * bi), y1 = __shfl_sync(0xffffffffu, y, 22 + 3 * bi),
                         y2 = __shfl_sync(0xffffffffu, y, 23 + 3 * bi);
            const double* Cb = Ci + 9 * bi;
            const double dx = fdot3(Cb[3 * ii], y0, Cb[3 * ii + 1], y1, Cb[3 * ii + 2], y2);
            if (pd && rhs) xn[ri] = st[36 + ri] + dx;
            if (lane == 0) s_pd = pd;
        }
        __syncthreads();
        if (!s_pd) {
            if (tid == 0 && (!COOP || vb == 0)) atomicOr(&dev->flags, FLAG_GN_NOTPD);
            return false;
        }
        // where the next pass's terms go: the device state, or (COOP) this
        // block's shared copies, which block 0 also writes to the device
        const bool to_dev = !COOP || vb == 0;
        if (warp == 0) {
            // The FP32 pose -> anchor matrices of the next pass, straight from
            // xi (the critical path): Ra^T Exp(xi_theta) R_prior = Exp(w) A0 with
            // w = Ra^T xi_theta and A0 = Ra^T R_prior = R(q0), so
            // M = R(quat_exp(w) (x) q0) (unit to rounding) and b = b0 + Ra^T xi_t.
            // Lanes 0..2: w; lane 3: |xi_theta|^2; lanes 9..11: Ra^T xi_t.
            const bool tl = lane >= 9 && lane < 12;
            const int r = lane < 3 ? lane : (tl ? lane - 9 : 0);
            const bool sq = lane == 3;
            const double* v = tl ? xn : xn + 3;
            const double d = fdot3(sq ? v[0] : Ci[r], v[0], sq ? v[1] : Ci[3 + r], v[1],
                                   sq ? v[2] : Ci[6 + r], v[2]);
            const double w[3] = {__shfl_sync(0xffffffffu, d, 0), __shfl_sync(0xffffffffu, d, 1),
                                 __shfl_sync(0xffffffffu, d, 2)};
            const double th2 = __shfl_sync(0xffffffffu, d, 3);
            const double qr = warp_quat_mul_component(warp_quat_exp_component(w, th2), st + 116);
            const double q0 = __shfl_sync(0xffffffffu, qr, 0), q1 = __shfl_sync(0xffffffffu, qr, 1),
                         q2 = __shfl_sync(0xffffffffu, qr, 2), q3 = __shfl_sync(0xffffffffu, qr, 3);
            const double me = quat_R_entry_rn(q0, q1, q2, q3, lane < 9 ? lane : 0);
            const double be = st[120 + r] + d;
            if (COOP) {
                if (lane < 9) sM[lane] = (float)me;
                else if (tl) sb[lane - 9] = (float)be;
            }
            if (to_dev) {
                if (lane < 9) dev->rel[lane] = (float)me;
                else if (tl) dev->rel[lane] = (float)be;
            }
        } else if (warp == 1) {   // the FP64 pose of the new iterate (the state mean after the last pass)
            const double qn = warp_quat_exp_mul_unit(xn + 3, st + 49);
            if (to_dev) {
                if (lane < 4) dev->cur_pose[3 + lane] = qn;
                if (lane < 3) dev->cur_pose[lane] = st[53 + lane] + xn[lane];
                if (lane < 6) dev->xi[lane] = xn[lane];
            }
            if (COOP && lane < 6) st[36 + lane] = xn[lane];
        } else if (warp == 2) {   // meanwhile: the prior's anchor-frame terms of the new iterate
            if (!COOP) {
                warp_gn_prior_terms(Ci, st, xn, dev->gn_Ci + 9, dev->gn_Lp, dev->gn_m, dev->gn_Ji, &sm[2][0]);
            } else {   // into the staged slots (Ci's second block, L', m), J_l^-1 beside them
                double* ji = &sm[5][0];   // (the scratch takes sm[2] and part of sm[3])
                warp_gn_prior_terms(Ci, st, xn, st + 65, st + 74, st + 110, ji, &sm[2][0]);
                __syncwarp();
                if (to_dev) {
                    for (int e = lane; e < 60; e += 32) {
                        if (e < 9) dev->gn_Ci[9 + e] = st[65 + e];
                        else if (e < 45) dev->gn_Lp[e - 9] = st[74 + e - 9];
                        else if (e < 51) dev->gn_m[e - 45] = st[110 + e - 45];
                        else dev->gn_Ji[e - 51] = ji[e - 51];
                    }
                }
            }
        }
        if (COOP) __syncthreads();   // the next pass reads the new terms and matrices
        return true;
    }

    // MODE == TRACK_LAPLACE.  Divergence guard: a flag raised by this step's
    // prediction (prior not positive definite) or by a Gauss-Newton pass
    // rejects the step; the posterior stays as it was and the map update
    // that follows lists no tile.
    if (s_flags != 0) {
        if (tid == 0) {
            dev->rejected = 1;
            dev->ne_out[78] = S[L::oCost];
            dev->ne_out[79] = S[L::oCount];
        }
        return true;
    }
    // Sigma = (2 Ht + Mi^T L Mi)^-1 in world-frame perturbations, Mi =
    // diag(I, J_l(xi_theta)^-1).  With Ht = T Ht' T^T (T = diag(Ra, Ra), Ht' the
    // anchor-frame sum) and Mi^T L Mi = T L' T^T (L' = Ci^T L Ci of the final
    // iterate, warp_gn_prior_terms), Sigma = T (2 Ht' + L')^-1 T^T: the sums
    // enter the FP64 inverse with one FMA each, and the inverse is rotated once.
    const double* Lp = st + 170;
    const double* Ji = st + 206;
    const double* Rs = st + 215;   // Ra of the anchor
    double* Sa = sx[0];   // (2 Ht' + L')^-1
    double* U = sx[1];    // Sa T^T
    double* Sp = sx[4];   // pose covariance after the EMA
    double* Dp = sx[5];   // D' = D Mi
    double* DS = sx[6];   // D' Sp
    double* mats = sx[7]; // the new mean's FP32 matrices (c2w, w2c), as doubles
    double vel = 0.0;
    if (warp == 0) {
        // lane e < 21: entry (li, lm) of the lower triangle of 2 Ht' + L' (Ht' as its
        // upper triangle, row-major: (r, c), r <= c, at 5 r - r (r - 1) / 2 + c)
        int li = 0, lm = 0;
        if (lane < 21) {
#pragma unroll
            for (int i = 1; i < 6; ++i)
                if (lane >= tri6(i, 0)) li = i;
            lm = lane - tri6(li, 0);
        }
        const double a = fma(2.0, S[L::oHT + 5 * lm - lm * (lm - 1) / 2 + li], Lp[6 * li + lm]);
        bool pd;
        double x[6];
        warp_spd6_inverse(a, &pd, x);
        if (lane < 6)
#pragma unroll
            for (int k = 0; k < 6; ++k) Sa[6 * k + lane] = x[k];
        if (lane == 0) s_ok = pd;
    } else if (warp == 1) {   // meanwhile: D' = D Mi (D' = D on the translation columns)
#pragma unroll
        for (int round = 0; round < 2; ++round) {
            const int e = lane + 32 * round;
            const int i = e < 36 ? e / 6 : 0, j = e < 36 ? e % 6 : 3, jj = j < 3 ? 0 : j - 3;
            const double* Dr = st + 56 + 6 * i;
            const double v = fdot3(Dr[3], Ji[jj], Dr[4], Ji[3 + jj], Dr[5], Ji[6 + jj]);
            if (e < 36) Dp[e] = sel64(j < 3, Dr[j < 3 ? j : 0], v);
        }
    } else if (warp == 2 && lane < 6) {   // v = vbar + D xi
        double dv = 0.0;
        for (int k = 0; k < 6; ++k) dv = fma(st[56 + 6 * lane + k], st[36 + k], dv);
        vel = (lane < 3 ? st[164 + lane] : st[167 + lane - 3]) + dv;
    } else if (warp == 3) {   // the new mean's FP32 matrices
        double pose[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) pose[i] = dev->cur_pose[i];
        warp_mats_c2w(pose, (float*)&mats[0]);    // 12 floats in mats[0..5]
        warp_mats_w2c(pose, (float*)&mats[6]);    // 12 floats in mats[6..11]
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) {
            dev->flags |= FLAG_LAPLACE_NOTPD;
            dev->rejected = 1;
            dev->ne_out[78] = S[L::oCost];
            dev->ne_out[79] = S[L::oCount];
        }
        return true;
    }
    if (tid < 36) {   // U = Sa T^T: U[r][j] = sum_l Sa[r][3 bj + l] Ra[jj][l]
        const int r = tid / 6, j = tid % 6, bj = j / 3, jj = j % 3;
        U[tid] = fdot3(Sa[6 * r + 3 * bj], Rs[3 * jj], Sa[6 * r + 3 * bj + 1], Rs[3 * jj + 1], Sa[6 * r + 3 * bj + 2],
                       Rs[3 * jj + 2]);
    }
    __syncthreads();
    const bool first = s_nloc == 0;
    if (tid < 36) {   // the Laplace covariance T U, then the EMA (App. F.2)
        const int i = tid / 6, j = tid % 6, bi = i / 3, ii = i % 3;
        const double sl = fdot3(Rs[3 * ii], U[6 * (3 * bi) + j], Rs[3 * ii + 1], U[6 * (3 * bi + 1) + j], Rs[3 * ii + 2],
                                U[6 * (3 * bi + 2) + j]);
        Sp[tid] = first ? sl : fma(P.ema, st[92 + tid], (1.0 - P.ema) * sl);
    }
    __syncthreads();
    if (tid < 36) {   // DS = D' Sp
        const int i = tid / 6, j = tid % 6;
        double a = 0.0;
        for (int k = 0; k < 6; ++k) a = fma(Dp[6 * i + k], Sp[6 * k + j], a);
        DS[tid] = a;
    }
    __syncthreads();
    if (tid < 144) {   // cov = [[Sp, Sp D'^T], [D' Sp, D' Sp D'^T + S_vel]]
        const int i = tid / 12, j = tid % 12;
        double c;
        if (i < 6 && j < 6) {
            c = 0.5 * (Sp[6 * i + j] + Sp[6 * j + i]);
        } else if (i >= 6 && j < 6) {
            c = DS[6 * (i - 6) + j];
        } else if (i < 6 && j >= 6) {
            c = DS[6 * (j - 6) + i];
        } else {
            const int a = i - 6, b = j - 6;
            double s1 = 0.0, s2 = 0.0;
            for (int k = 0; k < 6; ++k) {
                s1 = fma(DS[6 * a + k], Dp[6 * b + k], s1);
                s2 = fma(DS[6 * b + k], Dp[6 * a + k], s2);
            }
            c = 0.5 * (s1 + s2) + 0.5 * (st[128 + 6 * a + b] + st[128 + 6 * b + a]);
        }
        dev->cov[tid] = c;
    }
    if (warp == 2 && lane < 6) {
        if (lane < 3) dev->v[lane] = vel;
        else dev->w[lane - 3] = vel;
    } else if (warp == 5) {   // the new mean, its FP32 matrices, the count
        const float* m32 = (const float*)mats;
        if (lane < 12) {
            dev->c2w[lane] = m32[lane];
            dev->w2c[lane] = m32[12 + lane];
        }
        if (lane < 3) dev->t[lane] = dev->cur_pose[lane];
        if (lane < 4) dev->q[lane] = dev->cur_pose[3 + lane];
        if (lane == 0) {
            dev->n_localised += 1;
            dev->rejected = 0;
            dev->ne_out[78] = S[L::oCost];
            dev->ne_out[79] = S[L::oCount];
        }
    }
    return true;
}

}  // namespace prism
