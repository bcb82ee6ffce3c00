// linalg64.cuh — small FP64 linear algebra for the state kernels (6x6 and
// 12x12 matrices, row-major), run by one thread or spread over a block.
// Multiply-adds are written as fma (the library is compiled without
// implicit contraction), so each result is the same in every kernel.
#pragma once

#include <cuda_runtime.h>

namespace prism {

// a0 b0 + a1 b1 + a2 b2 as fma(a0, b0, fma(a1, b1, a2 b2))
__device__ __forceinline__ double fdot3(double a0, double b0, double a1, double b1, double a2, double b2) {
    return fma(a0, b0, fma(a1, b1, a2 * b2));
}

// c ? x : y as one predicated select (PTX selp.f64).  Both operands are
// computed by every lane, so that a lane-dependent choice does not split a
// warp into groups that each issue the FP64 instructions feeding it (each
// issue costs ~64 cycles on GB300's FP64 pipe, whatever lanes are active).
__device__ __forceinline__ double sel64(bool c, double x, double y) {
    double r;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %3, 0;\n\tselp.f64 %0, %1, %2, p;\n\t}"
        : "=d"(r) : "d"(x), "d"(y), "r"((int)c));
    return r;
}

__device__ inline void mat3vec(const double* A, const double* x, double* y) {
    for (int i = 0; i < 3; ++i) y[i] = fdot3(A[3 * i], x[0], A[3 * i + 1], x[1], A[3 * i + 2], x[2]);
}

// Coefficients of Exp and J_l as functions of th^2.  For th < 1/4 they are
// the Taylor series of sin(th)/th, (1 - cos th)/th^2 and (th - sin th)/th^3
// (truncation below 1e-17 there), avoiding FP64 sin/cos on the short
// dependent chains of the filter; larger angles use sin/cos.
__device__ inline void so3_coeffs(double th2, double& a, double& b, double& c) {
    if (th2 < 0.0625) {
        const double x = th2;
        a = fma(x, fma(x, fma(x, fma(x, fma(x, -1.0 / 39916800, 1.0 / 362880), -1.0 / 5040), 1.0 / 120), -1.0 / 6), 1.0);
        b = fma(x, fma(x, fma(x, fma(x, fma(x, -1.0 / 479001600, 1.0 / 3628800), -1.0 / 40320), 1.0 / 720), -1.0 / 24),
                0.5);
        c = fma(x, fma(x, fma(x, fma(x, fma(x, -1.0 / 6227020800.0, 1.0 / 39916800), -1.0 / 362880), 1.0 / 5040),
                       -1.0 / 120),
                1.0 / 6);
    } else {
        const double th = sqrt(th2), sn = sin(th), cs = cos(th);
        a = sn / th;
        b = (1.0 - cs) / th2;
        c = (th - sn) / (th2 * th);
    }
}

// Entries (i, j) of K = [w]_x and of K^2 = w w^T - |w|^2 I, by selection
// (no indexed local array), for the lane-parallel Jacobians below.
__device__ __forceinline__ double skew_entry(const double w[3], int i, int j) {
    // K_ij = 0 on the diagonal, -w_k for j = i + 1 (mod 3), +w_k for j = i + 2, k = 3 - i - j
    const int k = 3 - i - j;
    const double wk = k == 0 ? w[0] : (k == 1 ? w[1] : w[2]);
    return i == j ? 0.0 : (j == (i + 1) % 3 ? -wk : wk);
}
__device__ __forceinline__ double skew2_entry(const double w[3], double th2, int i, int j) {
    const double wi = i == 0 ? w[0] : (i == 1 ? w[1] : w[2]);
    const double wj = j == 0 ? w[0] : (j == 1 ? w[1] : w[2]);
    return i == j ? fma(wi, wj, -th2) : wi * wj;
}

// Entry (i, j) of Exp(w) = I + a K + b K^2 (exp = true) or of J_l(w) =
// I + b K + c K^2 (exp = false), K = [w]_x: one branch-free expression, so
// that the lanes of a warp can evaluate entries of both.
__device__ __forceinline__ double so3_exp_jl_entry(const double w[3], bool exp, int i, int j) {
    double a, b, c;
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    so3_coeffs(th2, a, b, c);
    const double s1 = exp ? a : b, s2 = exp ? b : c;
    return fma(s1, skew_entry(w, i, j), fma(s2, skew2_entry(w, th2, i, j), i == j ? 1.0 : 0.0));
}

// Entry (i, j) of J_l(w) = I + b K + c K^2, K = [w]_x (the same operations
// whichever thread or kernel evaluates it).
__device__ inline double so3_jl_entry(const double w[3], int i, int j) {
    double a, b, c;
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    so3_coeffs(th2, a, b, c);
    return fma(b, skew_entry(w, i, j), fma(c, skew2_entry(w, th2, i, j), i == j ? 1.0 : 0.0));
}

// Entry (i, j) of the inverse left Jacobian of SO(3), I - K/2 + c K^2 with
// c = 1/th^2 - (1 + cos th) / (2 th sin th); for th < 1/4 its Taylor series
// 1/12 + th^2/720 + th^4/30240 + th^6/1209600 + th^8/47900160 (the same
// operations in every lane).
__device__ inline double so3_jl_inv_entry(const double w[3], int i, int j) {
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    double c;
    if (th2 < 0.0625) {
        c = fma(th2, fma(th2, fma(th2, fma(th2, 1.0 / 47900160, 1.0 / 1209600), 1.0 / 30240), 1.0 / 720), 1.0 / 12);
    } else {
        const double th = sqrt(th2);
        c = 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
    }
    return fma(-0.5, skew_entry(w, i, j), fma(c, skew2_entry(w, th2, i, j), i == j ? 1.0 : 0.0));
}

// Unit quaternion of Exp(w): (cos(th/2), sin(th/2)/th w), with the half-angle
// coefficients from so3_coeffs' series at th/2.
__device__ inline void quat_exp(const double w[3], double q[4]) {
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    double ch, sh;
    if (th2 < 0.25) {   // x = (th/2)^2 < 1/16
        const double x = 0.25 * th2;
        ch = fma(x, fma(x, fma(x, fma(x, fma(x, -1.0 / 3628800, 1.0 / 40320), -1.0 / 720), 1.0 / 24), -0.5), 1.0);
        sh = 0.5 * fma(x, fma(x, fma(x, fma(x, fma(x, -1.0 / 39916800, 1.0 / 362880), -1.0 / 5040), 1.0 / 120),
                              -1.0 / 6),
                       1.0);
    } else {
        const double th = sqrt(th2);
        ch = cos(0.5 * th);
        sh = sin(0.5 * th) / th;
    }
    q[0] = ch; q[1] = sh * w[0]; q[2] = sh * w[1]; q[3] = sh * w[2];
}

// Hamilton product a (x) b (w first).
__device__ inline void quat_mul(const double* a, const double* b, double* q) {
    q[0] = fma(a[0], b[0], -fma(a[1], b[1], fma(a[2], b[2], a[3] * b[3])));
    q[1] = fma(a[0], b[1], fma(a[1], b[0], fma(a[2], b[3], -(a[3] * b[2]))));
    q[2] = fma(a[0], b[2], fma(-a[1], b[3], fma(a[2], b[0], a[3] * b[1])));
    q[3] = fma(a[0], b[3], fma(a[1], b[2], fma(-a[2], b[1], a[3] * b[0])));
}

// Normalised, with w >= 0.
__device__ inline void quat_normalise(double* q) {
    double r = rsqrt(fma(q[0], q[0], fdot3(q[1], q[1], q[2], q[2], q[3], q[3])));
    if (q[0] < 0.0) r = -r;
    for (int i = 0; i < 4; ++i) q[i] *= r;
}

// Component c = lane & 3 of quat_exp(w) (the operations of quat_exp), with
// th2 = |w|^2 given; every lane of the warp must call it.
__device__ __forceinline__ double warp_quat_exp_component(const double w[3], double th2) {
    const int c = (threadIdx.x & 31) & 3;
    const double w0 = w[0], w1 = w[1], w2 = w[2];
    double qe;
    if (th2 < 0.25) {   // the half-angle series of quat_exp: ch (lane c = 0), sh (c > 0)
        const double x = 0.25 * th2;
        const bool c0 = c == 0;
        const double p = fma(x, fma(x, fma(x, fma(x, fma(x, c0 ? -1.0 / 3628800 : -1.0 / 39916800,
                                                         c0 ? 1.0 / 40320 : 1.0 / 362880),
                                                  c0 ? -1.0 / 720 : -1.0 / 5040),
                                           c0 ? 1.0 / 24 : 1.0 / 120),
                                    c0 ? -0.5 : -1.0 / 6),
                             1.0);
        const double sh = 0.5 * p;
        qe = sel64(c0, p, sh * (c == 1 ? w0 : (c == 2 ? w1 : w2)));
    } else {
        double q4[4];
        quat_exp(w, q4);
        qe = c == 0 ? q4[0] : (c == 1 ? q4[1] : (c == 2 ? q4[2] : q4[3]));
    }
    return qe;
}

// Component c = lane & 3 of the Hamilton product a (x) q (the operations of
// quat_mul), a given by component in lanes 0..3 (`ac` on lane c); every lane
// of the warp must call it.
__device__ __forceinline__ double warp_quat_mul_component(double ac, const double* q) {
    const int c = (threadIdx.x & 31) & 3;
    const double a0 = __shfl_sync(0xffffffffu, ac, 0), a1 = __shfl_sync(0xffffffffu, ac, 1),
                 a2 = __shfl_sync(0xffffffffu, ac, 2), a3 = __shfl_sync(0xffffffffu, ac, 3);
    const int p0 = c, p1 = c ^ 1, p2 = c ^ 2, p3 = c ^ 3;
    const double t3 = a3 * q[p3];
    return fma(a0, q[p0], fma(sel64(c == 0 || c == 2, -a1, a1), q[p1],
                              fma(sel64(c == 0 || c == 3, -a2, a2), q[p2], sel64(c == 0 || c == 1, -t3, t3))));
}

// normalise(quat_exp(w) (x) q) with w >= 0 (the operations of quat_exp,
// quat_mul and quat_normalise), computed by the 32 lanes of one warp with
// quaternion component c = lane & 3 in lane c; returns that component.
__device__ __forceinline__ double warp_quat_exp_mul(const double w[3], const double* q) {
    const int c = (threadIdx.x & 31) & 3;
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    const double qm = warp_quat_mul_component(warp_quat_exp_component(w, th2), q);
    // normalised, w >= 0 (quat_normalise)
    const double n0 = __shfl_sync(0xffffffffu, qm, 0), n1 = __shfl_sync(0xffffffffu, qm, 1),
                 n2 = __shfl_sync(0xffffffffu, qm, 2), n3 = __shfl_sync(0xffffffffu, qm, 3);
    double rn = rsqrt(fma(n0, n0, fdot3(n1, n1, n2, n2, n3, n3)));
    if (n0 < 0.0) rn = -rn;
    return (c == 0 ? n0 : (c == 1 ? n1 : (c == 2 ? n2 : n3))) * rn;
}

// normalise(quat_exp(w) (x) q) for a unit q, the normalisation by the
// first-order term of 1 / sqrt(n) around n = 1: with both factors unit to
// rounding, n = |qe (x) q|^2 = 1 + delta, |delta| ~ 1e-15, and
// 1 / sqrt(1 + delta) = 1 - delta / 2 + O(delta^2) is 1.5 - 0.5 n to FP64
// rounding (one FMA in place of the reciprocal square root's chain); w >= 0
// as in warp_quat_exp_mul.  Every lane of the warp must call it.
__device__ __forceinline__ double warp_quat_exp_mul_unit(const double w[3], const double* q) {
    const int c = (threadIdx.x & 31) & 3;
    const double th2 = fdot3(w[0], w[0], w[1], w[1], w[2], w[2]);
    const double qm = warp_quat_mul_component(warp_quat_exp_component(w, th2), q);
    const double n0 = __shfl_sync(0xffffffffu, qm, 0), n1 = __shfl_sync(0xffffffffu, qm, 1),
                 n2 = __shfl_sync(0xffffffffu, qm, 2), n3 = __shfl_sync(0xffffffffu, qm, 3);
    double rn = fma(-0.5, fma(n0, n0, fdot3(n1, n1, n2, n2, n3, n3)), 1.5);
    if (n0 < 0.0) rn = -rn;
    return (c == 0 ? n0 : (c == 1 ? n1 : (c == 2 ? n2 : n3))) * rn;
}

__device__ inline void mat3inv(const double* A, double* B) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    B[0] = c00 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

// Unit quaternion (w >= 0) of a rotation matrix (Shepperd's method).
__device__ inline void R_to_quat(const double* R, double* q) {
    double tr = R[0] + R[4] + R[8], s;
    if (tr > 0.0) {
        s = 2.0 * sqrt(tr + 1.0);
        q[0] = 0.25 * s; q[1] = (R[7] - R[5]) / s; q[2] = (R[2] - R[6]) / s; q[3] = (R[3] - R[1]) / s;
    } else if (R[0] > R[4] && R[0] > R[8]) {
        s = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);
        q[0] = (R[7] - R[5]) / s; q[1] = 0.25 * s; q[2] = (R[1] + R[3]) / s; q[3] = (R[2] + R[6]) / s;
    } else if (R[4] > R[8]) {
        s = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);
        q[0] = (R[2] - R[6]) / s; q[1] = (R[1] + R[3]) / s; q[2] = 0.25 * s; q[3] = (R[5] + R[7]) / s;
    } else {
        s = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);
        q[0] = (R[3] - R[1]) / s; q[1] = (R[2] + R[6]) / s; q[2] = (R[5] + R[7]) / s; q[3] = 0.25 * s;
    }
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double sg = q[0] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < 4; ++i) q[i] = sg * q[i] / n;
}

// Rotation of a unit quaternion (value path; not the decision recipe).

// ------------------------------------------------ one-warp FP64 6x6 solve
// GB300's FP64 pipe retires about one warp instruction per 64 cycles per SM
// sub-partition, so a short FP64 chain costs its instruction count.  The
// two functions below keep that count low: a reciprocal whose seed comes
// from the FP32 unit, and a factorisation that needs one reciprocal per
// column and two FP64 instructions per column for all entries at once.

// Packed lower-triangle position of entry (i, j), i >= j, of a 6x6 matrix.
__host__ __device__ constexpr int tri6(int i, int j) { return i * (i + 1) / 2 + j; }

// True iff d is a positive, finite, normal double whose exponent leaves
// room for rcp64 (2^-1022 <= d < 2^1022), tested on its bits.
__device__ __forceinline__ bool pivot_ok(double d) {
    const int hi = __double2hiint(d);
    const int e = (hi >> 20) & 0x7ff;
    return hi >= 0 && e >= 1 && e <= 2044;
}

// 1/d for d with pivot_ok(d): a seed y with relative error e = 1 - d y, then
// one step of the third-order iteration y' = y (1 + e + e^2), the geometric
// series of 1/d = y / (1 - e) cut after e^2, whose relative error is e^3.
// The seed is the single-precision approximate reciprocal (PTX
// rcp.approx.ftz.f32, relative error about 2^-23) of d's mantissa cut to 20
// bits, rescaled by the exponent with integer operations: |e| below
// 2^-19.5, so the step leaves 2^-58.5 (about 0.02 unit in the last place)
// under the final rounding: a result within one unit in the last place of
// 1/d.  Only the step's three dependent FMAs use the FP64 pipe.
__device__ __forceinline__ double rcp64(double d) {
    const int hi = __double2hiint(d);
    const int e = (hi >> 20) & 0x7ff;
    const float m = __int_as_float(0x3f800000 | ((hi & 0xfffff) << 3));   // mantissa in [1, 2)
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));                // in (0.5, 1]
    const int rb = __float_as_int(r);
    const int ye = ((rb >> 23) & 0xff) - 127 + 2046 - e;                 // biased exponent of r 2^(1023 - e)
    const double y0 = __hiloint2double((ye << 20) | ((rb & 0x7fffff) >> 3), (rb & 7) << 29);
    const double er = fma(-d, y0, 1.0);
    return fma(y0, fma(er, er, er), y0);
}

// Solves A x = b for a 6x6 symmetric positive definite A on one warp by the
// square-root-free Cholesky factorisation A = L D L^T (L unit lower
// triangular, D diagonal).  Lane e < 21 brings entry (i, j), e = tri6(i, j),
// of A's lower triangle in `a`; lane 21 + i brings b_i.  Column j: the
// pivot d_j = a_jj, l_ij = a_ij / d_j below it, and every trailing entry and
// right-hand side row i > j takes a_im -= (a_ij a_mj) / d_j (b_i -= (a_ij
// b_j) / d_j: the forward substitution with L rides along; the product is
// formed while the pivot's reciprocal is computed, so that one FMA follows
// the reciprocal on the chain from pivot to pivot); then z = D^-1 y and the
// back substitution with L^T.  Returns x_i in lane 21 + i (other lanes: junk);
// *pd: every pivot passed pivot_ok (the same on every lane).  All 32 lanes
// must call it.
__device__ __forceinline__ double warp_ldlt6_solve(double a, bool* pd) {
    const int lane = threadIdx.x & 31;
    const bool rhs = lane >= 21 && lane < 27;
    // this lane's row li and column lm (6: the right-hand side)
    int li = 0, lm = 0;
    if (lane < 21) {
#pragma unroll
        for (int i = 1; i < 6; ++i)
            if (lane >= tri6(i, 0)) li = i;
        lm = lane - tri6(li, 0);
    } else if (rhs) {
        li = lane - 21;
        lm = 6;
    } else {
        li = 5;
        lm = 6;
    }
    bool ok = true;
    double rown = 0.0;   // 1 / d_li, for this lane's row
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = __shfl_sync(0xffffffffu, a, tri6(j, j));
        ok = ok && pivot_ok(d);
        const double rj = rcp64(d);
        rown = sel64(li == j, rj, rown);
        const bool below = li > j;                             // rows that column j updates
        const double aij = __shfl_sync(0xffffffffu, a, below ? tri6(li, j) : 0);
        const int src_m = lm == 6 ? 21 + j : (lm > j ? tri6(lm, j) : 0);
        const double amj = __shfl_sync(0xffffffffu, a, src_m);
        const double lij = aij * rj;
        const double upd = fma(-(aij * amj), rj, a);
        // the factor L_ij, kept for the back substitution; a trailing entry
        // (lm <= li) or a right-hand side (lm = 6)
        a = sel64(below && lm == j, lij, sel64(below && lm > j, upd, a));
    }
    // z = D^-1 y on the right-hand-side lanes
    double x = a * rown;
    // back substitution: x_k is final once the rows below it are done
#pragma unroll
    for (int k = 5; k >= 1; --k) {
        const double xk = __shfl_sync(0xffffffffu, x, 21 + k);
        const double lki = __shfl_sync(0xffffffffu, a, li < k ? tri6(k, li) : 0);
        const double nx = fma(-lki, xk, x);
        x = sel64(rhs && li < k, nx, x);
    }
    *pd = ok;
    return x;
}

// The inverse of a 6x6 symmetric positive definite A on one warp: the
// factorisation A = L D L^T of warp_ldlt6_solve (lane e < 21 brings entry
// (i, j), e = tri6(i, j), of A's lower triangle; the other lanes' values are
// not used), then lane c < 6 solves L D L^T x = e_c (forward substitution,
// D^-1, back substitution), so that x[0..5] of lane c is column c of A^-1
// (other lanes: junk).  *pd: every pivot passed pivot_ok (every lane).  All
// 32 lanes must call it.
__device__ __forceinline__ void warp_spd6_inverse(double a, bool* pd, double x[6]) {
    const int lane = threadIdx.x & 31;
    const bool tri = lane < 21;
    int li = 5, lm = 6;
    if (tri) {
        li = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
            if (lane >= tri6(i, 0)) li = i;
        lm = lane - tri6(li, 0);
    }
    bool ok = true;
    double r[6];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = __shfl_sync(0xffffffffu, a, tri6(j, j));
        ok = ok && pivot_ok(d);
        r[j] = rcp64(d);
        const bool below = tri && li > j;
        const double aij = __shfl_sync(0xffffffffu, a, below ? tri6(li, j) : 0);
        const double amj = __shfl_sync(0xffffffffu, a, below && lm > j ? tri6(lm, j) : 0);
        const double lij = aij * r[j];
        const double upd = fma(-(aij * amj), r[j], a);
        a = sel64(below && lm == j, lij, sel64(below && lm > j, upd, a));
    }
    // column c = lane of A^-1; L_ik (i > k) is in lane tri6(i, k)
    const int c = lane < 6 ? lane : 0;
    double y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double s = sel64(i == c, 1.0, 0.0);
#pragma unroll
        for (int k = 0; k < i; ++k) s = fma(-__shfl_sync(0xffffffffu, a, tri6(i, k)), y[k], s);
        y[i] = s;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] *= r[i];
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s = fma(-__shfl_sync(0xffffffffu, a, tri6(k, i)), x[k], s);
        x[i] = s;
    }
    *pd = ok;
}

// The prior's terms of a Gauss-Newton iterate in anchor-frame coordinates.
// The normal equations (C^T H' C + L) dxi = -(C^T g' + L xi), with
// C = diag(Ra^T, Ra^T J_l(xi_theta)) mapping tangent steps to anchor-frame
// perturbations, become (H' + L') y = -(g' + m) in y = C dxi, with
// Ci = C^-1 = diag(Ra, J_l(xi_theta)^-1 Ra), L' = Ci^T L Ci and m = Ci^T L xi;
// then dxi = Ci y.  One warp (all 32 lanes call it) computes, from Ra (3x3
// row-major), L (6x6) and xi: ci1 = J_l(xi_theta)^-1 Ra (9), lp = L' (36,
// row-major), m (6) and ji = J_l(xi_theta)^-1 (9).  scratch: 69 doubles of
// shared memory.
__device__ __forceinline__ void warp_gn_prior_terms(const double* Ra, const double* L, const double* xi, double* ci1,
                                                    double* lp, double* m, double* ji, double* scratch) {
    const int lane = threadIdx.x & 31;
    double* Ji = scratch;         // J_l^-1 (9)
    double* Ci = scratch + 9;     // diag blocks of Ci: Ra (9), J_l^-1 Ra (9)
    double* T = scratch + 27;     // L Ci (36)
    double* Lx = scratch + 63;    // L xi (6)
    if (lane < 9) {
        const double v = so3_jl_inv_entry(xi + 3, lane / 3, lane % 3);
        Ji[lane] = v;
        ji[lane] = v;
    } else if (lane < 18) {
        Ci[lane - 9] = Ra[lane - 9];
    }
    __syncwarp();
    if (lane < 6) {
        double lx = 0.0;
        for (int k = 0; k < 6; ++k) lx = fma(L[6 * lane + k], xi[k], lx);
        Lx[lane] = lx;
    } else if (lane >= 8 && lane < 17) {   // J_l^-1 Ra
        const int e = lane - 8, i = e / 3, j = e % 3;
        const double v = fdot3(Ji[3 * i], Ra[j], Ji[3 * i + 1], Ra[3 + j], Ji[3 * i + 2], Ra[6 + j]);
        Ci[9 + e] = v;
        ci1[e] = v;
    }
    __syncwarp();
    // T[k][j] = sum over the block of j: L[k][3 bj + l] Ci_bj[l][jj]; lanes 4..9 of the
    // second round: m_i = sum over the block of i: Ci_bi[k][ii] (L xi)[3 bi + k]
#pragma unroll
    for (int round = 0; round < 2; ++round) {
        const int e = lane + 32 * round;
        const bool tm = e < 36, mm = round == 1 && lane >= 4 && lane < 10;
        const int k = tm ? e / 6 : 0, j = tm ? e % 6 : 0, bj = j / 3, jj = j % 3;
        const int i = mm ? lane - 4 : 0, bi = i / 3, ii = i % 3;
        const double* Cb = Ci + 9 * (mm ? bi : bj);
        const double a0 = mm ? Cb[ii] : L[6 * k + 3 * bj], a1 = mm ? Cb[3 + ii] : L[6 * k + 3 * bj + 1],
                     a2 = mm ? Cb[6 + ii] : L[6 * k + 3 * bj + 2];
        const double c0 = mm ? Lx[3 * bi] : Cb[jj], c1 = mm ? Lx[3 * bi + 1] : Cb[3 + jj],
                     c2 = mm ? Lx[3 * bi + 2] : Cb[6 + jj];
        const double v = fdot3(a0, c0, a1, c1, a2, c2);
        if (tm) T[e] = v;
        else if (mm) m[i] = v;
    }
    __syncwarp();
    // L' = Ci^T T: L'[i][j] = sum over the block of i: Ci_bi[k][ii] T[3 bi + k][j]
#pragma unroll
    for (int round = 0; round < 2; ++round) {
        const int e = lane + 32 * round;
        if (round == 1 && e >= 36) break;
        const int i = e / 6, j = e % 6, bi = i / 3, ii = i % 3;
        const double* Cb = Ci + 9 * bi;
        lp[e] = fdot3(Cb[ii], T[6 * (3 * bi) + j], Cb[3 + ii], T[6 * (3 * bi + 1) + j], Cb[6 + ii],
                      T[6 * (3 * bi + 2) + j]);
    }
}

// Block-cooperative inverse of an N x N SPD matrix (A and Ainv in shared
// or global memory): warp 0 factors it (lane i holding row i) into the
// shared scratch L / rdiag, then thread j solves for column j (unrolled);
// the result is symmetrised.  Every thread of the block must call it.  Returns false (on
// every thread) if not PD.
template <int N>
__device__ inline bool spd_inverse_block(const double* A, double* Ainv, double* L, double* rdiag, int* ok) {
    static_assert(N <= 32, "one row a lane");
    if (threadIdx.x < 32) {
        // right-looking Cholesky on warp 0, lane i holding row i: each step is
        // one warp instruction for all rows (GB300's FP64 pipe is paced by
        // warp instructions, not lanes)
        const int lane = threadIdx.x, row = lane < N ? lane : N - 1;
        double a[N], r[N];
#pragma unroll
        for (int j = 0; j < N; ++j) a[j] = A[row * N + j];
        bool pd = true;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double d = __shfl_sync(0xffffffffu, a[j], j);
            pd = pd && d > 0.0 && isfinite(d);
            const double rj = rsqrt(d);
            r[j] = rj;
            if (lane > j) a[j] = a[j] * rj;   // L_ij
#pragma unroll
            for (int m = j + 1; m < N; ++m) {
                const double lmj = __shfl_sync(0xffffffffu, a[j], m);
                if (lane >= m) a[m] = fma(-a[j], lmj, a[m]);
            }
        }
        if (lane < N) {
            rdiag[lane] = r[lane];
#pragma unroll
            for (int j = 0; j < N; ++j)
                if (j < lane) L[lane * N + j] = a[j];
        }
        if (lane == 0) *ok = pd ? 1 : 0;
    }
    __syncthreads();
    const bool good = *ok != 0;
    if (good && threadIdx.x < N) {
        const int c = threadIdx.x;
        double y[N], x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = i == c ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < i; ++k) s = fma(-L[i * N + k], y[k], s);
            y[i] = s * rdiag[i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
#pragma unroll
            for (int k = i + 1; k < N; ++k) s = fma(-L[k * N + i], x[k], s);
            x[i] = s * rdiag[i];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) Ainv[i * N + c] = x[i];
    }
    __syncthreads();
    if (good)
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            if (i < j) {
                const double m = 0.5 * (Ainv[i * N + j] + Ainv[j * N + i]);
                Ainv[i * N + j] = Ainv[j * N + i] = m;
            }
        }
    __syncthreads();
    return good;
}

// C = A (N x K) * B (K x M), computed by the threads of a block (element per
// thread); operands in shared memory.
template <int N, int K, int M>
__device__ inline void block_matmul(const double* A, const double* B, double* C) {
    for (int e = threadIdx.x; e < N * M; e += blockDim.x) {
        const int i = e / M, j = e % M;
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < K; ++l) s = fma(A[i * K + l], B[l * M + j], s);
        C[e] = s;
    }
    __syncthreads();
}

// C = A (N x K) * B^T (B: M x K)
template <int N, int K, int M>
__device__ inline void block_matmul_nt(const double* A, const double* B, double* C) {
    for (int e = threadIdx.x; e < N * M; e += blockDim.x) {
        const int i = e / M, j = e % M;
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < K; ++l) s = fma(A[i * K + l], B[j * K + l], s);
        C[e] = s;
    }
    __syncthreads();
}

}  // namespace prism
