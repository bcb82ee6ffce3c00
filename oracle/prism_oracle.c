/* PRISM filter oracle — plain FP64 CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never
 * does.  It shares no code with the CUDA library.  Build with
 *     gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread -o liboracle.so prism_oracle.c -lm
 * (-ffp-contract=off: every a*b+c below is two rounded operations unless it
 * is written as fma/fmaf).
 *
 * What each function follows (arXiv 2212.02988):
 *   or_render            App. B, ray points p = c + d r, d in {eps, 2 eps, ...};
 *                        trilinear field f_M; first point with f_occ > tau;
 *                        d* = alpha d_k + (1 - alpha) d_{k-1}; colour "analogously".
 *   or_render_backward   its adjoint (App. B: the emission is differentiable):
 *                        gradients of a weighted sum of the rendered depth and
 *                        colour with respect to the map means and the pose.
 *   or_depth_mask        App. F.3, ignore invalid and strongly discontinuous depth.
 *   or_anchor_normals    App. E.3, "normal of the rendered depth image".
 *   or_residuals         App. E.3, Eq. pointtoplanelaplace: point-to-plane and
 *                        photometric L1 terms against the previous rendered frame,
 *                        gates of App. F.2; residuals and pose Jacobians per pixel.
 *   or_normal_equations  their IRLS-weighted normal equations with the Laplace
 *                        scales of App. F.2, and the scaled J^T J of Sec. 4.1.
 *   or_predict           App. E.1 (transition, linearisation), Eq. statepropagation,
 *                        App. E.2 (split into pose prior and velocity conditional).
 *   or_localise          App. E.3 MAP objective minimised by Gauss-Newton with
 *                        IRLS weights; Sec. 4.1 Laplace covariance (2 J^T J)^-1;
 *                        App. F.2 EMA 0.8; Sec. 3.3.2 full-state recombination.
 *   or_fuse              App. D, Eq. mapupdategauss: per-voxel Gaussian product
 *                        with f_update = [-f_sdf, f_rgb]; App. F.2 frustum and
 *                        truncation rule, sigma_update = 1.
 *
 * Integer decisions use the FP32 recipe written out at each site (the device
 * kernels follow the same recipe); all values are FP64.
 *
 * The loops over rays (or_render), pixels (or_residuals, or_normal_equations)
 * and voxels (or_fuse) run on POSIX threads; each result is bit-identical for
 * any thread count (see parallel_for).  Build with -pthread.
 */
#define _POSIX_C_SOURCE 200809L
#include "prism_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ threads */
/* Work that is independent per item (a ray, a pixel, a row of voxels) is
 * split into ranges that worker threads take in turn.  Every item writes
 * only its own outputs; integer counts are added per worker (exact in any
 * order);
 * floating-point sums over items are formed per fixed chunk of items and the
 * chunk sums added in chunk order, neither depending on the thread count.
 * So every result is bit-identical for any number of threads. */
static int g_threads = 0;   /* 0: every online processor */

void or_set_threads(int32_t n) { g_threads = n > 0 ? n : 0; }

int32_t or_get_threads(void) {
    if (g_threads > 0) return g_threads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int32_t)n : 1;
}

typedef void (*range_fn)(void* ctx, long begin, long end, int job);
typedef struct {
    range_fn fn;
    void* ctx;
    long n, grain;
    long* next;   /* shared: the first item not yet taken */
    int job;
} range_job;

/* A worker takes ranges of `grain` items in turn until none is left. */
static void* run_ranges(void* arg) {
    range_job* j = (range_job*)arg;
    for (;;) {
        long b = __atomic_fetch_add(j->next, j->grain, __ATOMIC_RELAXED);
        if (b >= j->n) break;
        j->fn(j->ctx, b, b + j->grain < j->n ? b + j->grain : j->n, j->job);
    }
    return NULL;
}

#define OR_MAX_THREADS 256

/* fn(ctx, begin, end, job) over [0, n) in ranges of `grain` items, taken by
 * at most or_get_threads() workers; returns the number of workers (job ids
 * 0 .. workers - 1; a worker may receive several ranges). */
static int parallel_for(long n, long grain, range_fn fn, void* ctx) {
    if (grain < 1) grain = 1;
    long ranges = (n + grain - 1) / grain;
    int T = or_get_threads();
    if (T > OR_MAX_THREADS) T = OR_MAX_THREADS;
    if ((long)T > ranges) T = ranges > 0 ? (int)ranges : 1;
    long next = 0;
    range_job jobs[OR_MAX_THREADS];
    pthread_t th[OR_MAX_THREADS];
    int started[OR_MAX_THREADS];
    for (int t = 0; t < T; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].n = n;
        jobs[t].grain = grain;
        jobs[t].next = &next;
        jobs[t].job = t;
        started[t] = t > 0 && pthread_create(&th[t], NULL, run_ranges, &jobs[t]) == 0;
    }
    run_ranges(&jobs[0]);   /* the caller works too; a worker that failed to start leaves its share to the others */
    for (int t = 1; t < T; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    return T;
}

/* ------------------------------------------------------------ small linear algebra */
static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_vec(const double A[9], const double x[3], double y[3]) {
    for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

static void mat3_tvec(const double A[9], const double x[3], double y[3]) {
    for (int i = 0; i < 3; ++i) y[i] = A[i] * x[0] + A[3 + i] * x[1] + A[6 + i] * x[2];
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void skew3(const double w[3], double K[9]) {
    K[0] = 0; K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2]; K[4] = 0; K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0]; K[8] = 0;
}

/* C (n x m) = A (n x k) B (k x m), row-major */
static void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}

static void transpose(const double* A, double* T, int n, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
}

/* Cholesky factor of a symmetric n x n matrix (n <= 12); 0 if not positive definite. */
static int cholesky(const double* A, double* L, int n) {
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0) || !isfinite(s)) return 0;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return 1;
}

/* Solve A x = b with A symmetric positive definite; 0 on failure. */
static int spd_solve(const double* A, const double* b, double* x, int n) {
    double L[144], y[12];
    if (!cholesky(A, L, n)) return 0;
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
    return 1;
}

/* Inverse of a symmetric positive definite matrix, column by column. */
static int spd_inverse(const double* A, double* Ainv, int n) {
    double e[12], x[12];
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) e[i] = (i == j) ? 1.0 : 0.0;
        if (!spd_solve(A, e, x, n)) return 0;
        for (int i = 0; i < n; ++i) Ainv[i * n + j] = x[i];
    }
    for (int i = 0; i < n; ++i)       /* exact symmetry */
        for (int j = i + 1; j < n; ++j) {
            double m = 0.5 * (Ainv[i * n + j] + Ainv[j * n + i]);
            Ainv[i * n + j] = Ainv[j * n + i] = m;
        }
    return 1;
}

/* Inverse of a general 3x3 matrix by the adjugate. */
static void mat3_inverse(const double A[9], double B[9]) {
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

/* ------------------------------------------------------------------ rotations */
/* A pose with its quaternion normalised: q / sqrt(((w*w + x*x) + y*y) + z*z).
 * Every entry point normalises the poses it is given, once, with exactly
 * these operations (the device library does the same at its boundary). */
static void normalise_pose(const double in[7], double out[7]) {
    double n = sqrt(((in[3] * in[3] + in[4] * in[4]) + in[5] * in[5]) + in[6] * in[6]);
    for (int a = 0; a < 3; ++a) out[a] = in[a];
    for (int a = 0; a < 4; ++a) out[3 + a] = in[3 + a] / n;
}

/* Rotation matrix of a unit quaternion (w, x, y, z).  This is also the FP64
 * recipe from which the FP32 decision matrices are rounded, so its operation
 * order is fixed: products first, then the sums of the standard formula. */
static void quat_to_R(const double qin[4], double R[9]) {
    double w = qin[0], x = qin[1], y = qin[2], z = qin[3];
    double xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    double wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0 - 2.0 * (yy + zz); R[1] = 2.0 * (xy - wz);       R[2] = 2.0 * (xz + wy);
    R[3] = 2.0 * (xy + wz);       R[4] = 1.0 - 2.0 * (xx + zz); R[5] = 2.0 * (yz - wx);
    R[6] = 2.0 * (xz - wy);       R[7] = 2.0 * (yz + wx);       R[8] = 1.0 - 2.0 * (xx + yy);
}

/* Exp map of so(3) (Rodrigues). */
static void so3_exp(const double w[3], double R[9]) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double K[9], K2[9], a, b;
    skew3(w, K);
    mat3_mul(K, K, K2);
    if (th < 1e-8) { a = 1.0 - th * th / 6.0; b = 0.5 - th * th / 24.0; }
    else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
    for (int i = 0; i < 9; ++i) R[i] = ((i % 4) == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* Left Jacobian of SO(3): Exp(phi + d) ~= Exp(J_l(phi) d) Exp(phi). */
static void so3_jl(const double w[3], double J[9]) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double K[9], K2[9], a, b;
    skew3(w, K);
    mat3_mul(K, K, K2);
    if (th < 1e-6) { a = 0.5 - th * th / 24.0; b = 1.0 / 6.0 - th * th / 120.0; }
    else { a = (1.0 - cos(th)) / (th * th); b = (th - sin(th)) / (th * th * th); }
    for (int i = 0; i < 9; ++i) J[i] = ((i % 4) == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* Unit quaternion of a rotation matrix (w >= 0). */
static void R_to_quat(const double R[9], double q[4]) {
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
    double sg = q[0] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < 4; ++i) q[i] = sg * q[i] / n;
}

/* ---------------------------------------------------------- FP32 decision helpers */
static inline float lerp32(float a, float b, float t) { return fmaf(t, b - a, a); }

/* Camera-frame point of pixel (u, v) at z-depth z, FP32 recipe:
 * (z * ((u - cx) * (1/fx)), z * ((v - cy) * (1/fy)), z). */
static inline void backproject32(const or_params* P, int u, int v, float z, float out[3]) {
    float cx = (float)P->cx, cy = (float)P->cy;
    float ifx = (float)(1.0 / P->fx), ify = (float)(1.0 / P->fy);
    out[0] = z * (((float)u - cx) * ifx);
    out[1] = z * (((float)v - cy) * ify);
    out[2] = z;
}

/* y = M x + b in FP32 as fmaf(M0, x0, fmaf(M1, x1, fmaf(M2, x2, b))) per row. */
static inline void affine32(const float M[9], const float b[3], const float x[3], float y[3]) {
    for (int r = 0; r < 3; ++r)
        y[r] = fmaf(M[3 * r], x[0], fmaf(M[3 * r + 1], x[1], fmaf(M[3 * r + 2], x[2], b[r])));
}

/* =================================================================== render */
/* Map layout: linear, z-major, x fastest: index (k * ny + j) * nx + i;
 * rgb interleaved, 3 values per voxel. */
static inline long vidx(const or_params* P, int i, int j, int k) {
    return ((long)k * P->ny + j) * (long)P->nx + i;
}

typedef struct { int x0, x1, y0, y1, z0, z1; float fx, fy, fz; } cell_t;

/* FP32 recipe for sample k of a ray given in grid units (cg, rg):
 * d = (float)k * eps; g = fmaf(d, rg, cg); inside iff -0.5 <= g < n - 0.5 per axis;
 * i0 = floor(g), f = g - i0, corners clamped to [0, n-1]. */
static int sample_cell(const or_params* P, const float cg[3], const float rg[3], float eps32, int k,
                       cell_t* c) {
    float d = (float)k * eps32;
    float g[3];
    int n[3] = {P->nx, P->ny, P->nz};
    int lo[3], hi[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
        g[a] = fmaf(d, rg[a], cg[a]);
        if (!(g[a] >= -0.5f && g[a] < (float)n[a] - 0.5f)) return 0;
    }
    for (int a = 0; a < 3; ++a) {
        float fl = floorf(g[a]);
        int i0 = (int)fl;
        f[a] = g[a] - fl;
        lo[a] = i0 < 0 ? 0 : i0;
        hi[a] = i0 + 1 > n[a] - 1 ? n[a] - 1 : i0 + 1;
    }
    c->x0 = lo[0]; c->x1 = hi[0]; c->y0 = lo[1]; c->y1 = hi[1]; c->z0 = lo[2]; c->z1 = hi[2];
    c->fx = f[0]; c->fy = f[1]; c->fz = f[2];
    return 1;
}

/* FP32 trilinear (the decision value): lerp along x, then y, then z. */
static float trilinear32(const or_params* P, const double* m, int stride, int ch, const cell_t* c) {
#define V(i, j, k) ((float)m[vidx(P, i, j, k) * stride + ch])
    float c00 = lerp32(V(c->x0, c->y0, c->z0), V(c->x1, c->y0, c->z0), c->fx);
    float c10 = lerp32(V(c->x0, c->y1, c->z0), V(c->x1, c->y1, c->z0), c->fx);
    float c01 = lerp32(V(c->x0, c->y0, c->z1), V(c->x1, c->y0, c->z1), c->fx);
    float c11 = lerp32(V(c->x0, c->y1, c->z1), V(c->x1, c->y1, c->z1), c->fx);
#undef V
    float c0 = lerp32(c00, c10, c->fy);
    float c1 = lerp32(c01, c11, c->fy);
    return lerp32(c0, c1, c->fz);
}

/* FP64 trilinear (the value): sum of the 8 corners times product weights. */
static double trilinear64(const or_params* P, const double* m, int stride, int ch, const cell_t* c) {
    double fx = c->fx, fy = c->fy, fz = c->fz, s = 0.0;
    int xs[2] = {c->x0, c->x1}, ys[2] = {c->y0, c->y1}, zs[2] = {c->z0, c->z1};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                double w = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy) * (e ? fz : 1.0 - fz);
                s += w * m[vidx(P, xs[a], ys[b], zs[e]) * stride + ch];
            }
    return s;
}

typedef struct {
    const or_params* P;
    const double *occ, *rgb;
    const int32_t* pix;
    double* depth;
    double* rgb_out;
    uint8_t* mask;
    int32_t* hitk;
    double pose[7];
    float R32[9], c32[3], o32[3];
    long kmax;
    int64_t nsamp[OR_MAX_THREADS];
} render_ctx;

/* Rays n in [begin, end). */
static void render_rays(void* arg, long begin, long end, int job) {
    render_ctx* X = (render_ctx*)arg;
    const or_params* P = X->P;
    float inv_vs = (float)(1.0 / P->voxel), eps32 = (float)P->eps, tau32 = (float)P->tau;
    float cx = (float)P->cx, cy = (float)P->cy;
    float ifx = (float)(1.0 / P->fx), ify = (float)(1.0 / P->fy);
    int64_t nsamp = 0;
    for (long n = begin; n < end; ++n) {
        int p = X->pix ? X->pix[n] : (int)n;
        int u = p % P->width, v = p / P->width;
        /* ray direction r = R dir_c / |R dir_c|, dir_c = ((u-cx)/fx, (v-cy)/fy, 1) */
        float dx = ((float)u - cx) * ifx, dy = ((float)v - cy) * ify;
        float w[3], r[3], cg[3], rg[3];
        for (int a = 0; a < 3; ++a) w[a] = fmaf(X->R32[3 * a], dx, fmaf(X->R32[3 * a + 1], dy, X->R32[3 * a + 2]));
        float inv_n = 1.0f / sqrtf(fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2])));
        for (int a = 0; a < 3; ++a) {
            r[a] = w[a] * inv_n;
            cg[a] = fmaf(X->c32[a] - X->o32[a], inv_vs, -0.5f);
            rg[a] = r[a] * inv_vs;
        }
        /* march: first k with f_occ(p_k) > tau */
        cell_t prev, cur;
        int k = 1, hit = 0;
        for (; k <= X->kmax; ++k) {
            if (!sample_cell(P, cg, rg, eps32, k, &cur)) break;
            ++nsamp;
            if (trilinear32(P, X->occ, 1, 0, &cur) > tau32) { hit = 1; break; }
            prev = cur;
        }
        double d_out = 0.0, col[3] = {0, 0, 0};
        int hk = 0;
        if (hit && k == 1) hk = -1;          /* camera inside matter: no valid depth */
        if (hit && k >= 2) {
            hk = k;
            double f0 = trilinear64(P, X->occ, 1, 0, &prev), f1 = trilinear64(P, X->occ, 1, 0, &cur);
            double alpha = (P->tau - f0) / (f1 - f0);
            double dk = k * P->eps, dk1 = (k - 1) * P->eps;
            double dstar = alpha * dk + (1.0 - alpha) * dk1;
            /* z-depth: the unit ray's camera-z component is 1/|dir_c| */
            double dcx = (u - P->cx) / P->fx, dcy = (v - P->cy) / P->fy;
            d_out = dstar / sqrt(dcx * dcx + dcy * dcy + 1.0);
            for (int ch = 0; ch < 3; ++ch)
                col[ch] = alpha * trilinear64(P, X->rgb, 3, ch, &cur) +
                          (1.0 - alpha) * trilinear64(P, X->rgb, 3, ch, &prev);
        }
        if (X->depth) X->depth[n] = d_out;
        if (X->rgb_out) for (int ch = 0; ch < 3; ++ch) X->rgb_out[3 * n + ch] = col[ch];
        if (X->mask) X->mask[n] = (uint8_t)(hk >= 2);
        if (X->hitk) X->hitk[n] = hk;
    }
    X->nsamp[job] += nsamp;
}

int or_render(const or_params* P, const double* occ, const double* rgb, const double pose_in[7],
              const int32_t* pix, int32_t npix, double* depth, double* rgb_out, uint8_t* mask,
              int32_t* hitk, int64_t* n_samples) {
    render_ctx* X = (render_ctx*)calloc(1, sizeof(render_ctx));
    if (!X) return -2;
    double R[9];
    normalise_pose(pose_in, X->pose);
    quat_to_R(X->pose + 3, R);
    /* FP32 ray set-up (decision recipe) */
    for (int i = 0; i < 9; ++i) X->R32[i] = (float)R[i];
    for (int a = 0; a < 3; ++a) { X->c32[a] = (float)X->pose[a]; X->o32[a] = (float)P->origin[a]; }
    X->kmax = P->max_depth > 0 ? (long)floor(P->max_depth / P->eps) : 0x7fffffffL;
    X->P = P; X->occ = occ; X->rgb = rgb; X->pix = npix > 0 && pix ? pix : NULL;
    X->depth = depth; X->rgb_out = rgb_out; X->mask = mask; X->hitk = hitk;
    long total = npix > 0 && pix ? npix : (long)P->width * P->height;
    int jobs = parallel_for(total, 64, render_rays, X);
    int64_t nsamp = 0;
    for (int j = 0; j < jobs; ++j) nsamp += X->nsamp[j];
    if (n_samples) *n_samples = nsamp;
    free(X);
    return 0;
}

/* ============================================================ render adjoint */
/* Gradient of  L = sum_pixels gD * depth + sum_pixels,c gC_c * rgb_c  with
 * respect to the occupancy and colour means and to a world-frame
 * perturbation of the camera pose (t' = t + dt, R' = Exp(dtheta) R), for
 * the render of App. B.  With the hit between samples k-1 and k:
 *   alpha = (tau - f0) / (f1 - f0),  depth = (alpha d_k + (1 - alpha) d_{k-1}) / |dir_c|,
 *   rgb_c = alpha C_c(p_k) + (1 - alpha) C_c(p_{k-1}),
 *   dL/dalpha = gD eps / |dir_c| + sum_c gC_c (C_c(p_k) - C_c(p_{k-1})),
 *   dL/df0 = dL/dalpha (alpha - 1) / (f1 - f0),  dL/df1 = -dL/dalpha alpha / (f1 - f0);
 * each trilinear value passes its gradient to its 8 corners with the
 * trilinear weights, and to its sample position p with grad_p = grad_g / vs;
 * p_k = c + d_k r gives dL/dt += gp_k and dL/dtheta += d_k (r x gp_k).  The
 * hit index is held fixed (it is piecewise constant in the inputs). */
static void trilinear64_grad(const or_params* P, const double* m, int stride, int ch, const cell_t* c,
                             double g[3]) {
    double fx = c->fx, fy = c->fy, fz = c->fz;
    int xs[2] = {c->x0, c->x1}, ys[2] = {c->y0, c->y1}, zs[2] = {c->z0, c->z1};
    g[0] = g[1] = g[2] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                double v = m[vidx(P, xs[a], ys[b], zs[e]) * stride + ch];
                double wx = a ? fx : 1.0 - fx, wy = b ? fy : 1.0 - fy, wz = e ? fz : 1.0 - fz;
                g[0] += (a ? 1.0 : -1.0) * wy * wz * v;
                g[1] += wx * (b ? 1.0 : -1.0) * wz * v;
                g[2] += wx * wy * (e ? 1.0 : -1.0) * v;
            }
}

static void scatter64(const or_params* P, double* gm, int stride, int ch, const cell_t* c, double gval) {
    double fx = c->fx, fy = c->fy, fz = c->fz;
    int xs[2] = {c->x0, c->x1}, ys[2] = {c->y0, c->y1}, zs[2] = {c->z0, c->z1};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                double w = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy) * (e ? fz : 1.0 - fz);
                gm[vidx(P, xs[a], ys[b], zs[e]) * stride + ch] += gval * w;
            }
}

int or_render_backward(const or_params* P, const double* occ, const double* rgb, const double pose_in[7],
                       const double* gD, const double* gC, double* g_occ, double* g_rgb, double g_pose[6]) {
    double R[9], pose[7];
    normalise_pose(pose_in, pose);
    quat_to_R(pose + 3, R);
    float R32[9], c32[3], o32[3];
    for (int i = 0; i < 9; ++i) R32[i] = (float)R[i];
    for (int a = 0; a < 3; ++a) { c32[a] = (float)pose[a]; o32[a] = (float)P->origin[a]; }
    float inv_vs = (float)(1.0 / P->voxel), eps32 = (float)P->eps, tau32 = (float)P->tau;
    float cx = (float)P->cx, cy = (float)P->cy;
    float ifx = (float)(1.0 / P->fx), ify = (float)(1.0 / P->fy);
    long kmax = P->max_depth > 0 ? (long)floor(P->max_depth / P->eps) : 0x7fffffffL;
    for (int i = 0; i < 6; ++i) g_pose[i] = 0.0;
    for (int p = 0; p < P->width * P->height; ++p) {
        int u = p % P->width, v = p / P->width;
        double gd = gD ? gD[p] : 0.0, gc[3] = {0, 0, 0};
        if (gC) for (int c = 0; c < 3; ++c) gc[c] = gC[3 * p + c];
        if (gd == 0.0 && gc[0] == 0.0 && gc[1] == 0.0 && gc[2] == 0.0) continue;
        /* march (same decisions as or_render) */
        float dx = ((float)u - cx) * ifx, dy = ((float)v - cy) * ify;
        float w[3], cg[3], rg[3];
        for (int a = 0; a < 3; ++a) w[a] = fmaf(R32[3 * a], dx, fmaf(R32[3 * a + 1], dy, R32[3 * a + 2]));
        float inv_n = 1.0f / sqrtf(fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2])));
        for (int a = 0; a < 3; ++a) {
            cg[a] = fmaf(c32[a] - o32[a], inv_vs, -0.5f);
            rg[a] = (w[a] * inv_n) * inv_vs;
        }
        cell_t prev, cur;
        int k = 1, hit = 0;
        for (; k <= kmax; ++k) {
            if (!sample_cell(P, cg, rg, eps32, k, &cur)) break;
            if (trilinear32(P, occ, 1, 0, &cur) > tau32) { hit = 1; break; }
            prev = cur;
        }
        if (!hit || k < 2) continue;
        /* values and gradients in FP64 */
        double f0 = trilinear64(P, occ, 1, 0, &prev), f1 = trilinear64(P, occ, 1, 0, &cur);
        double alpha = (P->tau - f0) / (f1 - f0);
        double dcx = (u - P->cx) / P->fx, dcy = (v - P->cy) / P->fy;
        double ndir = sqrt(dcx * dcx + dcy * dcy + 1.0);
        double C0[3], C1[3];
        for (int c = 0; c < 3; ++c) {
            C0[c] = trilinear64(P, rgb, 3, c, &prev);
            C1[c] = trilinear64(P, rgb, 3, c, &cur);
        }
        double gA = gd * P->eps / ndir;
        for (int c = 0; c < 3; ++c) gA += gc[c] * (C1[c] - C0[c]);
        double gf0 = gA * (alpha - 1.0) / (f1 - f0), gf1 = -gA * alpha / (f1 - f0);
        if (g_occ) {
            scatter64(P, g_occ, 1, 0, &prev, gf0);
            scatter64(P, g_occ, 1, 0, &cur, gf1);
        }
        if (g_rgb)
            for (int c = 0; c < 3; ++c) {
                scatter64(P, g_rgb, 3, c, &prev, gc[c] * (1.0 - alpha));
                scatter64(P, g_rgb, 3, c, &cur, gc[c] * alpha);
            }
        /* pose: positions of samples k-1 and k */
        double dirw[3], r[3];
        double dc[3] = {dcx, dcy, 1.0};
        mat3_vec(R, dc, dirw);
        for (int a = 0; a < 3; ++a) r[a] = dirw[a] / ndir;
        const cell_t* cells[2] = {&prev, &cur};
        double gfs[2] = {gf0, gf1}, wa[2] = {1.0 - alpha, alpha}, ds[2] = {(k - 1) * P->eps, k * P->eps};
        for (int s = 0; s < 2; ++s) {
            double gp[3], tmp[3], rx[3];
            trilinear64_grad(P, occ, 1, 0, cells[s], gp);
            for (int a = 0; a < 3; ++a) gp[a] *= gfs[s];
            for (int c = 0; c < 3; ++c) {
                trilinear64_grad(P, rgb, 3, c, cells[s], tmp);
                for (int a = 0; a < 3; ++a) gp[a] += gc[c] * wa[s] * tmp[a];
            }
            for (int a = 0; a < 3; ++a) gp[a] /= P->voxel;
            cross3(r, gp, rx);
            for (int a = 0; a < 3; ++a) {
                g_pose[a] += gp[a];
                g_pose[3 + a] += ds[s] * rx[a];
            }
        }
    }
    return 0;
}

/* ============================================================ depth validity */
/* Pixel valid iff D > 0, finite, and every in-image 4-neighbour Dn satisfies
 * fabsf(D - Dn) <= disc in FP32 (App. F.3: invalid or discontinuous depth). */
typedef struct {
    const or_params* P;
    const float* depth;
    uint8_t* mask;
} mask_ctx;

/* Rows v in [begin, end). */
static void mask_rows(void* arg, long begin, long end, int job) {
    (void)job;
    mask_ctx* X = (mask_ctx*)arg;
    int W = X->P->width, H = X->P->height;
    const float* depth = X->depth;
    float disc = (float)X->P->disc;
    for (int v = (int)begin; v < (int)end; ++v)
        for (int u = 0; u < W; ++u) {
            float d = depth[v * W + u];
            int ok = (d > 0.0f) && isfinite(d);
            int nu[4] = {u - 1, u + 1, u, u}, nv[4] = {v, v, v - 1, v + 1};
            for (int e = 0; e < 4 && ok; ++e) {
                if (nu[e] < 0 || nu[e] >= W || nv[e] < 0 || nv[e] >= H) continue;
                if (!(fabsf(d - depth[nv[e] * W + nu[e]]) <= disc)) ok = 0;
            }
            X->mask[v * W + u] = (uint8_t)ok;
        }
}

void or_depth_mask(const or_params* P, const float* depth, uint8_t* mask) {
    mask_ctx X = {P, depth, mask};
    parallel_for(P->height, 8, mask_rows, &X);
}

/* ============================================================ anchor normals */
/* n = normalize((P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1))), turned to face
 * the camera; valid iff the pixel and its 4 neighbours are valid and it is
 * not on the image border.  FP32 recipe for n32 (used for decisions) and the
 * same construction in FP64 for n64 (used for values). */
typedef struct {
    const or_params* P;
    const float* depth;
    const uint8_t* mask;
    double* n64;
    float* n32;
    uint8_t* nvalid;
} normals_ctx;

/* Rows v in [begin, end). */
static void normal_rows(void* arg, long begin, long end, int job) {
    (void)job;
    normals_ctx* X = (normals_ctx*)arg;
    const or_params* P = X->P;
    const float* depth = X->depth;
    const uint8_t* mask = X->mask;
    double* n64 = X->n64;
    float* n32 = X->n32;
    uint8_t* nvalid = X->nvalid;
    int W = P->width, H = P->height;
    for (int v = (int)begin; v < (int)end; ++v)
        for (int u = 0; u < W; ++u) {
            int p = v * W + u;
            int ok = u >= 1 && u <= W - 2 && v >= 1 && v <= H - 2 && mask[p] && mask[p - 1] &&
                     mask[p + 1] && mask[p - W] && mask[p + W];
            float nn[3] = {0, 0, 0};
            double nd[3] = {0, 0, 0};
            if (ok) {
                float a[3], b[3], c[3], d[3], e1[3], e2[3], cr[3], pc[3];
                backproject32(P, u + 1, v, depth[p + 1], a);
                backproject32(P, u - 1, v, depth[p - 1], b);
                backproject32(P, u, v + 1, depth[p + W], c);
                backproject32(P, u, v - 1, depth[p - W], d);
                backproject32(P, u, v, depth[p], pc);
                for (int i = 0; i < 3; ++i) { e1[i] = a[i] - b[i]; e2[i] = c[i] - d[i]; }
                float t0 = e1[1] * e2[2], t1 = e1[2] * e2[1];
                cr[0] = t0 - t1;
                t0 = e1[2] * e2[0]; t1 = e1[0] * e2[2];
                cr[1] = t0 - t1;
                t0 = e1[0] * e2[1]; t1 = e1[1] * e2[0];
                cr[2] = t0 - t1;
                float n2 = fmaf(cr[0], cr[0], fmaf(cr[1], cr[1], cr[2] * cr[2]));
                if (!(n2 > 0.0f) || !isfinite(n2)) ok = 0;
                else {
                    float inv = 1.0f / sqrtf(n2);
                    for (int i = 0; i < 3; ++i) nn[i] = cr[i] * inv;
                    float dp = fmaf(nn[0], pc[0], fmaf(nn[1], pc[1], nn[2] * pc[2]));
                    int flip = dp > 0.0f;
                    if (flip) for (int i = 0; i < 3; ++i) nn[i] = -nn[i];
                    /* FP64 value of the same normal */
                    double A[3], B[3], C[3], Dd[3], E1[3], E2[3], CR[3];
                    int us[4] = {u + 1, u - 1, u, u}, vs[4] = {v, v, v + 1, v - 1};
                    double* pts[4] = {A, B, C, Dd};
                    for (int s = 0; s < 4; ++s) {
                        double z = depth[vs[s] * W + us[s]];
                        pts[s][0] = z * (us[s] - P->cx) / P->fx;
                        pts[s][1] = z * (vs[s] - P->cy) / P->fy;
                        pts[s][2] = z;
                    }
                    for (int i = 0; i < 3; ++i) { E1[i] = A[i] - B[i]; E2[i] = C[i] - Dd[i]; }
                    cross3(E1, E2, CR);
                    double nr = sqrt(CR[0] * CR[0] + CR[1] * CR[1] + CR[2] * CR[2]);
                    for (int i = 0; i < 3; ++i) nd[i] = (flip ? -1.0 : 1.0) * CR[i] / nr;
                }
            }
            if (!ok) { nn[0] = nn[1] = nn[2] = 0.0f; nd[0] = nd[1] = nd[2] = 0.0; }
            for (int i = 0; i < 3; ++i) {
                if (n32) n32[3 * p + i] = nn[i];
                if (n64) n64[3 * p + i] = nd[i];
            }
            if (nvalid) nvalid[p] = (uint8_t)ok;
        }
}

void or_anchor_normals(const or_params* P, const float* depth, const uint8_t* mask,
                       double* n64, float* n32, uint8_t* nvalid) {
    normals_ctx X = {P, depth, mask, n64, n32, nvalid};
    parallel_for(P->height, 8, normal_rows, &X);
}

/* ===================================================== residuals + normal equations */
typedef struct {
    const or_params* P;
    const float *a_depth, *a_rgb, *o_depth, *o_rgb;
    const uint8_t *a_mask, *o_mask, *a_nval;
    const float* a_n32;
    const double* a_n64;
    double pose[7], anchor_pose[7], R[9], Ra[9];
    float M32[9], b32[3];
    double* r;
    double* J;
    int32_t* assoc;
    uint8_t* kept;
} resid_ctx;

/* Pixels p in [begin, end). */
static void residual_pixels(void* arg, long begin, long end, int job) {
    (void)job;
    resid_ctx* X = (resid_ctx*)arg;
    const or_params* P = X->P;
    const int W = P->width, H_ = P->height;
    const float *a_depth = X->a_depth, *a_rgb = X->a_rgb, *o_depth = X->o_depth, *o_rgb = X->o_rgb;
    const double *R = X->R, *Ra = X->Ra, *pose = X->pose, *anchor_pose = X->anchor_pose;
    double *r = X->r, *J = X->J;
    float fx32 = (float)P->fx, fy32 = (float)P->fy, cx32 = (float)P->cx, cy32 = (float)P->cy;
    float gate_geo = (float)P->gate_geo, gate_rgb = (float)P->gate_rgb;
    for (long pl = begin; pl < end; ++pl) {
            const int p = (int)pl, u = p % W, v = p / W;
            X->kept[p] = 0;
            X->assoc[2 * p] = X->assoc[2 * p + 1] = -1;
            for (int k = 0; k < 4; ++k) r[4 * p + k] = 0.0;
            for (int k = 0; k < 24; ++k) J[24 * p + k] = 0.0;
            if (!X->o_mask[p]) continue;
            /* ---- decisions, FP32 recipe ---- */
            float z = o_depth[p], P32[3], X32[3];
            backproject32(P, u, v, z, P32);
            affine32(X->M32, X->b32, P32, X32);
            if (!(X32[2] > 0.0f)) continue;
            float iz = 1.0f / X32[2];
            float up = fmaf(fx32 * X32[0], iz, cx32), vp = fmaf(fy32 * X32[1], iz, cy32);
            float nu = floorf(up + 0.5f), nv = floorf(vp + 0.5f);
            if (!(nu >= 0.0f && nu <= (float)(W - 1) && nv >= 0.0f && nv <= (float)(H_ - 1))) continue;
            int iu = (int)nu, iv = (int)nv, q = iv * W + iu;
            if (!X->a_nval[q]) continue;
            float bu = floorf(up), bv = floorf(vp);
            if (!(bu >= 0.0f && bu <= (float)(W - 2) && bv >= 0.0f && bv <= (float)(H_ - 2))) continue;
            int ju = (int)bu, jv = (int)bv, b00 = jv * W + ju;
            const uint8_t* am = X->a_mask;
            if (!(am[b00] && am[b00 + 1] && am[b00 + W] && am[b00 + W + 1])) continue;
            X->assoc[2 * p] = q;
            X->assoc[2 * p + 1] = b00;
            float a32 = up - bu, c32 = vp - bv;
            float ph[3], e[3];
            const float* n32 = X->a_n32;
            backproject32(P, iu, iv, a_depth[q], ph);
            for (int i = 0; i < 3; ++i) e[i] = ph[i] - X32[i];
            float rg32 = fmaf(n32[3 * q], e[0], fmaf(n32[3 * q + 1], e[1], n32[3 * q + 2] * e[2]));
            if (!(fabsf(rg32) <= gate_geo)) continue;
            int gated = 0;
            for (int ch = 0; ch < 3 && !gated; ++ch) {
                float top = lerp32(a_rgb[3 * b00 + ch], a_rgb[3 * (b00 + 1) + ch], a32);
                float bot = lerp32(a_rgb[3 * (b00 + W) + ch], a_rgb[3 * (b00 + W + 1) + ch], a32);
                float r32 = lerp32(top, bot, c32) - o_rgb[3 * p + ch];
                if (!(fabsf(r32) <= gate_rgb)) gated = 1;
            }
            if (gated) continue;
            X->kept[p] = 1;
            /* ---- values, FP64 ---- */
            double Pc[3] = {z * (u - P->cx) / P->fx, z * (v - P->cy) / P->fy, (double)z};
            double y[3], rel[3], Xa[3];
            mat3_vec(R, Pc, y);                                  /* world offset from camera */
            for (int i = 0; i < 3; ++i) rel[i] = y[i] + pose[i] - anchor_pose[i];
            mat3_tvec(Ra, rel, Xa);                              /* point in the anchor frame */
            double za = a_depth[q];
            double ph64[3] = {za * (iu - P->cx) / P->fx, za * (iv - P->cy) / P->fy, za};
            const double* nq = X->a_n64 + 3 * q;
            double aX[4][3];
            r[4 * p] = nq[0] * (ph64[0] - Xa[0]) + nq[1] * (ph64[1] - Xa[1]) + nq[2] * (ph64[2] - Xa[2]);
            for (int i = 0; i < 3; ++i) aX[0][i] = -nq[i];
            double upd = P->fx * Xa[0] / Xa[2] + P->cx, vpd = P->fy * Xa[1] / Xa[2] + P->cy;
            double aa = upd - ju, cc = vpd - jv;
            double du_dX[3] = {P->fx / Xa[2], 0.0, -P->fx * Xa[0] / (Xa[2] * Xa[2])};
            double dv_dX[3] = {0.0, P->fy / Xa[2], -P->fy * Xa[1] / (Xa[2] * Xa[2])};
            for (int ch = 0; ch < 3; ++ch) {
                double I00 = a_rgb[3 * b00 + ch], I10 = a_rgb[3 * (b00 + 1) + ch];
                double I01 = a_rgb[3 * (b00 + W) + ch], I11 = a_rgb[3 * (b00 + W + 1) + ch];
                double val = (1 - aa) * (1 - cc) * I00 + aa * (1 - cc) * I10 + (1 - aa) * cc * I01 +
                             aa * cc * I11;
                double gu = (1 - cc) * (I10 - I00) + cc * (I11 - I01);
                double gv = (1 - aa) * (I01 - I00) + aa * (I11 - I10);
                r[4 * p + 1 + ch] = val - o_rgb[3 * p + ch];
                for (int i = 0; i < 3; ++i) aX[1 + ch][i] = gu * du_dX[i] + gv * dv_dX[i];
            }
            for (int k = 0; k < 4; ++k) {
                double aw[3];
                double* Jk = J + 24 * p + 6 * k;
                mat3_vec(Ra, aX[k], aw);                         /* gradient wrt the world point */
                Jk[0] = aw[0]; Jk[1] = aw[1]; Jk[2] = aw[2];
                cross3(y, aw, Jk + 3);                           /* d r / d dtheta = y x aw */
            }
    }
}

/* Residuals of the objective of App. E.3 (Eq. pointtoplanelaplace) for every
 * observed pixel at camera pose `pose`, against the anchor observation
 * rendered at `anchor_pose`:
 *   r[4p]     = <p_hat - X, n_hat>            (point-to-plane, anchor frame)
 *   r[4p+1+c] = I_hat_c(pi(X)) - I_c(p)       (photometric, bilinear in the anchor)
 * X is the observed point moved into the anchor camera; p_hat, n_hat come
 * from the nearest anchor pixel.  J[24p + 6k + i] is d r_k / d xi_i for a
 * world-frame perturbation of the camera pose, t' = t + dt, R' = Exp(dtheta) R,
 * xi = (dt, dtheta).  kept[p] = 1 iff the pixel passed every validity check
 * and both gates (App. F.2); assoc[2p] = nearest anchor pixel, assoc[2p+1] =
 * the bilinear cell's top-left pixel (-1 when not associated). */
int or_residuals(const or_params* P, const double anchor_in[7], const float* a_depth,
                 const float* a_rgb, const double pose_in[7], const float* o_depth, const float* o_rgb,
                 double* r, double* J, int32_t* assoc, uint8_t* kept) {
    resid_ctx X;
    memset(&X, 0, sizeof(X));
    normalise_pose(anchor_in, X.anchor_pose);
    normalise_pose(pose_in, X.pose);
    int W = P->width, H_ = P->height, N = W * H_;
    uint8_t* a_mask = (uint8_t*)malloc(N);
    uint8_t* o_mask = (uint8_t*)malloc(N);
    uint8_t* a_nval = (uint8_t*)malloc(N);
    float* a_n32 = (float*)malloc(sizeof(float) * 3 * N);
    double* a_n64 = (double*)malloc(sizeof(double) * 3 * N);
    if (!a_mask || !o_mask || !a_nval || !a_n32 || !a_n64) {
        free(a_mask); free(o_mask); free(a_nval); free(a_n32); free(a_n64);
        return -2;
    }
    or_depth_mask(P, a_depth, a_mask);
    or_depth_mask(P, o_depth, o_mask);
    or_anchor_normals(P, a_depth, a_mask, a_n64, a_n32, a_nval);

    double Mrel[9], d[3], brel[3];
    const double *pose = X.pose, *anchor_pose = X.anchor_pose;
    double *R = X.R, *Ra = X.Ra;
    quat_to_R(pose + 3, R);
    quat_to_R(anchor_pose + 3, Ra);
    /* FP64 recipe of the relative transform current-camera -> anchor-camera,
     * rounded once to FP32 for the decisions:
     * Mrel = Ra^T R (sum order k = 0, 1, 2), brel = Ra^T (t - ta). */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Mrel[3 * i + j] = (Ra[i] * R[j] + Ra[3 + i] * R[3 + j]) + Ra[6 + i] * R[6 + j];
    for (int a = 0; a < 3; ++a) d[a] = pose[a] - anchor_pose[a];
    for (int i = 0; i < 3; ++i) brel[i] = (Ra[i] * d[0] + Ra[3 + i] * d[1]) + Ra[6 + i] * d[2];
    for (int i = 0; i < 9; ++i) X.M32[i] = (float)Mrel[i];
    for (int i = 0; i < 3; ++i) X.b32[i] = (float)brel[i];
    X.P = P;
    X.a_depth = a_depth; X.a_rgb = a_rgb; X.o_depth = o_depth; X.o_rgb = o_rgb;
    X.a_mask = a_mask; X.o_mask = o_mask; X.a_nval = a_nval; X.a_n32 = a_n32; X.a_n64 = a_n64;
    X.r = r; X.J = J; X.assoc = assoc; X.kept = kept;
    parallel_for(N, 1024, residual_pixels, &X);
    free(a_mask); free(o_mask); free(a_nval); free(a_n32); free(a_n64);
    return 0;
}

/* Sums over the kept residuals of one chunk of pixels [begin, end), in
 * pixel order: H (36), g (6), Ht (36), cost, count. */
#define OR_NE_CHUNK 1024
#define OR_NE_VALUES 80
typedef struct {
    const or_params* P;
    const double *r, *J;
    const uint8_t* kept;
    long npix;
    double* chunk_sums;   /* OR_NE_VALUES per chunk */
} ne_ctx;

static void ne_chunks(void* arg, long begin, long end, int job) {
    (void)job;
    ne_ctx* X = (ne_ctx*)arg;
    const or_params* P = X->P;
    for (long c = begin; c < end; ++c) {
        double* S = X->chunk_sums + OR_NE_VALUES * c;
        double *H = S, *g = S + 36, *Ht = S + 42;
        memset(S, 0, sizeof(double) * OR_NE_VALUES);
        long p_end = (c + 1) * OR_NE_CHUNK < X->npix ? (c + 1) * OR_NE_CHUNK : X->npix;
        for (long p = c * OR_NE_CHUNK; p < p_end; ++p) {
            if (!X->kept[p]) continue;
            for (int k = 0; k < 4; ++k) {
                double b = k == 0 ? P->b_geo : P->b_rgb, fl = k == 0 ? P->floor_geo : P->floor_rgb;
                double res = X->r[4 * p + k], ar = fabs(res);
                double w = 1.0 / (b * (ar > fl ? ar : fl)), ib2 = 1.0 / (b * b);
                const double* Jk = X->J + 24 * p + 6 * k;
                for (int i = 0; i < 6; ++i) {
                    g[i] += w * Jk[i] * res;
                    for (int j = 0; j < 6; ++j) {
                        H[6 * i + j] += w * Jk[i] * Jk[j];
                        Ht[6 * i + j] += ib2 * Jk[i] * Jk[j];
                    }
                }
                S[78] += ar / b;
            }
            S[79] += 1.0;
        }
    }
}

/* Sums over the kept residuals (or_residuals):
 *   H  = sum w J^T J,  g = sum w J^T r   with IRLS weights w = 1/(b max(|r|, floor)),
 *   Ht = sum J^T J / b^2                  (Laplace, Sec. 4.1),
 *   stats = (sum |r|/b, kept pixels).
 * Each sum is formed over chunks of OR_NE_CHUNK consecutive pixels (pixel
 * order within a chunk), then over the chunks in order. */
int or_normal_equations(const or_params* P, const double anchor_pose[7], const float* a_depth,
                        const float* a_rgb, const double pose[7], const float* o_depth,
                        const float* o_rgb, double H[36], double g[6], double Ht[36],
                        double stats[2]) {
    int N = P->width * P->height;
    long nchunk = (N + OR_NE_CHUNK - 1) / OR_NE_CHUNK;
    double* r = (double*)malloc(sizeof(double) * 4 * N);
    double* J = (double*)malloc(sizeof(double) * 24 * N);
    int32_t* assoc = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    uint8_t* kept = (uint8_t*)malloc(N);
    double* cs = (double*)malloc(sizeof(double) * OR_NE_VALUES * (nchunk > 0 ? nchunk : 1));
    int rc = (!r || !J || !assoc || !kept || !cs) ? -2
             : or_residuals(P, anchor_pose, a_depth, a_rgb, pose, o_depth, o_rgb, r, J, assoc, kept);
    if (rc) { free(r); free(J); free(assoc); free(kept); free(cs); return rc ? rc : -2; }
    ne_ctx X = {P, r, J, kept, N, cs};
    parallel_for(nchunk, 1, ne_chunks, &X);
    double S[OR_NE_VALUES];
    memset(S, 0, sizeof(S));
    for (long c = 0; c < nchunk; ++c)
        for (int v = 0; v < OR_NE_VALUES; ++v) S[v] += cs[OR_NE_VALUES * c + v];
    memcpy(H, S, sizeof(double) * 36);
    memcpy(g, S + 36, sizeof(double) * 6);
    memcpy(Ht, S + 42, sizeof(double) * 36);
    stats[0] = S[78];
    stats[1] = S[79];
    free(r); free(J); free(assoc); free(kept); free(cs);
    return 0;
}

/* ================================================================ prediction */
/* App. E.1 transition (Euler integration of acceleration, then of velocity,
 * with the printed (dt)^2 read as dt), linearised to first order around the
 * propagated mean; Eq. statepropagation; split (App. E.2) into the pose
 * prior N(mu_p, S_pp) and the velocity conditional N(v; vbar + D dp, S_vel).
 * Controls from the IMU window (App. E.1: "IMU readings as controls"):
 *   u_lin = R_mid mean(acc) + g, R_mid the orientation half a step ahead
 *           (mean specific force over the window, rotated to the world);
 *   u_ang = (R_end w_end - w_prev) / dt, w_end the least-squares line through
 *           the window's gyro samples evaluated at its last sample time, and
 *           R_end the orientation a full step ahead. */
int or_predict(const or_params* P, const or_state* s, const double* imu, int32_t n_imu, double dt,
               or_prior* out) {
    if (!(dt > 0.0)) return -1;
    double R[9], sp[7], spn[7];
    for (int a = 0; a < 3; ++a) sp[a] = s->t[a];
    for (int a = 0; a < 4; ++a) sp[3 + a] = s->q[a];
    normalise_pose(sp, spn);
    quat_to_R(spn + 3, R);
    double acc[3] = {0, 0, 0}, gyr[3] = {0, 0, 0}, tm = 0.0, tend = -1e300;
    for (int i = 0; i < n_imu; ++i) {
        tm += imu[7 * i] / n_imu;
        if (imu[7 * i] > tend) tend = imu[7 * i];
        for (int a = 0; a < 3; ++a) { acc[a] += imu[7 * i + 1 + a] / n_imu; gyr[a] += imu[7 * i + 4 + a] / n_imu; }
    }
    double u_lin[3] = {0, 0, 0}, u_ang[3] = {0, 0, 0};
    if (n_imu > 0) {
        /* gyro at the window's end: mean + slope * (t_end - t_mean) */
        double stt = 0.0, stg[3] = {0, 0, 0}, gend[3];
        for (int i = 0; i < n_imu; ++i) {
            double dtm = imu[7 * i] - tm;
            stt += dtm * dtm;
            for (int a = 0; a < 3; ++a) stg[a] += dtm * (imu[7 * i + 4 + a] - gyr[a]);
        }
        for (int a = 0; a < 3; ++a) gend[a] = gyr[a] + (stt > 0.0 ? stg[a] / stt * (tend - tm) : 0.0);
        double wm[3], half[3], full[3], Rh[9], Rf[9], Rmid[9], Rend[9], am[3], we[3];
        mat3_vec(R, gyr, wm);
        for (int a = 0; a < 3; ++a) { half[a] = 0.5 * dt * wm[a]; full[a] = dt * wm[a]; }
        so3_exp(half, Rh);
        so3_exp(full, Rf);
        mat3_mul(Rh, R, Rmid);
        mat3_mul(Rf, R, Rend);
        mat3_vec(Rmid, acc, am);
        mat3_vec(Rend, gend, we);
        for (int a = 0; a < 3; ++a) {
            u_lin[a] = am[a] + (a == 2 ? -P->gravity : 0.0);
            u_ang[a] = (we[a] - s->w[a]) / dt;
        }
    }
    /* propagated mean */
    double v[3], w[3], wdt[3], Rw[9], Rn[9];
    for (int a = 0; a < 3; ++a) {
        v[a] = s->v[a] + u_lin[a] * dt;
        w[a] = s->w[a] + u_ang[a] * dt;
        out->v[a] = v[a];
        out->w[a] = w[a];
        out->t[a] = s->t[a] + v[a] * dt;
        wdt[a] = w[a] * dt;
    }
    so3_exp(wdt, Rw);
    mat3_mul(Rw, R, Rn);
    R_to_quat(Rn, out->q);
    /* linearisation: dp' = A dp + B dv',  A = diag(I, Exp(w dt)), B = diag(dt I, J_l(w dt) dt) */
    double Jl[9];
    so3_jl(wdt, Jl);
    double A[36] = {0}, B[36] = {0};
    for (int i = 0; i < 3; ++i) {
        A[6 * i + i] = 1.0;
        B[6 * i + i] = dt;
        for (int j = 0; j < 3; ++j) {
            A[6 * (3 + i) + 3 + j] = Rw[3 * i + j];
            B[6 * (3 + i) + 3 + j] = Jl[3 * i + j] * dt;
        }
    }
    /* joint map of (dp, dv) at t-1 plus noise: dv' = dv + n_v, dp' = A dp + B dv' + n_p */
    double F[144] = {0}, Ft[144], T1[144], Sig[144];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            F[12 * i + j] = A[6 * i + j];
            F[12 * i + 6 + j] = B[6 * i + j];
        }
    for (int i = 0; i < 6; ++i) F[12 * (6 + i) + 6 + i] = 1.0;
    transpose(F, Ft, 12, 12);
    matmul(F, s->cov, T1, 12, 12, 12);
    matmul(T1, Ft, Sig, 12, 12, 12);
    double Qv[6], Qp[6];
    for (int i = 0; i < 3; ++i) {
        Qv[i] = P->sigma_vel[0] * P->sigma_vel[0];
        Qv[3 + i] = P->sigma_vel[1] * P->sigma_vel[1];
        Qp[i] = P->sigma_pose[0] * P->sigma_pose[0];
        Qp[3 + i] = P->sigma_pose[1] * P->sigma_pose[1];
    }
    /* noise covariance: [[B Qv B^T + Qp, B Qv], [Qv B^T, Qv]] */
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s_ = 0.0;
            for (int k = 0; k < 6; ++k) s_ += B[6 * i + k] * Qv[k] * B[6 * j + k];
            Sig[12 * i + j] += s_ + (i == j ? Qp[i] : 0.0);
            Sig[12 * i + 6 + j] += B[6 * i + j] * Qv[j];
            Sig[12 * (6 + j) + i] += B[6 * i + j] * Qv[j];
        }
    for (int i = 0; i < 6; ++i) Sig[12 * (6 + i) + 6 + i] += Qv[i];
    for (int i = 0; i < 12; ++i)                    /* exact symmetry */
        for (int j = i + 1; j < 12; ++j) {
            double m = 0.5 * (Sig[12 * i + j] + Sig[12 * j + i]);
            Sig[12 * i + j] = Sig[12 * j + i] = m;
        }
    memcpy(out->cov, Sig, sizeof(Sig));
    /* split: S_pp, D = S_vp S_pp^-1, S_vel = S_vv - D S_pv */
    double Spp[36], Svp[36], Svv[36], Spv[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            Spp[6 * i + j] = Sig[12 * i + j];
            Spv[6 * i + j] = Sig[12 * i + 6 + j];
            Svp[6 * i + j] = Sig[12 * (6 + i) + j];
            Svv[6 * i + j] = Sig[12 * (6 + i) + 6 + j];
        }
    memcpy(out->cov_pp, Spp, sizeof(Spp));
    if (!spd_inverse(Spp, out->prec_pp, 6)) return -4;
    matmul(Svp, out->prec_pp, out->D, 6, 6, 6);
    double DS[36];
    matmul(out->D, Spv, DS, 6, 6, 6);
    for (int i = 0; i < 36; ++i) out->cov_vel[i] = Svv[i] - DS[i];
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            double m = 0.5 * (out->cov_vel[6 * i + j] + out->cov_vel[6 * j + i]);
            out->cov_vel[6 * i + j] = out->cov_vel[6 * j + i] = m;
        }
    return 0;
}

/* ============================================================== localisation */
/* Pose at tangent coordinates xi around the prior mean: t = t_mu + xi_t,
 * R = Exp(xi_theta) R_mu. */
static void retract(const or_prior* pr, const double xi[6], double pose[7]) {
    double Rm[9], E[9], Rn[9], pm[7], pmn[7];
    for (int a = 0; a < 3; ++a) pm[a] = pr->t[a];
    for (int a = 0; a < 4; ++a) pm[3 + a] = pr->q[a];
    normalise_pose(pm, pmn);
    quat_to_R(pmn + 3, Rm);
    so3_exp(xi + 3, E);
    mat3_mul(E, Rm, Rn);
    for (int a = 0; a < 3; ++a) pose[a] = pr->t[a] + xi[a];
    R_to_quat(Rn, pose + 3);
}

/* M = blkdiag(I, J_l(xi_theta)): maps tangent steps to world-frame perturbations. */
static void tangent_map(const double xi[6], double M[36]) {
    double Jl[9];
    so3_jl(xi + 3, Jl);
    memset(M, 0, sizeof(double) * 36);
    for (int i = 0; i < 3; ++i) {
        M[6 * i + i] = 1.0;
        for (int j = 0; j < 3; ++j) M[6 * (3 + i) + 3 + j] = Jl[3 * i + j];
    }
}

/* ============================================== the paper's pose optimiser */
/* SplitMix64 (Steele, Lea and Flood 2014): the state advances by the golden
 * gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
 * variant-13 finaliser.  Output i of the sequence started at `seed`. */
uint64_t or_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform pixel of n: floor(n u) with u = (high 32 bits) / 2^32. */
uint32_t or_sample_pixel(uint64_t seed, uint64_t i, uint32_t n) {
    return (uint32_t)(((or_splitmix64(seed, i) >> 32) * (uint64_t)n) >> 32);
}

/* App. F.2 ("Pose optimisation"): Adam with its momentum disabled (beta1 = 0,
 * so the first moment is the gradient itself), separate step sizes for the
 * translation and rotation components, adam_steps steps, each evaluating the
 * objective of App. E.3 on adam_pixels pixels drawn uniformly (with
 * replacement) from the image; gated and invalid pixels contribute nothing.
 * The data term's gradient is the L1 subgradient sum sign(r)/b dr/dxi over
 * the drawn pixels, scaled by (pixels in the image) / adam_pixels so that it
 * estimates the full-image objective, whose prior term 1/2 xi^T L xi adds
 * L xi.  Second moment v_s = beta2 v_{s-1} + (1 - beta2) g^2, bias-corrected;
 * xi -= lr g / (sqrt(v_hat) + eps). */
int or_adam(const or_params* P, const or_prior* pr, const double anchor_pose[7], const float* a_depth,
            const float* a_rgb, const float* o_depth, const float* o_rgb, uint64_t counter0,
            double xi_out[6], double* xi_trace) {
    const int N = P->width * P->height, S = P->adam_steps, K = P->adam_pixels;
    double* r = (double*)malloc(sizeof(double) * 4 * N);
    double* J = (double*)malloc(sizeof(double) * 24 * N);
    int32_t* assoc = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    uint8_t* kept = (uint8_t*)malloc(N);
    if (!r || !J || !assoc || !kept) { free(r); free(J); free(assoc); free(kept); return -2; }
    double xi[6] = {0, 0, 0, 0, 0, 0}, v[6] = {0, 0, 0, 0, 0, 0}, pose[7], M[36];
    double b2t = 1.0;
    for (int s = 1; s <= S; ++s) {
        retract(pr, xi, pose);
        if (or_residuals(P, anchor_pose, a_depth, a_rgb, pose, o_depth, o_rgb, r, J, assoc, kept)) {
            free(r); free(J); free(assoc); free(kept);
            return -2;
        }
        double gw[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k < K; ++k) {
            const uint32_t p = or_sample_pixel(P->adam_seed, counter0 + (uint64_t)(s - 1) * K + k, (uint32_t)N);
            if (!kept[p]) continue;
            for (int res = 0; res < 4; ++res) {
                const double b = res == 0 ? P->b_geo : P->b_rgb, rr = r[4 * p + res];
                const double sg = rr > 0.0 ? 1.0 : (rr < 0.0 ? -1.0 : 0.0);
                for (int i = 0; i < 6; ++i) gw[i] += sg / b * J[24 * p + 6 * res + i];
            }
        }
        tangent_map(xi, M);
        const double scale = (double)N / (double)K;
        double g[6];
        for (int i = 0; i < 6; ++i) {
            double mg = 0.0, lx = 0.0;
            for (int k = 0; k < 6; ++k) { mg += M[6 * k + i] * gw[k]; lx += pr->prec_pp[6 * i + k] * xi[k]; }
            g[i] = scale * mg + lx;
        }
        b2t *= P->adam_beta2;
        for (int i = 0; i < 6; ++i) {
            v[i] = P->adam_beta2 * v[i] + (1.0 - P->adam_beta2) * g[i] * g[i];
            const double vhat = v[i] / (1.0 - b2t), lr = i < 3 ? P->adam_lr_t : P->adam_lr_r;
            xi[i] -= lr * g[i] / (sqrt(vhat) + P->adam_eps);
        }
        if (xi_trace) for (int i = 0; i < 6; ++i) xi_trace[6 * (s - 1) + i] = xi[i];
    }
    for (int i = 0; i < 6; ++i) xi_out[i] = xi[i];
    free(r); free(J); free(assoc); free(kept);
    return 0;
}

int or_localise(const or_params* P, const or_prior* pr, const or_state* prev,
                const float* a_depth, const float* a_rgb, const float* o_depth, const float* o_rgb,
                or_state* out, or_loc_diag* diag) {
    double anchor[7], xi[6] = {0, 0, 0, 0, 0, 0}, pose[7];
    for (int a = 0; a < 3; ++a) anchor[a] = prev->t[a];
    for (int a = 0; a < 4; ++a) anchor[3 + a] = prev->q[a];
    double H[36], g[6], Ht[36], st[2], M[36], Mt[36], T[36], Hx[36], gx[6], step[6];
    if (P->optimiser == 1) {   /* the paper's Adam; draws numbered from the frame's count */
        const uint64_t c0 = (uint64_t)prev->n_localised * (uint64_t)P->adam_steps * (uint64_t)P->adam_pixels;
        if (or_adam(P, pr, anchor, a_depth, a_rgb, o_depth, o_rgb, c0, xi, NULL)) return -2;
    }
    for (int it = 0; P->optimiser != 1 && it < P->n_gn; ++it) {
        retract(pr, xi, pose);
        if (or_normal_equations(P, anchor, a_depth, a_rgb, pose, o_depth, o_rgb, H, g, Ht, st)) return -2;
        /* normal equations in xi: (M^T H M + L) step = -(M^T g + L xi) */
        tangent_map(xi, M);
        transpose(M, Mt, 6, 6);
        matmul(Mt, H, T, 6, 6, 6);
        matmul(T, M, Hx, 6, 6, 6);
        for (int i = 0; i < 6; ++i) {
            double s = 0.0, lx = 0.0;
            for (int k = 0; k < 6; ++k) { s += Mt[6 * i + k] * g[k]; lx += pr->prec_pp[6 * i + k] * xi[k]; }
            gx[i] = -(s + lx);
        }
        for (int i = 0; i < 36; ++i) Hx[i] += pr->prec_pp[i];
        if (!spd_solve(Hx, gx, step, 6)) return -4;
        for (int i = 0; i < 6; ++i) xi[i] += step[i];
    }
    retract(pr, xi, pose);
    if (or_normal_equations(P, anchor, a_depth, a_rgb, pose, o_depth, o_rgb, H, g, Ht, st)) return -2;
    /* Laplace: Sigma = (2 Jt^T Jt + prior)^-1 in world-frame perturbation
     * coordinates at the optimum; the prior Hessian L (in xi) becomes M^-T L M^-1. */
    double Mi[36], Mit[36], Lp[36], Hl[36], Slap[36];
    tangent_map(xi, M);
    memset(Mi, 0, sizeof(Mi));
    {
        double J3[9], J3i[9];
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) J3[3 * i + j] = M[6 * (3 + i) + 3 + j];
        mat3_inverse(J3, J3i);
        for (int i = 0; i < 3; ++i) {
            Mi[6 * i + i] = 1.0;
            for (int j = 0; j < 3; ++j) Mi[6 * (3 + i) + 3 + j] = J3i[3 * i + j];
        }
    }
    transpose(Mi, Mit, 6, 6);
    matmul(Mit, pr->prec_pp, T, 6, 6, 6);
    matmul(T, Mi, Lp, 6, 6, 6);
    for (int i = 0; i < 36; ++i) Hl[i] = 2.0 * Ht[i] + Lp[i];
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            double m = 0.5 * (Hl[6 * i + j] + Hl[6 * j + i]);
            Hl[6 * i + j] = Hl[6 * j + i] = m;
        }
    if (!spd_inverse(Hl, Slap, 6)) return -4;
    /* EMA over time (App. F.2) */
    double Sp[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double prevS = prev->cov[12 * i + j];
            Sp[6 * i + j] = prev->n_localised > 0 ? P->ema * prevS + (1.0 - P->ema) * Slap[6 * i + j]
                                                  : Slap[6 * i + j];
        }
    /* recombination (Sec. 3.3.2): v | p = vbar + D xi(p); at the optimum
     * v = vbar + D xi*; in the new pose coordinates D' = D M^-1. */
    double Dp[36], DS[36], Dpt[36], DSD[36];
    matmul(pr->D, Mi, Dp, 6, 6, 6);
    memset(out, 0, sizeof(*out));
    for (int a = 0; a < 3; ++a) out->t[a] = pose[a];
    for (int a = 0; a < 4; ++a) out->q[a] = pose[3 + a];
    for (int i = 0; i < 6; ++i) {
        double dv = 0.0;
        for (int k = 0; k < 6; ++k) dv += pr->D[6 * i + k] * xi[k];
        if (i < 3) out->v[i] = pr->v[i] + dv;
        else out->w[i - 3] = pr->w[i - 3] + dv;
    }
    matmul(Dp, Sp, DS, 6, 6, 6);          /* cov(v, p) = D' S_p */
    transpose(Dp, Dpt, 6, 6);
    matmul(DS, Dpt, DSD, 6, 6, 6);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            out->cov[12 * i + j] = Sp[6 * i + j];
            out->cov[12 * (6 + i) + j] = DS[6 * i + j];
            out->cov[12 * j + 6 + i] = DS[6 * i + j];
            out->cov[12 * (6 + i) + 6 + j] = DSD[6 * i + j] + pr->cov_vel[6 * i + j];
        }
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j) {
            double m = 0.5 * (out->cov[12 * i + j] + out->cov[12 * j + i]);
            out->cov[12 * i + j] = out->cov[12 * j + i] = m;
        }
    out->n_localised = prev->n_localised + 1;
    if (diag) {
        diag->cost = st[0];
        diag->n_pixels = st[1];
        for (int i = 0; i < 6; ++i) diag->xi[i] = xi[i];
    }
    return 0;
}

/* =================================================================== map update */
/* Per voxel centre: projective SDF against the observed depth at pose `pose`
 * (nearest pixel), updated iff the centre is in the frustum (z > 0, pixel in
 * the image, valid depth) and between the camera and surface + trunc; then
 * the Gaussian product of Eq. mapupdategauss with precision 1/update_var:
 *   L' = L + Lu,  mu' = (L mu + Lu f) / L',  f = [-clamp(sdf, -trunc, trunc), rgb].
 * Colour is updated only where |sdf| <= trunc.  Returns the number of voxels
 * whose occupancy was updated. */
typedef struct {
    const or_params* P;
    double *occ, *rgb, *var_occ, *var_rgb;
    const float *depth, *rgb_obs;
    const uint8_t* mask;
    double pose[7], R[9];
    float M32[9], b32[3], o32[3];
    int64_t n_upd[OR_MAX_THREADS];
} fuse_ctx;

/* Voxel slices z in [begin, end). */
static void fuse_slices(void* arg, long begin, long end, int job) {
    fuse_ctx* X = (fuse_ctx*)arg;
    const or_params* P = X->P;
    const int W = P->width, H = P->height;
    const double *pose = X->pose, *R = X->R;
    float vs32 = (float)P->voxel, trunc32 = (float)P->trunc;
    float fx32 = (float)P->fx, fy32 = (float)P->fy, cx32 = (float)P->cx, cy32 = (float)P->cy;
    double Lu = 1.0 / P->update_var;
    int64_t n_upd = 0;
    for (long kl = begin; kl < end; ++kl)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                const int k = (int)kl;
                /* ---- decisions, FP32 recipe ---- */
                float pc[3] = {fmaf((float)i + 0.5f, vs32, X->o32[0]), fmaf((float)j + 0.5f, vs32, X->o32[1]),
                               fmaf((float)k + 0.5f, vs32, X->o32[2])};
                float Xc32[3];
                affine32(X->M32, X->b32, pc, Xc32);
                if (!(Xc32[2] > 0.0f)) continue;
                float iz = 1.0f / Xc32[2];
                float u = fmaf(fx32 * Xc32[0], iz, cx32), v = fmaf(fy32 * Xc32[1], iz, cy32);
                float nu = floorf(u + 0.5f), nv = floorf(v + 0.5f);
                if (!(nu >= 0.0f && nu <= (float)(W - 1) && nv >= 0.0f && nv <= (float)(H - 1))) continue;
                int p = (int)nv * W + (int)nu;
                if (!X->mask[p]) continue;
                float sdf32 = X->depth[p] - Xc32[2];
                if (!(sdf32 >= -trunc32)) continue;
                int colour = fabsf(sdf32) <= trunc32;
                /* ---- values, FP64 ---- */
                double pw[3] = {P->origin[0] + (i + 0.5) * P->voxel, P->origin[1] + (j + 0.5) * P->voxel,
                                P->origin[2] + (k + 0.5) * P->voxel};
                double rel[3] = {pw[0] - pose[0], pw[1] - pose[1], pw[2] - pose[2]}, Xc[3];
                mat3_tvec(R, rel, Xc);
                double sdf = (double)X->depth[p] - Xc[2];
                double f = -(sdf < P->trunc ? (sdf > -P->trunc ? sdf : -P->trunc) : P->trunc);
                long vi = vidx(P, i, j, k);
                double L = 1.0 / X->var_occ[vi], Ln = L + Lu;
                X->occ[vi] = (L * X->occ[vi] + Lu * f) / Ln;
                X->var_occ[vi] = 1.0 / Ln;
                ++n_upd;
                if (colour) {
                    double Lc = 1.0 / X->var_rgb[vi], Lcn = Lc + Lu;
                    for (int ch = 0; ch < 3; ++ch)
                        X->rgb[3 * vi + ch] = (Lc * X->rgb[3 * vi + ch] + Lu * (double)X->rgb_obs[3 * p + ch]) / Lcn;
                    X->var_rgb[vi] = 1.0 / Lcn;
                }
            }
    X->n_upd[job] += n_upd;
}

int64_t or_fuse(const or_params* P, double* occ, double* rgb, double* var_occ, double* var_rgb,
                const double pose_in[7], const float* depth, const float* rgb_obs) {
    fuse_ctx* X = (fuse_ctx*)calloc(1, sizeof(fuse_ctx));
    if (!X) return -2;
    normalise_pose(pose_in, X->pose);
    int W = P->width, H = P->height;
    uint8_t* mask = (uint8_t*)malloc((size_t)W * H);
    if (!mask) { free(X); return -2; }
    or_depth_mask(P, depth, mask);
    const double* pose = X->pose;
    double* R = X->R;
    quat_to_R(pose + 3, R);
    /* FP64 recipe of the world->camera transform, rounded once to FP32:
     * M = R^T, b = -((R0i t0 + R1i t1) + R2i t2). */
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) X->M32[3 * i + j] = (float)R[3 * j + i];
        X->b32[i] = (float)(-((R[i] * pose[0] + R[3 + i] * pose[1]) + R[6 + i] * pose[2]));
        X->o32[i] = (float)P->origin[i];
    }
    X->P = P; X->occ = occ; X->rgb = rgb; X->var_occ = var_occ; X->var_rgb = var_rgb;
    X->depth = depth; X->rgb_obs = rgb_obs; X->mask = mask;
    int jobs = parallel_for(P->nz, 1, fuse_slices, X);
    int64_t n_upd = 0;
    for (int j = 0; j < jobs; ++j) n_upd += X->n_upd[j];
    free(mask);
    free(X);
    return n_upd;
}
