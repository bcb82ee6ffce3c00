// prism_dev.cuh — device-side building blocks shared by the PRISM kernels:
// the launch parameter block, the map layout, the FP64 pose recipe
// that produces the FP32 decision matrices, and the FP32 decision recipe
// (every operation written with an explicit IEEE-rounded intrinsic so that
// the compiler cannot contract or reorder it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace prism {

// ------------------------------------------------ programmatic dependent launch
// Every kernel of the library starts with pdl_enter(): it waits until the
// grid before it in the stream has completed and its memory is visible
// (griddepcontrol.wait; a no-op when launched without the attribute), then
// lets the next grid be scheduled.  Launched through launch_pdl, a kernel's
// launch and block scheduling therefore overlap the tail of the kernel before
// it instead of following its completion.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ----------------------------------------------------------------- parameters
// Constants every kernel may need, filled once on the host (FP32 copies are
// single roundings of the FP64 configuration values).
struct KParams {
    int nx, ny, nz;            // voxels
    int nbx, nby, nbz;         // 8^3 tiles per axis (culling and fuse blocks)
    uint32_t px, py, pxy;      // padded plane: (nx + 2), (ny + 2), (nx + 2) (ny + 2)
    uint32_t npad;             // elements of a padded plane
    int W, H;                  // image size
    int kmax;                  // last ray sample index
    int bf16;                  // map storage is bf16
    int skip;                  // rays skip bricks whose occupancy bound stays below tau
    int nlev;                  // brick levels above the 4^3 bricks (0..3): level l has edge 4 * 2^l
    int bb_off[4];             // offset of level l's brick bounds in MapPlanes::bb
    int bb_len;                // brick bounds of all levels
    float o32[3];              // grid origin
    float vs32, inv_vs32;      // voxel size and its inverse
    float eps32, tau32, trunc32, disc32;
    float fx32, fy32, cx32, cy32, ifx32, ify32;
    float gate_geo32, gate_rgb32;
    float b_geo32, b_rgb32, floor_geo32, floor_rgb32;
    float upd_prec32;          // 1 / update_var
    double vs, origin[3], eps, tau, trunc;
    double fx, fy, cx, cy;
    double sigma_vel[2], sigma_pose[2];
    double ema, gravity, update_var;
    unsigned long long* check; // bounds-check build: the first index violation (device word), or null
};

// ------------------------------------------------------------ checked build
// Built with -DPRISM_CHECKED (libprism_checked.so), the kernels test the
// data-dependent indices of their gathers and scatters before the access:
// an index outside [0, n) skips the access (the result is then wrong, but
// nothing outside the buffer is touched) and the first violation is kept in
// *P.check as (site << 48) | (index & (2^48 - 1)).  Without the flag every
// test is the constant true and compiles away.
enum CheckSite : int {
    CHK_RENDER_CORNER = 1,   // a trilinear cell's last corner in a map plane (npad)
    CHK_RENDER_BRICK = 2,    // a brick bound (bb_len)
    CHK_TRACK_ANCHOR = 3,    // an anchor gather (W H)
    CHK_TRACK_PARTIAL = 4,   // a block's partial column (the partials' stride)
    CHK_FUSE_TILE = 5,       // a listed tile (nbx nby nbz)
    CHK_FUSE_VOXEL = 6,      // a voxel of a map plane (npad)
    CHK_FUSE_PIXEL = 7,      // a voxel's nearest pixel (W H)
    CHK_BWD_CORNER = 8,      // a gradient corner of the render adjoint (npad)
    CHK_PLAN = 9,            // a tile of the anchor render's order (tiles)
};

#ifdef PRISM_CHECKED
__device__ __forceinline__ bool check_index(unsigned long long* word, int site, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (word) atomicCAS(word, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
#define PRISM_IN_RANGE(P, site, i, n) ::prism::check_index((P).check, (site), (long long)(i), (long long)(n))
#else
#define PRISM_IN_RANGE(P, site, i, n) true
#endif

// Device-resident filter state (FP64).  One per handle.
struct DevState {
    // posterior q_t(s_t)
    double t[3], q[4], v[3], w[3];
    double cov[144];
    // prior from the prediction step
    double pt[3], pq[4], pv[3], pw[3];
    double pcov[144], cov_pp[36], prec_pp[36], D[36], cov_vel[36];
    // Gauss-Newton iterate: xi in the prior's tangent coordinates, and the pose it gives
    double xi[6];
    double cur_pose[7];
    // pose at which the current anchor was rendered
    double anchor_pose[7];
    // last exported normal equations: H(36), g(6), Ht(36), cost, count
    double ne_out[80];
    // render-adjoint pose gradient (world-frame perturbation)
    double grad_pose[6];
    // The prior's terms of the current Gauss-Newton iterate in anchor-frame
    // coordinates (linalg64.cuh, warp_gn_prior_terms), ready for the next
    // pass's finish: Ci = diag(R_a, J_l(xi_theta)^-1 R_a) (two 3x3 blocks),
    // L' = Ci^T L Ci and m = Ci^T L xi (L = prior pose precision)
    double gn_Ci[18];
    double gn_Lp[36];
    double gn_m[6];
    double gn_Ji[9];           // J_l(xi_theta)^-1 of the current iterate
    // constants of one localisation for the FP32 matrices of each iterate:
    // q0 = conj(q_anchor) (x) q_prior (the rotation Ra^T R_prior) and
    // b0 = Ra^T (t_prior - t_anchor)
    double gn_q0[4];
    double gn_b0[3];
    // FP32 decision matrices, each computed once per pose by the FP64 recipe:
    float c2w[12];             // state mean, camera -> world: R (9), centre (3)
    float w2c[12];             // state mean, world -> camera: M (9), b (3)
    float rel[12];             // Gauss-Newton pose -> anchor camera: M (9), b (3)
    float aux[12];             // a pose given by the host (render or one objective evaluation)
    int n_localised;
    int flags;                 // bit 0: GN system not PD; bit 1: Laplace system not PD; bit 2: prior not PD;
                               // bit 3: a grid-wide wait of the localisation timed out
                               // (cleared by each prediction, set by the kernels of that step)
    int rejected;              // the last localisation raised a flag: the posterior was left as it was and
                               // the step's map update lists no tile (0 after creation or a state write)
    int pad1;
};

enum : int { FLAG_GN_NOTPD = 1, FLAG_LAPLACE_NOTPD = 2, FLAG_PRIOR_NOTPD = 4, FLAG_SYNC_TIMEOUT = 8 };

// Work counters (device, accumulated with warp-aggregated atomics).
struct DevStats {
    unsigned long long render_rays, render_samples, render_hits;
    unsigned long long render_unique_corners;   // only with detail counters on
    unsigned long long fuse_updates, fuse_colour_updates, track_pixels;
};

// ------------------------------------------------------------- map layout
// Each map plane is stored linear (x fastest, then y, then z) with a
// one-voxel ghost border: voxel (x, y, z), x in [-1, nx], sits at
// (x + 1) + px ((y + 1) + py (z + 1)), and every ghost holds a copy of the
// edge voxel it clamps to.  A trilinear cell with lower corner (x0, y0, z0),
// x0 in [-1, nx - 1], then reads 8 values at fixed offsets {0, 1, px, px + 1,
// pxy, ...} from one base index, and gets exactly the values that clamping
// the corner indices to [0, n - 1] would give.
__device__ __forceinline__ uint32_t pad_index(const KParams& P, int x, int y, int z) {
    return (uint32_t)(x + 1) + P.px * ((uint32_t)(y + 1) + P.py * (uint32_t)(z + 1));
}

template <bool BF16>
__device__ __forceinline__ float map_load(const void* plane, uint32_t i) {
    if constexpr (BF16) {
        return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(plane) + i));
    } else {
        return __ldg(reinterpret_cast<const float*>(plane) + i);
    }
}
template <bool BF16>
__device__ __forceinline__ float map_load_rw(const void* plane, uint32_t i) {
    if constexpr (BF16) {
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(plane)[i]);
    } else {
        return reinterpret_cast<const float*>(plane)[i];
    }
}
// The value map_store<BF16> leaves in a plane for v (what a later load reads).
template <bool BF16>
__device__ __forceinline__ float map_round(float v) {
    if constexpr (BF16) return __bfloat162float(__float2bfloat16_rn(v));
    else return v;
}
template <bool BF16>
__device__ __forceinline__ void map_store(void* plane, uint32_t i, float v) {
    if constexpr (BF16) {
        reinterpret_cast<__nv_bfloat16*>(plane)[i] = __float2bfloat16_rn(v);
    } else {
        reinterpret_cast<float*>(plane)[i] = v;
    }
}

// --------------------------------------------------------- FP32 decision recipe
__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
    return __fmaf_rn(t, __fsub_rn(b, a), a);
}

// Camera-frame point of pixel (u, v) at z-depth z:
// (z * ((u - cx) * (1/fx)), z * ((v - cy) * (1/fy)), z).
__device__ __forceinline__ void backproject_rn(const KParams& P, int u, int v, float z, float out[3]) {
    out[0] = __fmul_rn(z, __fmul_rn(__fsub_rn((float)u, P.cx32), P.ifx32));
    out[1] = __fmul_rn(z, __fmul_rn(__fsub_rn((float)v, P.cy32), P.ify32));
    out[2] = z;
}

// Depth validity (App. F.3, reading R19): valid iff d > 0, finite, and every
// in-image 4-neighbour dn has |d - dn| <= disc (FP32).
__device__ __forceinline__ bool depth_valid(const KParams& P, const float* __restrict__ depth, int u, int v) {
    const int p = v * P.W + u;
    const float d = depth[p];
    bool ok = (d > 0.0f) && isfinite(d);
    if (ok && u > 0) ok = fabsf(__fsub_rn(d, depth[p - 1])) <= P.disc32;
    if (ok && u < P.W - 1) ok = fabsf(__fsub_rn(d, depth[p + 1])) <= P.disc32;
    if (ok && v > 0) ok = fabsf(__fsub_rn(d, depth[p - P.W])) <= P.disc32;
    if (ok && v < P.H - 1) ok = fabsf(__fsub_rn(d, depth[p + P.W])) <= P.disc32;
    return ok;
}

// y_r = fma(M_r0, x0, fma(M_r1, x1, fma(M_r2, x2, b_r)))
__device__ __forceinline__ void affine_rn(const float M[9], const float b[3], const float x[3], float y[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        y[r] = __fmaf_rn(M[3 * r], x[0], __fmaf_rn(M[3 * r + 1], x[1], __fmaf_rn(M[3 * r + 2], x[2], b[r])));
}

// ----------------------------------------------------------- FP64 pose recipe
// Poses enter the library normalised (host poses at the C ABI with the FP64
// operations of normalise_pose there; device poses by the value path), so
// the recipe needs no square root or division.  R(q) of a unit quaternion
// (w, x, y, z), products formed first:
//   R = [1 - 2(yy + zz), 2(xy - wz), 2(xz + wy);
//        2(xy + wz), 1 - 2(xx + zz), 2(yz - wx);
//        2(xz - wy), 2(yz + wx), 1 - 2(xx + yy)]
// rounded once to FP32 for the camera-to-world matrices, and combined for
//   world-to-camera  M = R^T, b = -((R0i t0 + R1i t1) + R2i t2),
//   pose -> anchor   M = Ra^T R, b = Ra^T (t - ta)  (sums in the order k = 0, 1, 2),
// each operation rounded once (dot3_rn), then rounded to FP32.

// (a0*b0 + a1*b1) + a2*b2, each operation rounded
__device__ __forceinline__ double dot3_rn(double a0, double b0, double a1, double b1, double a2, double b2) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a0, b0), __dmul_rn(a1, b1)), __dmul_rn(a2, b2));
}

// ------------------------------------------------- warp-parallel pose recipe
// GB300's FP64 pipe retires about one warp instruction per 64 cycles per
// SM sub-partition whatever the number of active lanes, so the FP64 chains
// below put independent entries into the lanes of one warp: every lane runs
// the same branch-free instruction stream on its own operands (selected by
// lane), and each entry is computed with exactly the operations of the
// recipe above.

// Entry e (0..8, row-major) of R(q): 2 (p + s r) with products
// p, r of two quaternion components, s = +-1, and 1 - that on the diagonal
// (a - b is evaluated as a + (-b), which IEEE rounds identically).
__device__ __forceinline__ double quat_R_entry_rn(double w, double x, double y, double z, int e) {
    // per entry: component indices (a, b, c, d) of p = q_a q_b, r = q_c q_d, sign of r, diagonal
    // 0: yy+zz D; 1: xy-wz; 2: xz+wy; 3: xy+wz; 4: xx+zz D; 5: yz-wx; 6: xz-wy; 7: yz+wx; 8: xx+yy D
    constexpr uint32_t kA = 0x19956u, kB = 0x1fdbau, kC = 0x20303u, kD = 0x267efu;   // 2 bits an entry
    constexpr uint32_t kNeg = 0x62u, kDiag = 0x111u;                                   // 1 bit an entry
    const int sh = 2 * e;
    auto pick = [&](uint32_t tab) {
        const uint32_t k = (tab >> sh) & 3u;
        return k == 0u ? w : (k == 1u ? x : (k == 2u ? y : z));
    };
    const double p = __dmul_rn(pick(kA), pick(kB));
    const double r = __dmul_rn(pick(kC), pick(kD));
    const double u = __dmul_rn(2.0, __dadd_rn(p, ((kNeg >> e) & 1u) ? -r : r));
    const double du = __dsub_rn(1.0, u);
    return ((kDiag >> e) & 1u) ? du : u;
}

// The FP32 camera-to-world, world-to-camera and pose-to-anchor matrices of
// the recipe above (R then t; M then b), computed by the 32
// lanes of one warp (all must call; lanes outside the outputs compute and
// discard).  out entries are written by lanes 0..11.
__device__ __forceinline__ void warp_mats_c2w(const double* pose, float* out) {
    const int lane = threadIdx.x & 31;
    const double Re = quat_R_entry_rn(pose[3], pose[4], pose[5], pose[6], lane < 9 ? lane : 0);
    if (lane < 9) out[lane] = (float)Re;
    else if (lane < 12) out[lane] = (float)pose[lane - 9];
}

__device__ __forceinline__ void warp_mats_w2c(const double* pose, float* out) {
    const int lane = threadIdx.x & 31;
    const double Re = quat_R_entry_rn(pose[3], pose[4], pose[5], pose[6], lane < 9 ? lane : 0);
    // out[3i + j] = R[3j + i]; out[9 + i] = -dot3(R[i], t0, R[3 + i], t1, R[6 + i], t2)
    const int e = lane < 9 ? 3 * (lane % 3) + lane / 3 : 0;
    const double tr = __shfl_sync(0xffffffffu, Re, e);
    const int i = lane >= 9 && lane < 12 ? lane - 9 : 0;
    const double a0 = __shfl_sync(0xffffffffu, Re, i), a1 = __shfl_sync(0xffffffffu, Re, 3 + i),
                 a2 = __shfl_sync(0xffffffffu, Re, 6 + i);
    const double bv = -dot3_rn(a0, pose[0], a1, pose[1], a2, pose[2]);
    if (lane < 9) out[lane] = (float)tr;
    else if (lane < 12) out[lane] = (float)bv;
}

__device__ __forceinline__ void warp_mats_rel(const double* pose, const double* anchor, float* out) {
    const int lane = threadIdx.x & 31;
    // lanes 0..8: R(pose) entries; lanes 9..17: R(anchor) entries
    const bool pa = lane < 9;
    const double* q = pa ? pose + 3 : anchor + 3;
    const double Re = quat_R_entry_rn(q[0], q[1], q[2], q[3], pa ? lane : (lane < 18 ? lane - 9 : 0));
    // element e = lane (< 12): i = row; M[i][j] = dot3(Ra[i], R[j], Ra[3+i], R[3+j], Ra[6+i], R[6+j]),
    // b[i] = dot3(Ra[i], d0, Ra[3+i], d1, Ra[6+i], d2) with d = t - ta
    const int e = lane < 12 ? lane : 0;
    const int i = e < 9 ? e / 3 : e - 9, j = e % 3;
    const double a0 = __shfl_sync(0xffffffffu, Re, 9 + i), a1 = __shfl_sync(0xffffffffu, Re, 12 + i),
                 a2 = __shfl_sync(0xffffffffu, Re, 15 + i);
    const double r0 = __shfl_sync(0xffffffffu, Re, j), r1 = __shfl_sync(0xffffffffu, Re, 3 + j),
                 r2 = __shfl_sync(0xffffffffu, Re, 6 + j);
    const bool mrow = e < 9;
    const double b0 = mrow ? r0 : __dsub_rn(pose[0], anchor[0]);
    const double b1 = mrow ? r1 : __dsub_rn(pose[1], anchor[1]);
    const double b2 = mrow ? r2 : __dsub_rn(pose[2], anchor[2]);
    const double v = dot3_rn(a0, b0, a1, b1, a2, b2);
    if (lane < 12) out[lane] = (float)v;
}

// --------------------------------------------------------- warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Warp reduce-scatter of 32 values per lane: on return v[0] of lane l holds
// the warp's sum of value l.  A butterfly: at offset w each lane keeps the
// half of its live values selected by bit w of its lane index and adds the
// partner's copy of that half (31 shuffles instead of 32 x 5 for 32 separate
// sums; the order of the additions is fixed).
__device__ __forceinline__ void warp_reduce_scatter32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = upper ? v[i] : v[i + w];
            const float keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
}

// The occupancy bounds (max v, max |v|) of the eight 4^3 sub-tiles of the
// 8^3 tile (bx, by, bz), from a 256-thread block whose thread t holds the
// voxel (t & 7, (t >> 3) & 7, (t >> 6) + 4 h) of the tile in v[h], a[h]
// (every thread must call it).  Sub-tile (sx, sy, sz) of the map's grid of
// 4^3 sub-tiles is stored at sx + 2 nbx (sy + 2 nby sz).  Warp w holds the
// y rows 4 (w & 1) .. + 3 of z layer w >> 1 of each half, and lane bit 2 is
// the x half: the other lane bits are reduced by shuffles, the four z layers
// of a half through shared memory.
__device__ __forceinline__ void subtile_bounds_store(const KParams& P, float2* tb, int bx, int by, int bz,
                                                     const float* v, const float* a) {
    __shared__ float s_v[2][8][2], s_a[2][8][2];   // [z half][warp][x half]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float m = v[h], am = a[h];
#pragma unroll
        for (int o = 1; o <= 16; o <<= 1) {
            if (o == 4) continue;
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        }
        if ((lane & ~4) == 0) {
            s_v[h][w][lane >> 2] = m;
            s_a[h][w][lane >> 2] = am;
        }
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int sx = threadIdx.x & 1, sy = (threadIdx.x >> 1) & 1, sz = threadIdx.x >> 2;
        float m = -INFINITY, am = 0.0f;
#pragma unroll
        for (int zl = 0; zl < 4; ++zl) {
            m = fmaxf(m, s_v[sz][2 * zl + sy][sx]);
            am = fmaxf(am, s_a[sz][2 * zl + sy][sx]);
        }
        tb[(2 * bx + sx) + 2 * P.nbx * ((2 * by + sy) + 2 * P.nby * (2 * bz + sz))] = make_float2(m, am);
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace prism
