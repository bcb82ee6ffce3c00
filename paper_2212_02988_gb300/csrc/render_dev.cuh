// render_dev.cuh — device bodies of the map-mean render of App. B and of the
// anchor it leaves for the localisation (App. E.3, App. F.3), shared by the
// single-stream kernels (render.cu) and the batched serving kernels
// (serve_kernels.cu).
//
// The render: one thread per pixel, 16x8-pixel blocks of 4 warps, each warp an
// 8x4 pixel tile so that a warp's rays stay close and their trilinear cells
// share cache lines.  Each ray marches d_k = k eps, k = 1, 2, ... through the
// occupancy plane (8 gathered corners per sample, FP32 lerps) and
// stops at the first sample with occupancy > tau (reading R1) or at the first
// sample outside the grid (R5).  The occupancy plane is linear with a ghost
// border (prism_dev.cuh), so a sample costs 8 loads at fixed offsets from
// one base index.  The hit depth and colour are the alpha
// interpolation between samples k-1 and k (App. B, R7); the colour planes are
// read only there.  The decision arithmetic follows the documented FP32
// recipe with explicitly rounded intrinsics (no contraction), so sample
// positions, corner indices and hit indices are reproducible bit for bit.
#pragma once

#include "kernels.h"
#include "prism_dev.cuh"

namespace prism {

namespace render_detail {

// Trilinear value at a cell given by its padded base index and in-cell
// weights: lerps along x, then y, then z (the FP32 recipe).  With PX > 0 the
// plane strides are compile-time constants (cubic grids of PX - 2 voxels a
// side), so the 8 loads are immediate offsets from one address.
template <bool BF16, int PX>
__device__ __forceinline__ float trilinear(const void* plane, uint32_t base, uint32_t px_rt, uint32_t pxy_rt,
                                           float fx, float fy, float fz) {
    const uint32_t px = PX > 0 ? (uint32_t)PX : px_rt;
    const uint32_t pxy = PX > 0 ? (uint32_t)(PX * PX) : pxy_rt;
    float v000, v100, v010, v110, v001, v101, v011, v111;
    if constexpr (BF16) {
        const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(plane) + base;
        v000 = __bfloat162float(__ldg(q)); v100 = __bfloat162float(__ldg(q + 1));
        v010 = __bfloat162float(__ldg(q + px)); v110 = __bfloat162float(__ldg(q + px + 1));
        v001 = __bfloat162float(__ldg(q + pxy)); v101 = __bfloat162float(__ldg(q + pxy + 1));
        v011 = __bfloat162float(__ldg(q + pxy + px)); v111 = __bfloat162float(__ldg(q + pxy + px + 1));
    } else {
        const float* q = reinterpret_cast<const float*>(plane) + base;
        v000 = __ldg(q); v100 = __ldg(q + 1);
        v010 = __ldg(q + px); v110 = __ldg(q + px + 1);
        v001 = __ldg(q + pxy); v101 = __ldg(q + pxy + 1);
        v011 = __ldg(q + pxy + px); v111 = __ldg(q + pxy + px + 1);
    }
    const float c00 = lerp_rn(v000, v100, fx);
    const float c10 = lerp_rn(v010, v110, fx);
    const float c01 = lerp_rn(v001, v101, fx);
    const float c11 = lerp_rn(v011, v111, fx);
    const float c0 = lerp_rn(c00, c10, fy);
    const float c1 = lerp_rn(c01, c11, fy);
    return lerp_rn(c0, c1, fz);
}

// Sample k of a ray in grid units: position g = fma(k eps, rg, cg), lower
// cell corner floor(g) as a padded base index, in-cell weights g - floor(g).
struct Sample {
    uint32_t base;
    float fx, fy, fz;
    int ix, iy, iz;   // lower corner (x0, y0, z0), x0 in [-1, n - 1]
};

// floor(g) for |g| < 2^22 without a conversion instruction: adding
// 1.5 * 2^23 with rounding toward -inf leaves floor(g) in the low mantissa
// bits (the sum's ulp is 1), and subtracting it back is exact.
constexpr float kFloorMagic = 12582912.0f;   // 1.5 * 2^23
constexpr uint32_t kFloorMagicBits = 0x4B400000u;

__device__ __forceinline__ Sample cell_of(uint32_t px, uint32_t pxy, float gx, float gy, float gz) {
    const float tx = __fadd_rd(gx, kFloorMagic), ty = __fadd_rd(gy, kFloorMagic), tz = __fadd_rd(gz, kFloorMagic);
    Sample s;
    s.fx = __fsub_rn(gx, __fsub_rn(tx, kFloorMagic));
    s.fy = __fsub_rn(gy, __fsub_rn(ty, kFloorMagic));
    s.fz = __fsub_rn(gz, __fsub_rn(tz, kFloorMagic));
    // (x0 + 1) + px ((y0 + 1) + py (z0 + 1)) with x0 = bits(tx) - magic, ...
    // in wrapping 32-bit arithmetic; the constant folds the offsets.
    const uint32_t c = (1u - kFloorMagicBits) * (1u + px + pxy);
    s.base = __float_as_uint(tx) + px * __float_as_uint(ty) + pxy * __float_as_uint(tz) + c;
    s.ix = (int)(__float_as_uint(tx) - kFloorMagicBits);
    s.iy = (int)(__float_as_uint(ty) - kFloorMagicBits);
    s.iz = (int)(__float_as_uint(tz) - kFloorMagicBits);
    return s;
}

// Brick skipping.  A cell whose lower corner x0 lies in brick b = max(x0, 0) / 4
// (per axis) reads corners from the 4^3 sub-tiles b and b + 1 only; brick_bound
// is the bound of those 8 sub-tiles (MapPlanes::bb).  A trilinear value is a convex
// combination of its corners, so if the bound is below tau by more than the
// lerps' rounding (7 lerps, each within ~3 2^-24 of the corners' magnitude:
// 2^-18 (1 + max |corner|) is a safe margin), no sample in the brick can be a
// hit and the march may jump over it.
__device__ __forceinline__ float2 brick_bound(const KParams& P, const float2* __restrict__ tb, int bx, int by,
                                              int bz) {
    const int sx = 2 * P.nbx, sy = 2 * P.nby, sz = 2 * P.nbz;
    const int bx1 = min(bx + 1, sx - 1), by1 = min(by + 1, sy - 1), bz1 = min(bz + 1, sz - 1);
    float m = -INFINITY, a = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = c & 1 ? bx1 : bx, y = c & 2 ? by1 : by, z = c & 4 ? bz1 : bz;
        const float2 t = tb[x + sx * (y + sy * z)];
        m = fmaxf(m, t.x);
        a = fmaxf(a, t.y);
    }
    return make_float2(m, a);
}

// The brick bounds below one top-level brick (level P.nlev, index `top`),
// one 512-thread block: level 0 from the sub-tile bounds (brick_bound), level
// l + 1 as the max of its 8 children at level l.  A level-l brick covers the
// cells whose lower corner lies in its (4 * 2^l)^3 box, and each child bound
// already includes the sub-tiles one step beyond it, so the max is the bound
// of the sub-tiles those cells read.
__device__ __forceinline__ void brick_pyramid_block(const KParams& P, const MapPlanes& M, int top) {
    __shared__ float2 s_b[2][512];
    const int N = P.nlev, s = 1 << N, t = threadIdx.x;
    const int d0x = 2 * P.nbx, d0y = 2 * P.nby;
    const int dNx = d0x >> N, dNy = d0y >> N;
    const int Tx = top % dNx, Ty = (top / dNx) % dNy, Tz = top / (dNx * dNy);
    if (t < s * s * s) {
        const int x = Tx * s + t % s, y = Ty * s + (t / s) % s, z = Tz * s + t / (s * s);
        const float2 b = brick_bound(P, M.tb, x, y, z);
        M.bb[x + d0x * (y + d0y * z)] = b;
        s_b[0][t] = b;
    }
    for (int l = 1; l <= N; ++l) {
        __syncthreads();
        const int sl = s >> l, sc = 2 * sl;   // level-l bricks and their children per axis in this block
        if (t < sl * sl * sl) {
            const int lx = t % sl, ly = (t / sl) % sl, lz = t / (sl * sl);
            const float2* ch = s_b[(l - 1) & 1];
            float m = -INFINITY, a = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float2 v = ch[(2 * lx + (c & 1)) + sc * ((2 * ly + ((c >> 1) & 1)) + sc * (2 * lz + (c >> 2)))];
                m = fmaxf(m, v.x);
                a = fmaxf(a, v.y);
            }
            const float2 r = make_float2(m, a);
            const int dlx = d0x >> l, dly = d0y >> l;
            M.bb[P.bb_off[l] + (Tx * sl + lx) + dlx * ((Ty * sl + ly) + dly * (Tz * sl + lz))] = r;
            s_b[l & 1][t] = r;
        }
    }
    __syncthreads();   // the shared levels are reused by the block's next item
}

__device__ __forceinline__ bool brick_skippable(const KParams& P, const float2* __restrict__ bb, int brick) {
    const float2 t = __ldg(bb + brick);
    return t.x < P.tau32 - 0x1p-18f * (1.0f + t.y);
}

// The first sample index at or after which the ray may leave the level-lv
// brick (bx, by, bz): the exit distance of its cell-corner box [e b, e b + e),
// e = 4 * 2^lv (lower bound -1 for b = 0), pulled 1e-3 voxels inside, over
// eps, plus one.  irg are the
// reciprocals of the ray's grid direction (0 where it is 0) and ieps = 1 / eps;
// the products stand in for the quotients, whose rounding (and that of the
// sample positions) is far below the 1e-3 voxel margin.  Every sample before
// the returned index has its cell in the brick.
__device__ __forceinline__ int brick_exit(const KParams& P, int lv, int bx, int by, int bz, float irgx, float irgy,
                                          float irgz, float cgx, float cgy, float cgz, float ieps) {
    constexpr float m = 1e-3f;
    const float e = (float)(4 << lv);
    float dmin = INFINITY;
    const int b3[3] = {bx, by, bz};
    const float ir3[3] = {irgx, irgy, irgz}, cg3[3] = {cgx, cgy, cgz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = b3[a] == 0 ? -1.0f : e * (float)b3[a];
        const float hi = e * (float)(b3[a] + 1);
        if (ir3[a] > 0.0f) dmin = fminf(dmin, (hi - m - cg3[a]) * ir3[a]);
        else if (ir3[a] < 0.0f) dmin = fminf(dmin, (lo + m - cg3[a]) * ir3[a]);
    }
    const float kn = floorf(dmin * ieps) + 1.0f;
    return kn < (float)(P.kmax + 1) ? (int)kn : P.kmax + 1;
}

}  // namespace render_detail

// One 16x8-pixel tile (128 threads; warp w covers the 8x4 pixels at
// ((w & 1) 8, (w >> 1) 4) of the tile).  sR / sc: camera-to-world rotation
// and centre in shared memory.  Returns the thread's march steps (jumps
// and evaluating steps; 0 outside the image), the anchor render's tile cost.
//
// The march tests the grid bounds only for samples after k_safe, which a
// conservative FP32 bound (one voxel of margin, far above the rounding of the
// bound and of the sample positions) keeps inside the grid, and (with
// P.skip) jumps over 4^3 bricks whose occupancy bound shows that no sample
// in them can be a hit.  The samples evaluated, their corner indices and
// the hit index are those of the one-loop march over every sample; the
// value of a jumped-over sample k - 1 is recomputed at the hit.  With NS > 1
// (not with DETAIL) the march evaluates NS consecutive samples per step, so
// that a long ray has NS samples' loads in flight; it may also evaluate up
// to NS - 1 samples past the hit, or inside a brick it would have jumped
// from, none of which can change the hit (the first sample above tau) or
// the outputs.  The sample count (DevStats::render_samples) leaves out
// the samples evaluated past the hit.
template <bool BF16, bool DETAIL, int PX, int NS = 1>
__device__ __forceinline__ int render_tile(const KParams& P, const float* sR, const float* sc, const MapPlanes& M,
                                            float* __restrict__ depth, float* __restrict__ rgb,
                                            uint8_t* __restrict__ mask, int32_t* __restrict__ hitk,
                                            DevStats* __restrict__ stats, int tile_x, int tile_y) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = tile_x * 16 + (warp & 1) * 8 + (lane & 7);
    const int v = tile_y * 8 + (warp >> 1) * 4 + (lane >> 3);
    const bool active = u < P.W && v < P.H;
    const uint32_t px = PX > 0 ? (uint32_t)PX : P.px;
    const uint32_t pxy = PX > 0 ? (uint32_t)(PX * PX) : P.pxy;

    int nsamp = 0, hk = 0, steps = 0;
    unsigned int uniq = 0;   // distinct occupancy corners of this ray (DETAIL only)
    float out_d = 0.0f, out_r = 0.0f, out_g = 0.0f, out_b = 0.0f;
    if (active) {
        // ray set-up (FP32 recipe)
        float dx = __fmul_rn(__fsub_rn((float)u, P.cx32), P.ifx32);
        float dy = __fmul_rn(__fsub_rn((float)v, P.cy32), P.ify32);
        float w0 = __fmaf_rn(sR[0], dx, __fmaf_rn(sR[1], dy, sR[2]));
        float w1 = __fmaf_rn(sR[3], dx, __fmaf_rn(sR[4], dy, sR[5]));
        float w2 = __fmaf_rn(sR[6], dx, __fmaf_rn(sR[7], dy, sR[8]));
        float inv_n = __fdiv_rn(1.0f, __fsqrt_rn(__fmaf_rn(w0, w0, __fmaf_rn(w1, w1, __fmul_rn(w2, w2)))));
        float rgx = __fmul_rn(__fmul_rn(w0, inv_n), P.inv_vs32);
        float rgy = __fmul_rn(__fmul_rn(w1, inv_n), P.inv_vs32);
        float rgz = __fmul_rn(__fmul_rn(w2, inv_n), P.inv_vs32);
        float cgx = __fmaf_rn(__fsub_rn(sc[0], P.o32[0]), P.inv_vs32, -0.5f);
        float cgy = __fmaf_rn(__fsub_rn(sc[1], P.o32[1]), P.inv_vs32, -0.5f);
        float cgz = __fmaf_rn(__fsub_rn(sc[2], P.o32[2]), P.inv_vs32, -0.5f);
        const float hx = (float)P.nx - 0.5f, hy = (float)P.ny - 0.5f, hz = (float)P.nz - 0.5f;

        // k_safe: every sample k <= k_safe stays one voxel inside the grid
        int k_safe = 0;
        if (cgx >= 0.5f && cgx <= hx - 1.0f && cgy >= 0.5f && cgy <= hy - 1.0f && cgz >= 0.5f &&
            cgz <= hz - 1.0f) {
            float ks = (float)P.kmax;
            const float rg3[3] = {rgx, rgy, rgz}, cg3[3] = {cgx, cgy, cgz}, h3[3] = {hx, hy, hz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (rg3[a] > 0.0f) ks = fminf(ks, (h3[a] - 1.0f - cg3[a]) / (rg3[a] * P.eps32));
                else if (rg3[a] < 0.0f) ks = fminf(ks, (0.5f - cg3[a]) / (rg3[a] * P.eps32));
            }
            k_safe = ks > 0.0f ? (int)ks : 0;
            k_safe = k_safe < P.kmax ? k_safe : P.kmax;
        }

        float f = 0.0f, f_prev = 0.0f;
        bool prev_ok = false;   // f_prev holds the value of sample k - 1
        int k = 1;
        float kf = 1.0f;        // (float)k, exact below 2^24
        bool hit = false;
        render_detail::Sample cur;
        float pfx = -2.0f, pfy = -2.0f, pfz = -2.0f;
        bool fresh = true;      // DETAIL: the next evaluated sample starts a new run of corners
        int cur_brick = -1;
        bool cur_skip = false;
        const bool skip = P.skip && M.bb != nullptr;
        // for the brick exits: 1 / rg (0 where rg = 0) and 1 / eps
        const float irgx = rgx != 0.0f ? 1.0f / rgx : 0.0f, irgy = rgy != 0.0f ? 1.0f / rgy : 0.0f,
                    irgz = rgz != 0.0f ? 1.0f / rgz : 0.0f, ieps = 1.0f / P.eps32;
        while (k <= P.kmax) {
            ++steps;
            const float d = __fmul_rn(kf, P.eps32);
            const float gx = __fmaf_rn(d, rgx, cgx), gy = __fmaf_rn(d, rgy, cgy), gz = __fmaf_rn(d, rgz, cgz);
            if (k > k_safe && !(gx >= -0.5f && gx < hx && gy >= -0.5f && gy < hy && gz >= -0.5f && gz < hz)) break;
            cur = render_detail::cell_of(px, pxy, gx, gy, gz);
            if (skip) {
                const int bx = max(cur.ix, 0) >> 2, by = max(cur.iy, 0) >> 2, bz = max(cur.iz, 0) >> 2;
                const int brick = bx + 2 * P.nbx * (by + 2 * P.nby * bz);
                if (brick != cur_brick) {
                    cur_brick = brick;
                    cur_skip = PRISM_IN_RANGE(P, CHK_RENDER_BRICK, brick, P.bb_len) &&
                               render_detail::brick_skippable(P, M.bb, brick);
                }
                if (cur_skip) {   // no sample of this brick can be a hit: jump past it, or past
                                  // the largest skippable brick above it (the bounds of the
                                  // ancestors are loaded together, then the unbroken chain
                                  // of skippable ones is climbed)
                    bool up[3];
#pragma unroll
                    for (int l = 1; l <= 3; ++l) {
                        up[l - 1] = false;
                        if (l <= P.nlev) {
                            const int dlx = (2 * P.nbx) >> l, dly = (2 * P.nby) >> l;
                            const int qi = P.bb_off[l] + (bx >> l) + dlx * ((by >> l) + dly * (bz >> l));
                            up[l - 1] = PRISM_IN_RANGE(P, CHK_RENDER_BRICK, qi, P.bb_len) &&
                                        render_detail::brick_skippable(P, M.bb, qi);
                        }
                    }
                    const int lv = up[0] ? (up[1] ? (up[2] ? 3 : 2) : 1) : 0;
                    const int kn = render_detail::brick_exit(P, lv, bx >> lv, by >> lv, bz >> lv, irgx, irgy, irgz,
                                                             cgx, cgy, cgz, ieps);
                    k = kn > k ? kn : k + 1;
                    kf = (float)k;
                    prev_ok = false;
                    fresh = true;
                    continue;
                }
            }
            ++nsamp;
            if (DETAIL) {   // consecutive cells share 8 >> (axes changed) corners (steps below one voxel)
                const float flx = floorf(gx), fly = floorf(gy), flz = floorf(gz);
                const int ch = (flx != pfx) + (fly != pfy) + (flz != pfz);
                uniq += fresh ? 8u : 8u - (8u >> ch);
                pfx = flx; pfy = fly; pfz = flz;
                fresh = false;
            }
            if (!PRISM_IN_RANGE(P, CHK_RENDER_CORNER, (long long)cur.base + pxy + px + 1, P.npad)) break;
            if constexpr (NS > 1 && !DETAIL) {
                // samples k .. k + NS - 1 together: their 8 NS corner loads are
                // in flight at once.  A sample past kmax or leaving the grid
                // ends the group (it re-reads sample k's corners, in bounds, and
                // is ignored); one in a skippable brick is evaluated (its value
                // cannot pass tau).  The first value above tau is the hit.
                render_detail::Sample cs[NS];
                bool ok[NS];
                float fv[NS];
                cs[0] = cur;
                ok[0] = true;
#pragma unroll
                for (int j = 1; j < NS; ++j) {
                    const float dj = __fmul_rn(kf + (float)j, P.eps32);
                    const float jx = __fmaf_rn(dj, rgx, cgx), jy = __fmaf_rn(dj, rgy, cgy), jz = __fmaf_rn(dj, rgz, cgz);
                    const render_detail::Sample sj = render_detail::cell_of(px, pxy, jx, jy, jz);
                    ok[j] = ok[j - 1] && k + j <= P.kmax &&
                            (k + j <= k_safe || (jx >= -0.5f && jx < hx && jy >= -0.5f && jy < hy && jz >= -0.5f && jz < hz)) &&
                            PRISM_IN_RANGE(P, CHK_RENDER_CORNER, (long long)sj.base + pxy + px + 1, P.npad);
                    cs[j] = cur;
                    if (ok[j]) cs[j] = sj;
                }
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    fv[j] = render_detail::trilinear<BF16, PX>(M.occ, cs[j].base, px, pxy, cs[j].fx, cs[j].fy, cs[j].fz);
                int jh = -1, nv = 1;
                float f_last = fv[0];
#pragma unroll
                for (int j = NS - 1; j >= 0; --j)
                    if (ok[j] && fv[j] > P.tau32) jh = j;
#pragma unroll
                for (int j = 1; j < NS; ++j)
                    if (ok[j]) { nv = j + 1; f_last = fv[j]; }
                if (jh >= 0) {
#pragma unroll
                    for (int j = 0; j < NS; ++j)
                        if (j == jh) {
                            f = fv[j];
                            if (j > 0) { f_prev = fv[j - 1]; prev_ok = true; cur = cs[j]; }
                        }
                    nsamp += jh;
                    k += jh;
                    hit = true;
                    break;
                }
                nsamp += nv - 1;
                f_prev = f_last;
                prev_ok = true;
                k += nv;
                kf += (float)nv;
                continue;
            }
            f = render_detail::trilinear<BF16, PX>(M.occ, cur.base, px, pxy, cur.fx, cur.fy, cur.fz);
            if (f > P.tau32) { hit = true; break; }
            f_prev = f;
            prev_ok = true;
            ++k;
            kf += 1.0f;
        }
        if (hit && k == 1) hk = -1;
        if (hit && k >= 2) {
            hk = k;
            // sample k - 1, recomputed exactly (same recipe) instead of carried along
            const float d1 = __fmul_rn((float)(k - 1), P.eps32);
            const render_detail::Sample prev = render_detail::cell_of(px, pxy, __fmaf_rn(d1, rgx, cgx), __fmaf_rn(d1, rgy, cgy),
                                        __fmaf_rn(d1, rgz, cgz));
            if (PRISM_IN_RANGE(P, CHK_RENDER_CORNER, (long long)prev.base + pxy + px + 1, P.npad)) {
                // sample k - 1 was jumped over: its value, by the same recipe
                if (!prev_ok) f_prev = render_detail::trilinear<BF16, PX>(M.occ, prev.base, px, pxy, prev.fx, prev.fy, prev.fz);
                const float alpha = __fdiv_rn(P.tau32 - f_prev, f - f_prev);
                const float dk = __fmul_rn((float)k, P.eps32);
                const float dstar = fmaf(alpha, dk - d1, d1);
                out_d = dstar * inv_n;
                float a1 = render_detail::trilinear<BF16, PX>(M.r, cur.base, px, pxy, cur.fx, cur.fy, cur.fz);
                float a0 = render_detail::trilinear<BF16, PX>(M.r, prev.base, px, pxy, prev.fx, prev.fy, prev.fz);
                out_r = fmaf(alpha, a1 - a0, a0);
                a1 = render_detail::trilinear<BF16, PX>(M.g, cur.base, px, pxy, cur.fx, cur.fy, cur.fz);
                a0 = render_detail::trilinear<BF16, PX>(M.g, prev.base, px, pxy, prev.fx, prev.fy, prev.fz);
                out_g = fmaf(alpha, a1 - a0, a0);
                a1 = render_detail::trilinear<BF16, PX>(M.b, cur.base, px, pxy, cur.fx, cur.fy, cur.fz);
                a0 = render_detail::trilinear<BF16, PX>(M.b, prev.base, px, pxy, prev.fx, prev.fy, prev.fz);
                out_b = fmaf(alpha, a1 - a0, a0);
            }
        }
        const int p = v * P.W + u;
        if (depth) depth[p] = out_d;
        if (rgb) { rgb[3 * p] = out_r; rgb[3 * p + 1] = out_g; rgb[3 * p + 2] = out_b; }
        if (mask) mask[p] = (uint8_t)(hk >= 2);
        if (hitk) hitk[p] = hk;
    }
    if (stats) {
        unsigned long long s = warp_sum_u64((unsigned long long)nsamp);
        unsigned int hits = __popc(__ballot_sync(0xffffffffu, hk >= 2));
        unsigned int rays = __popc(__ballot_sync(0xffffffffu, active));
        if (DETAIL) {
            const unsigned long long q = warp_sum_u64((unsigned long long)uniq);
            if (lane == 0) atomicAdd(&stats->render_unique_corners, q);
        }
        if (lane == 0) {
            atomicAdd(&stats->render_samples, s);
            atomicAdd(&stats->render_hits, (unsigned long long)hits);
            atomicAdd(&stats->render_rays, (unsigned long long)rays);
        }
    }
    return steps;
}

// The order of an anchor render's tiles, heaviest predicted first.  A ray's
// march length varies by two orders of magnitude across the image (rays
// grazing a surface evaluate a sample at every step of a long run of bricks
// that cannot be skipped); rendered in raster order, the heavy tiles start
// last and their blocks run on after the other SMs have emptied.  The
// prediction is the last anchor render's cost (per tile, the sum over its
// warps of the warp's largest count of march steps, jumps over empty bricks
// included) at the tile each tile's centre ray falls in when seen from the
// last camera -- the ray's direction, then its point at the depth the last
// render saw in that direction (the parallax of the centre's move) --
// maximised over its 3x3 tile neighbourhood; a ray outside the last image
// counts as heaviest.  Tiles go into 64 cost buckets, the buckets are laid out
// heaviest first; within a bucket the order is arbitrary.  The order only
// decides when a tile is rendered, never what it renders.  One block (a
// multiple of 32 threads); key: one word of scratch per tile.
__device__ __forceinline__ void render_plan_block(const KParams& P, const RenderPlanIn& in) {
    constexpr int kBuckets = 64;
    constexpr uint32_t kUnknown = 0xffffffffu;
    __shared__ uint32_t hist[kBuckets], base[kBuckets], s_max;
    const int gx = (P.W + 15) >> 4, gy = (P.H + 7) >> 3, nt = gx * gy;
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_max = 0u;
    // R = R_lastᵀ R_next: the next camera's ray directions in the last camera's
    // frame; dc = R_lastᵀ (c_next - c_last): the next centre there
    float R[9], dc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = in.rot_last[i] * in.c2w[j] + in.rot_last[3 + i] * in.c2w[3 + j] +
                           in.rot_last[6 + i] * in.c2w[6 + j];
        dc[i] = in.rot_last[i] * (in.c2w[9] - in.rot_last[9]) + in.rot_last[3 + i] * (in.c2w[10] - in.rot_last[10]) +
                in.rot_last[6 + i] * (in.c2w[11] - in.rot_last[11]);
    }
    __syncthreads();
    uint32_t lmax = 0u;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const float dx = ((float)((t % gx) * 16 + 8) - P.cx32) * P.ifx32;
        const float dy = ((float)((t / gx) * 8 + 4) - P.cy32) * P.ify32;
        const float ex = R[0] * dx + R[1] * dy + R[2], ey = R[3] * dx + R[4] * dy + R[5];
        const float ez = R[6] * dx + R[7] * dy + R[8];
        uint32_t e = kUnknown;
        if (ez > 1e-6f) {
            float u = P.fx32 * ex / ez + P.cx32, v = P.fy32 * ey / ez + P.cy32;
            if (in.depth_last && u >= 0.0f && u < (float)P.W && v >= 0.0f && v < (float)P.H) {
                // parallax: the ray's point at the depth the last render saw in that
                // direction, projected into the last camera from the next centre
                const float z0 = in.depth_last[min((int)v, P.H - 1) * P.W + min((int)u, P.W - 1)];
                const float sz = (z0 - dc[2]) / ez;
                if (z0 > 0.0f && sz > 0.0f) {
                    const float px = dc[0] + sz * ex, py = dc[1] + sz * ey, pz = dc[2] + sz * ez;
                    if (pz > 1e-6f) {
                        u = P.fx32 * px / pz + P.cx32;
                        v = P.fy32 * py / pz + P.cy32;
                    }
                }
            }
            if (u >= 0.0f && u < (float)P.W && v >= 0.0f && v < (float)P.H) {
                const int tx = min((int)u >> 4, gx - 1), ty = min((int)v >> 3, gy - 1);
                const int x0 = max(tx - 1, 0), x2 = min(tx + 1, gx - 1);
                const int y0 = max(ty - 1, 0), y2 = min(ty + 1, gy - 1);
                const uint32_t* r0 = in.cost + y0 * gx;
                const uint32_t* r1 = in.cost + ty * gx;
                const uint32_t* r2 = in.cost + y2 * gx;
                e = max(max(max(r0[x0], r0[tx]), max(r0[x2], r1[x0])), max(max(r1[tx], r1[x2]), max(r2[x0], r2[tx])));
                e = max(e, r2[x2]);
                lmax = max(lmax, e);
            }
        }
        in.key[t] = e;
    }
    lmax = __reduce_max_sync(0xffffffffu, lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, lmax);
    __syncthreads();
    const unsigned long long mx = s_max > 0u ? s_max : 1u;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {   // the same thread wrote key[t] above
        const uint32_t e = in.key[t];
        const uint32_t k = e == kUnknown ? kBuckets - 1 : (uint32_t)((unsigned long long)e * (kBuckets - 1) / mx);
        in.key[t] = k;
        atomicAdd(&hist[k], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0u;
        for (int k = kBuckets - 1; k >= 0; --k) {
            base[k] = run;
            run += hist[k];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const uint32_t pos = atomicAdd(&base[in.key[t]], 1u);
        if (PRISM_IN_RANGE(P, CHK_PLAN, pos, nt)) in.order[pos] = t;
    }
}

__device__ __forceinline__ void depth_mask_px(const KParams& P, const float* __restrict__ depth,
                                              uint8_t* __restrict__ mask, int p) {
    mask[p] = (uint8_t)depth_valid(P, depth, p % P.W, p / P.W);
}

// Anchor packing (App. E.3, reading R18): per pixel
//   a0 = (n_x, n_y, n_z, z)  with z = 0 where the normal is invalid,
//   a1 = (r, g, b, 1 if the depth is valid else 0).
// n = normalize((P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1))), facing the camera.
// anchor_pack_core takes the pixel's depth dc and its neighbours' (dr: u + 1,
// dl: u - 1, dd: v + 1, du: v - 1), its depth validity mc and ok = it and its
// four neighbours are valid inside the image border; the two packers below
// only differ in where those come from.
__device__ __forceinline__ void anchor_pack_core(const KParams& P, int u, int v, float dc, float dr, float dl,
                                                 float dd, float du, bool mc, bool ok,
                                                 const float* __restrict__ rgb, float4* __restrict__ a0,
                                                 float4* __restrict__ a1, int p) {
    float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
    if (ok) {
        float a[3], b[3], c[3], d[3], pc[3];
        backproject_rn(P, u + 1, v, dr, a);
        backproject_rn(P, u - 1, v, dl, b);
        backproject_rn(P, u, v + 1, dd, c);
        backproject_rn(P, u, v - 1, du, d);
        backproject_rn(P, u, v, dc, pc);
        float e1[3], e2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { e1[i] = __fsub_rn(a[i], b[i]); e2[i] = __fsub_rn(c[i], d[i]); }
        float c0 = __fsub_rn(__fmul_rn(e1[1], e2[2]), __fmul_rn(e1[2], e2[1]));
        float c1 = __fsub_rn(__fmul_rn(e1[2], e2[0]), __fmul_rn(e1[0], e2[2]));
        float c2 = __fsub_rn(__fmul_rn(e1[0], e2[1]), __fmul_rn(e1[1], e2[0]));
        float nn = __fmaf_rn(c0, c0, __fmaf_rn(c1, c1, __fmul_rn(c2, c2)));
        if (!(nn > 0.0f) || !isfinite(nn)) {
            ok = false;
        } else {
            float inv = __fdiv_rn(1.0f, __fsqrt_rn(nn));
            n0 = __fmul_rn(c0, inv); n1 = __fmul_rn(c1, inv); n2 = __fmul_rn(c2, inv);
            float dp = __fmaf_rn(n0, pc[0], __fmaf_rn(n1, pc[1], __fmul_rn(n2, pc[2])));
            if (dp > 0.0f) { n0 = -n0; n1 = -n1; n2 = -n2; }
        }
    }
    if (!ok) n0 = n1 = n2 = 0.0f;
    a0[p] = make_float4(n0, n1, n2, ok ? dc : 0.0f);
    a1[p] = make_float4(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2], mc ? 1.0f : 0.0f);
}

// One pixel from global memory (the validity of the pixel and of its four
// neighbours evaluated here by depth_valid).
__device__ __forceinline__ void anchor_pack_px(const KParams& P, const float* __restrict__ depth,
                                               const float* __restrict__ rgb, float4* __restrict__ a0,
                                               float4* __restrict__ a1, int p) {
    const int u = p % P.W, v = p / P.W, W = P.W;
    const bool mc = depth_valid(P, depth, u, v);
    const bool ok = u >= 1 && u <= P.W - 2 && v >= 1 && v <= P.H - 2 && mc && depth_valid(P, depth, u - 1, v) &&
                    depth_valid(P, depth, u + 1, v) && depth_valid(P, depth, u, v - 1) &&
                    depth_valid(P, depth, u, v + 1);
    const float dc = depth[p];
    float dr = 0.0f, dl = 0.0f, dd = 0.0f, du = 0.0f;
    if (ok) {
        dr = depth[p + 1];
        dl = depth[p - 1];
        dd = depth[p + W];
        du = depth[p - W];
    }
    anchor_pack_core(P, u, v, dc, dr, dl, dd, du, mc, ok, rgb, a0, a1, p);
}

// One 32x8-pixel tile on a block of 256 threads: the depths of the tile and
// a 2-pixel halo, then the validity of the tile and a 1-pixel halo, go
// through shared memory (one global read of each depth), with the
// comparisons of depth_valid.
constexpr int kPackTW = 32, kPackTH = 8;

__device__ __forceinline__ void anchor_pack_tile(const KParams& P, const float* __restrict__ depth,
                                                 const float* __restrict__ rgb, float4* __restrict__ a0,
                                                 float4* __restrict__ a1, int tile_x, int tile_y) {
    constexpr int DW = kPackTW + 4, DH = kPackTH + 4, VW = kPackTW + 2, VH = kPackTH + 2;
    __shared__ float sd[DH][DW];
    __shared__ uint8_t sv[VH][VW];
    const int W = P.W, H = P.H, x0 = tile_x * kPackTW, y0 = tile_y * kPackTH, t = threadIdx.x;
    for (int e = t; e < DW * DH; e += blockDim.x) {
        const int r = e / DW, c = e % DW, u = x0 - 2 + c, v = y0 - 2 + r;
        sd[r][c] = (u >= 0 && u < W && v >= 0 && v < H) ? depth[v * W + u] : 0.0f;
    }
    __syncthreads();
    for (int e = t; e < VW * VH; e += blockDim.x) {
        const int r = e / VW, c = e % VW, u = x0 - 1 + c, v = y0 - 1 + r;
        bool ok = false;
        if (u >= 0 && u < W && v >= 0 && v < H) {   // depth_valid on the tile
            const float d = sd[r + 1][c + 1];
            ok = (d > 0.0f) && isfinite(d);
            if (ok && u > 0) ok = fabsf(__fsub_rn(d, sd[r + 1][c])) <= P.disc32;
            if (ok && u < W - 1) ok = fabsf(__fsub_rn(d, sd[r + 1][c + 2])) <= P.disc32;
            if (ok && v > 0) ok = fabsf(__fsub_rn(d, sd[r][c + 1])) <= P.disc32;
            if (ok && v < H - 1) ok = fabsf(__fsub_rn(d, sd[r + 2][c + 1])) <= P.disc32;
        }
        sv[r][c] = (uint8_t)ok;
    }
    __syncthreads();
    const int tx = t % kPackTW, ty = t / kPackTW, u = x0 + tx, v = y0 + ty;
    if (ty < kPackTH && u < W && v < H) {
        const int r = ty + 1, c = tx + 1;   // in sv; in sd: r + 1, c + 1
        const bool mc = sv[r][c] != 0;
        const bool ok = u >= 1 && u <= W - 2 && v >= 1 && v <= H - 2 && mc && sv[r][c - 1] && sv[r][c + 1] &&
                        sv[r - 1][c] && sv[r + 1][c];
        const float dc = sd[r + 1][c + 1];
        float dr = 0.0f, dl = 0.0f, dd = 0.0f, du = 0.0f;
        if (ok) {
            dr = sd[r + 1][c + 2];
            dl = sd[r + 1][c];
            dd = sd[r + 2][c + 1];
            du = sd[r][c + 1];
        }
        anchor_pack_core(P, u, v, dc, dr, dl, dd, du, mc, ok, rgb, a0, a1, v * W + u);
    }
}

}  // namespace prism
