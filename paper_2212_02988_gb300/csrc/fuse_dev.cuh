// fuse_dev.cuh — device body of the per-voxel map update, shared by the
// single-stream kernel (fuse.cu) and the batched serving kernels
// (serve_kernels.cu).
//
// The closed-form per-voxel map update of App. D (Eq. mapupdategauss) at the
// current state mean, with the frustum and truncation rule of App. F.2.
// One block per 8x8x8 tile of voxels (256 threads, two voxels each); a warp
// touches four 8-voxel rows of each plane.  Updated voxels on the grid's
// edge also refresh their ghost copies (the render's clamped corners).
// Per voxel centre: camera point, nearest pixel, projective sdf = D - z
// (reading R9); the voxel is updated iff z > 0, the pixel is inside the
// image with valid depth (App. F.3) and sdf >= -trunc.  The Gaussian product
// with update precision Lu = 1/sigma_update^2 is written in variance form,
//   var' = var / (1 + var Lu),   mu' = (mu + var Lu f) / (1 + var Lu),
// which is Lambda' = Lambda + Lu, mu' = (Lambda mu + Lu f) / Lambda'.
// f_occ = -clamp(sdf, -trunc, trunc) (App. D: f_update = [-f_sdf, f_rgb]);
// colour (one shared variance, reading R11) only where |sdf| <= trunc (R10).
// A voxel outside the update region is not written (its occupancy is read
// for the tile's bound), and a tile whose bounding sphere misses the view
// frustum exits at once; every other tile refreshes its occupancy bounds
// (kernels.h, MapPlanes::tb).
#pragma once

#include "kernels.h"
#include "prism_dev.cuh"

namespace prism {

namespace fuse_detail {

// Copy value v of edge voxel (x, y, z) into its ghost cells (up to 7).
template <bool BF16>
__device__ void store_ghosts(const KParams& P, void* plane, int x, int y, int z, float v) {
    int gx[3], gy[3], gz[3], nx = 0, ny = 0, nz = 0;
    gx[nx++] = x; gy[ny++] = y; gz[nz++] = z;
    if (x == 0) gx[nx++] = -1;
    if (x == P.nx - 1) gx[nx++] = P.nx;
    if (y == 0) gy[ny++] = -1;
    if (y == P.ny - 1) gy[ny++] = P.ny;
    if (z == 0) gz[nz++] = -1;
    if (z == P.nz - 1) gz[nz++] = P.nz;
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < ny; ++b)
            for (int c = 0; c < nz; ++c)
                if (a | b | c) map_store<BF16>(plane, pad_index(P, gx[a], gy[b], gz[c]), v);
}

}  // namespace fuse_detail

// Conservative frustum cull of tile (bx, by, bz): its bounding sphere
// (centre c, radius r, with a margin far above FP32 rounding) lies entirely
// behind the camera or outside a side plane of the pixel range
// u, v in [-1/2, W - 1/2) x [-1/2, H - 1/2).  sM / sb: world-to-camera.
__device__ __forceinline__ bool tile_outside_frustum(const KParams& P, const float* sM, const float* sb, int bx,
                                                     int by, int bz) {
    const float h = 4.0f * P.vs32;
    const float cw[3] = {P.o32[0] + (8 * bx + 4) * P.vs32, P.o32[1] + (8 * by + 4) * P.vs32,
                         P.o32[2] + (8 * bz + 4) * P.vs32};
    float c[3];
    for (int r = 0; r < 3; ++r) c[r] = sM[3 * r] * cw[0] + sM[3 * r + 1] * cw[1] + sM[3 * r + 2] * cw[2] + sb[r];
    const float rad = 1.7321f * h * 1.001f + 1e-4f;
    bool out = c[2] < -rad;
    auto plane = [&](float a, float b) {   // half-space a * x_axis + b * z >= 0, unit-normalised
        return rsqrtf(a * a + b * b);
    };
    const float l0 = P.cx32 + 0.5f, l1 = (float)P.W - 0.5f - P.cx32;
    const float t0 = P.cy32 + 0.5f, t1 = (float)P.H - 0.5f - P.cy32;
    out = out || (P.fx32 * c[0] + l0 * c[2]) * plane(P.fx32, l0) < -rad;
    out = out || (-P.fx32 * c[0] + l1 * c[2]) * plane(P.fx32, l1) < -rad;
    out = out || (P.fy32 * c[1] + t0 * c[2]) * plane(P.fy32, t0) < -rad;
    out = out || (-P.fy32 * c[1] + t1 * c[2]) * plane(P.fy32, t1) < -rad;
    return out;
}

// The world-to-camera matrices into shared memory (12 threads; the caller
// synchronises before use).
__device__ __forceinline__ void load_w2c(const float* __restrict__ w2c, float* sM, float* sb) {
    if (threadIdx.x < 12) {
        if (threadIdx.x < 9) sM[threadIdx.x] = w2c[threadIdx.x];
        else sb[threadIdx.x - 9] = w2c[threadIdx.x];
    }
}

// One 8x8x8 tile (256 threads); sM / sb: the world-to-camera matrices in
// shared memory, loaded by the caller; CULL: test the frustum first (else the
// caller has listed only tiles that pass it).
template <bool BF16, bool CULL = true>
__device__ __forceinline__ void fuse_tile(const KParams& P, const MapPlanes& M, const float* sM, const float* sb,
                                          const float* __restrict__ depth, const float* __restrict__ rgb,
                                          const uint8_t* __restrict__ mask, DevStats* __restrict__ stats,
                                          uint32_t tile) {
    __shared__ int s_skip;
    if (!PRISM_IN_RANGE(P, CHK_FUSE_TILE, tile, (long long)P.nbx * P.nby * P.nbz)) return;   // block-uniform
    const int bx = tile % P.nbx, by = (tile / P.nbx) % P.nby, bz = tile / (P.nbx * P.nby);
    if (CULL) {
        if (threadIdx.x == 0) s_skip = tile_outside_frustum(P, sM, sb, bx, by, bz);
        __syncthreads();
        if (s_skip) return;
    }
    const float fW1 = (float)(P.W - 1), fH1 = (float)(P.H - 1);
    unsigned int n_occ = 0, n_col = 0;
    // The thread's two voxels go through each stage together, so that each
    // stage's loads are in flight at once: (1) decisions up to the pixel, and
    // the pixel's mask and depth; (2) the update decision, and the map values
    // (and observed colour) of the voxels updated; (3) the updates.  The
    // occupancy of every voxel is read in (1) for the tile's bounds, which
    // take the value each voxel holds after the update.
    int x[2], y[2], z[2], pix[2];
    uint32_t idx[2];
    float X2[2], dep[2], mu[2];
    bool in[2], mk[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int within = threadIdx.x + 256 * h;
        x[h] = bx * 8 + (within & 7);
        y[h] = by * 8 + ((within >> 3) & 7);
        z[h] = bz * 8 + (within >> 6);
        idx[h] = pad_index(P, x[h], y[h], z[h]);
        // ---- decisions (FP32 recipe) ----
        float pc[3] = {__fmaf_rn(__fadd_rn((float)x[h], 0.5f), P.vs32, P.o32[0]),
                       __fmaf_rn(__fadd_rn((float)y[h], 0.5f), P.vs32, P.o32[1]),
                       __fmaf_rn(__fadd_rn((float)z[h], 0.5f), P.vs32, P.o32[2])};
        float X[3];
        affine_rn(sM, sb, pc, X);
        X2[h] = X[2];
        bool ok = X[2] > 0.0f;
        pix[h] = 0;
        if (ok) {
            const float iz = __fdiv_rn(1.0f, X[2]);
            const float u = __fmaf_rn(__fmul_rn(P.fx32, X[0]), iz, P.cx32);
            const float v = __fmaf_rn(__fmul_rn(P.fy32, X[1]), iz, P.cy32);
            const float nu = floorf(__fadd_rn(u, 0.5f)), nv = floorf(__fadd_rn(v, 0.5f));
            ok = nu >= 0.0f && nu <= fW1 && nv >= 0.0f && nv <= fH1;
            if (ok) pix[h] = (int)nv * P.W + (int)nu;
            ok = ok && PRISM_IN_RANGE(P, CHK_FUSE_PIXEL, pix[h], (long long)P.W * P.H);
        }
        in[h] = ok;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        mk[h] = false;
        dep[h] = 0.0f;
        if (in[h]) {
            mk[h] = mask[pix[h]] != 0;
            dep[h] = depth[pix[h]];
        }
        mu[h] = PRISM_IN_RANGE(P, CHK_FUSE_VOXEL, idx[h], P.npad) ? map_load_rw<BF16>(M.occ, idx[h]) : 0.0f;
        if (!PRISM_IN_RANGE(P, CHK_FUSE_VOXEL, idx[h], P.npad)) mk[h] = false;
    }
    bool upd[2], colour[2];
    float sdf[2], var[2], cvar[2], cr[2], cg[2], cb[2], o0[2], o1[2], o2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        sdf[h] = mk[h] ? __fsub_rn(dep[h], X2[h]) : 0.0f;
        upd[h] = mk[h] && sdf[h] >= -P.trunc32;
        colour[h] = upd[h] && fabsf(sdf[h]) <= P.trunc32;
        if (upd[h]) var[h] = map_load_rw<BF16>(M.var_occ, idx[h]);
        if (colour[h]) {
            cvar[h] = map_load_rw<BF16>(M.var_rgb, idx[h]);
            cr[h] = map_load_rw<BF16>(M.r, idx[h]);
            cg[h] = map_load_rw<BF16>(M.g, idx[h]);
            cb[h] = map_load_rw<BF16>(M.b, idx[h]);
            const float* o = rgb + 3 * pix[h];
            o0[h] = o[0];
            o1[h] = o[1];
            o2[h] = o[2];
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!upd[h]) continue;
        // ---- Gaussian product (FP32) ----
        const float f = -fminf(sdf[h], P.trunc32);
        const float vl = var[h] * P.upd_prec32;
        const float inv = 1.0f / (1.0f + vl);
        const bool edge = x[h] == 0 || y[h] == 0 || z[h] == 0 || x[h] == P.nx - 1 || y[h] == P.ny - 1 ||
                          z[h] == P.nz - 1;
        const float mu1 = fmaf(vl, f, mu[h]) * inv, var1 = var[h] * inv;
        map_store<BF16>(M.occ, idx[h], mu1);
        map_store<BF16>(M.var_occ, idx[h], var1);
        mu[h] = map_round<BF16>(mu1);
        if (edge) {
            fuse_detail::store_ghosts<BF16>(P, M.occ, x[h], y[h], z[h], mu[h]);
            fuse_detail::store_ghosts<BF16>(P, M.var_occ, x[h], y[h], z[h], map_round<BF16>(var1));
        }
        ++n_occ;
        if (colour[h]) {
            const float cl = cvar[h] * P.upd_prec32;
            const float cinv = 1.0f / (1.0f + cl);
            const float r1 = fmaf(cl, o0[h], cr[h]) * cinv, g1 = fmaf(cl, o1[h], cg[h]) * cinv,
                        b1 = fmaf(cl, o2[h], cb[h]) * cinv, v1 = cvar[h] * cinv;
            map_store<BF16>(M.r, idx[h], r1);
            map_store<BF16>(M.g, idx[h], g1);
            map_store<BF16>(M.b, idx[h], b1);
            map_store<BF16>(M.var_rgb, idx[h], v1);
            if (edge) {
                fuse_detail::store_ghosts<BF16>(P, M.r, x[h], y[h], z[h], map_round<BF16>(r1));
                fuse_detail::store_ghosts<BF16>(P, M.g, x[h], y[h], z[h], map_round<BF16>(g1));
                fuse_detail::store_ghosts<BF16>(P, M.b, x[h], y[h], z[h], map_round<BF16>(b1));
                fuse_detail::store_ghosts<BF16>(P, M.var_rgb, x[h], y[h], z[h], map_round<BF16>(v1));
            }
            ++n_col;
        }
    }
    // the occupancy bounds of the tile's 4^3 sub-tiles after this update (the
    // render's brick skipping)
    {
        const float am[2] = {fabsf(mu[0]), fabsf(mu[1])};
        subtile_bounds_store(P, M.tb, bx, by, bz, mu, am);
    }
    if (stats) {
        unsigned int a = (unsigned int)warp_sum_u64(n_occ), b = (unsigned int)warp_sum_u64(n_col);
        if ((threadIdx.x & 31) == 0 && (a | b)) {
            atomicAdd(&stats->fuse_updates, (unsigned long long)a);
            atomicAdd(&stats->fuse_colour_updates, (unsigned long long)b);
        }
    }
}

}  // namespace prism
