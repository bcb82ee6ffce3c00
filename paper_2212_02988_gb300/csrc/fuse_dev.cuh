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
// A voxel outside the update region is neither read nor written, and a
// tile whose bounding sphere misses the view frustum exits at once; every
// other tile refreshes its occupancy bound (kernels.h, MapPlanes::tb).
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
    const int bx = tile % P.nbx, by = (tile / P.nbx) % P.nby, bz = tile / (P.nbx * P.nby);
    if (CULL) {
        if (threadIdx.x == 0) s_skip = tile_outside_frustum(P, sM, sb, bx, by, bz);
        __syncthreads();
        if (s_skip) return;
    }
    const float fW1 = (float)(P.W - 1), fH1 = (float)(P.H - 1);
    unsigned int n_occ = 0, n_col = 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int within = threadIdx.x + 256 * half;
        const int x = bx * 8 + (within & 7), y = by * 8 + ((within >> 3) & 7), z = bz * 8 + (within >> 6);
        const uint32_t idx = pad_index(P, x, y, z);
        // ---- decisions (FP32 recipe) ----
        float pc[3] = {__fmaf_rn(__fadd_rn((float)x, 0.5f), P.vs32, P.o32[0]),
                       __fmaf_rn(__fadd_rn((float)y, 0.5f), P.vs32, P.o32[1]),
                       __fmaf_rn(__fadd_rn((float)z, 0.5f), P.vs32, P.o32[2])};
        float X[3];
        affine_rn(sM, sb, pc, X);
        bool upd = X[2] > 0.0f;
        float sdf = 0.0f;
        int pix = 0;
        if (upd) {
            const float iz = __fdiv_rn(1.0f, X[2]);
            const float u = __fmaf_rn(__fmul_rn(P.fx32, X[0]), iz, P.cx32);
            const float v = __fmaf_rn(__fmul_rn(P.fy32, X[1]), iz, P.cy32);
            const float nu = floorf(__fadd_rn(u, 0.5f)), nv = floorf(__fadd_rn(v, 0.5f));
            upd = nu >= 0.0f && nu <= fW1 && nv >= 0.0f && nv <= fH1;
            if (upd) {
                pix = (int)nv * P.W + (int)nu;
                upd = mask[pix] != 0;
                if (upd) {
                    sdf = __fsub_rn(depth[pix], X[2]);
                    upd = sdf >= -P.trunc32;
                }
            }
        }
        if (!upd) continue;
        const bool colour = fabsf(sdf) <= P.trunc32;
        // ---- Gaussian product (FP32) ----
        const float f = -fminf(sdf, P.trunc32);
        const float var = map_load_rw<BF16>(M.var_occ, idx);
        const float mu = map_load_rw<BF16>(M.occ, idx);
        const float vl = var * P.upd_prec32;
        const float inv = 1.0f / (1.0f + vl);
        const bool edge = x == 0 || y == 0 || z == 0 || x == P.nx - 1 || y == P.ny - 1 || z == P.nz - 1;
        const float mu1 = fmaf(vl, f, mu) * inv, var1 = var * inv;
        map_store<BF16>(M.occ, idx, mu1);
        map_store<BF16>(M.var_occ, idx, var1);
        if (edge) {
            fuse_detail::store_ghosts<BF16>(P, M.occ, x, y, z, map_load_rw<BF16>(M.occ, idx));
            fuse_detail::store_ghosts<BF16>(P, M.var_occ, x, y, z, map_load_rw<BF16>(M.var_occ, idx));
        }
        ++n_occ;
        if (colour) {
            const float cvar = map_load_rw<BF16>(M.var_rgb, idx);
            const float cl = cvar * P.upd_prec32;
            const float cinv = 1.0f / (1.0f + cl);
            const float* o = rgb + 3 * pix;
            map_store<BF16>(M.r, idx, fmaf(cl, o[0], map_load_rw<BF16>(M.r, idx)) * cinv);
            map_store<BF16>(M.g, idx, fmaf(cl, o[1], map_load_rw<BF16>(M.g, idx)) * cinv);
            map_store<BF16>(M.b, idx, fmaf(cl, o[2], map_load_rw<BF16>(M.b, idx)) * cinv);
            map_store<BF16>(M.var_rgb, idx, cvar * cinv);
            if (edge) {
                void* planes[4] = {M.r, M.g, M.b, M.var_rgb};
                for (int q = 0; q < 4; ++q) fuse_detail::store_ghosts<BF16>(P, planes[q], x, y, z, map_load_rw<BF16>(planes[q], idx));
            }
            ++n_col;
        }
    }
    // the occupancy bounds of the tile's 4^3 sub-tiles after this update (the
    // render's brick skipping)
    {
        float m[2], am[2];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int within = threadIdx.x + 256 * half;
            m[half] = map_load_rw<BF16>(M.occ, pad_index(P, bx * 8 + (within & 7), by * 8 + ((within >> 3) & 7),
                                                         bz * 8 + (within >> 6)));
            am[half] = fabsf(m[half]);
        }
        subtile_bounds_store(P, M.tb, bx, by, bz, m, am);
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
