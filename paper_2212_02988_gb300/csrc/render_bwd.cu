// render_bwd.cu — adjoint of the render of App. B (the emission is
// differentiable): gradients of  L = sum gD * depth + sum gC . rgb  with
// respect to the occupancy and colour means and to a world-frame
// perturbation of the camera pose (t' = t + dt, R' = Exp(dtheta) R).
//
// Nothing is stored by the forward: each thread re-marches its ray with the
// forward's FP32 recipe (so it finds the same hit sample k) and then, with
// alpha = (tau - f0) / (f1 - f0) between samples k-1 and k,
//   dL/dalpha = gD eps / |dir_c| + sum_c gC_c (C_c(p_k) - C_c(p_{k-1})),
//   dL/df0 = dL/dalpha (alpha - 1) / (f1 - f0),  dL/df1 = -dL/dalpha alpha / (f1 - f0),
// scatters each value's gradient to its 8 trilinear corners (FP32 atomics,
// the caller's linear map layout, edge corners clamped), and accumulates the
// pose gradient through the sample positions p_s = c + d_s r:
// dL/dt += gp_s, dL/dtheta += d_s (r x gp_s), gp_s = dL/dp_s.  The pose
// gradient is reduced per block and added to DevState::grad_pose in FP64.
#include "kernels.h"
#include "prism_dev.cuh"

namespace prism {

namespace {

struct Cell8 {
    int x0, x1, y0, y1, z0, z1;   // clamped corner coordinates
    uint32_t base;                // padded base index of the cell
    float fx, fy, fz;
};

__device__ __forceinline__ Cell8 cell8(const KParams& P, float gx, float gy, float gz) {
    const float flx = floorf(gx), fly = floorf(gy), flz = floorf(gz);
    Cell8 c;
    c.fx = __fsub_rn(gx, flx);
    c.fy = __fsub_rn(gy, fly);
    c.fz = __fsub_rn(gz, flz);
    const int ix = (int)flx, iy = (int)fly, iz = (int)flz;
    c.base = pad_index(P, ix, iy, iz);
    c.x0 = max(ix, 0); c.x1 = min(ix + 1, P.nx - 1);
    c.y0 = max(iy, 0); c.y1 = min(iy + 1, P.ny - 1);
    c.z0 = max(iz, 0); c.z1 = min(iz + 1, P.nz - 1);
    return c;
}

// The 8 corner values of a cell from a padded plane, order (x, y, z) bits.
template <bool BF16>
__device__ __forceinline__ void corners(const KParams& P, const void* plane, const Cell8& c, float v[8]) {
    const uint32_t b1 = c.base + P.px, b2 = c.base + P.pxy, b3 = b2 + P.px;
    v[0] = map_load<BF16>(plane, c.base); v[1] = map_load<BF16>(plane, c.base + 1);
    v[2] = map_load<BF16>(plane, b1);     v[3] = map_load<BF16>(plane, b1 + 1);
    v[4] = map_load<BF16>(plane, b2);     v[5] = map_load<BF16>(plane, b2 + 1);
    v[6] = map_load<BF16>(plane, b3);     v[7] = map_load<BF16>(plane, b3 + 1);
}

// Trilinear value (the forward's lerp order) and its gradient in cell units.
__device__ __forceinline__ float tri_value_grad(const float v[8], float fx, float fy, float fz, float g[3]) {
    const float c00 = lerp_rn(v[0], v[1], fx), c10 = lerp_rn(v[2], v[3], fx);
    const float c01 = lerp_rn(v[4], v[5], fx), c11 = lerp_rn(v[6], v[7], fx);
    const float c0 = lerp_rn(c00, c10, fy), c1 = lerp_rn(c01, c11, fy);
    const float dx00 = v[1] - v[0], dx10 = v[3] - v[2], dx01 = v[5] - v[4], dx11 = v[7] - v[6];
    g[0] = lerp_rn(lerp_rn(dx00, dx10, fy), lerp_rn(dx01, dx11, fy), fz);
    g[1] = lerp_rn(c10 - c00, c11 - c01, fz);
    g[2] = c1 - c0;
    return lerp_rn(c0, c1, fz);
}

// Add gval * (trilinear weight) to the 8 corners in the caller's linear layout.
__device__ __forceinline__ void scatter(const KParams& P, float* g, int stride, int ch, const Cell8& c, float gval) {
    const float wx[2] = {1.0f - c.fx, c.fx}, wy[2] = {1.0f - c.fy, c.fy}, wz[2] = {1.0f - c.fz, c.fz};
    const int xs[2] = {c.x0, c.x1}, ys[2] = {c.y0, c.y1}, zs[2] = {c.z0, c.z1};
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const size_t i = ((size_t)zs[e] * P.ny + ys[b]) * P.nx + xs[a];
                atomicAdd(g + i * stride + ch, gval * wx[a] * wy[b] * wz[e]);
            }
}

}  // namespace

template <bool BF16>
__global__ void __launch_bounds__(128) k_render_bwd(KParams P, const float* __restrict__ mats, MapPlanes M,
                                                    const float* __restrict__ gD, const float* __restrict__ gC,
                                                    float* __restrict__ g_occ, float* __restrict__ g_rgb,
                                                    DevState* __restrict__ dev) {
    pdl_enter();
    __shared__ float sR[9], sc[3];
    __shared__ float sred[4][6];
    if (threadIdx.x < 12) {
        if (threadIdx.x < 9) sR[threadIdx.x] = mats[threadIdx.x];
        else sc[threadIdx.x - 9] = mats[threadIdx.x];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int v = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    float gpose[6] = {0, 0, 0, 0, 0, 0};
    if (u < P.W && v < P.H) {
        const int p = v * P.W + u;
        const float gd = gD ? gD[p] : 0.0f;
        const float gc[3] = {gC ? gC[3 * p] : 0.0f, gC ? gC[3 * p + 1] : 0.0f, gC ? gC[3 * p + 2] : 0.0f};
        if (gd != 0.0f || gc[0] != 0.0f || gc[1] != 0.0f || gc[2] != 0.0f) {
            // ray set-up and march: the forward's FP32 recipe
            const float dx = __fmul_rn(__fsub_rn((float)u, P.cx32), P.ifx32);
            const float dy = __fmul_rn(__fsub_rn((float)v, P.cy32), P.ify32);
            const float w0 = __fmaf_rn(sR[0], dx, __fmaf_rn(sR[1], dy, sR[2]));
            const float w1 = __fmaf_rn(sR[3], dx, __fmaf_rn(sR[4], dy, sR[5]));
            const float w2 = __fmaf_rn(sR[6], dx, __fmaf_rn(sR[7], dy, sR[8]));
            const float inv_n = __fdiv_rn(1.0f, __fsqrt_rn(__fmaf_rn(w0, w0, __fmaf_rn(w1, w1, __fmul_rn(w2, w2)))));
            const float r0 = __fmul_rn(w0, inv_n), r1 = __fmul_rn(w1, inv_n), r2 = __fmul_rn(w2, inv_n);
            const float rgx = __fmul_rn(r0, P.inv_vs32), rgy = __fmul_rn(r1, P.inv_vs32), rgz = __fmul_rn(r2, P.inv_vs32);
            const float cgx = __fmaf_rn(__fsub_rn(sc[0], P.o32[0]), P.inv_vs32, -0.5f);
            const float cgy = __fmaf_rn(__fsub_rn(sc[1], P.o32[1]), P.inv_vs32, -0.5f);
            const float cgz = __fmaf_rn(__fsub_rn(sc[2], P.o32[2]), P.inv_vs32, -0.5f);
            const float hx = (float)P.nx - 0.5f, hy = (float)P.ny - 0.5f, hz = (float)P.nz - 0.5f;
            int k = 1;
            bool hit = false;
            for (; k <= P.kmax; ++k) {
                const float d = __fmul_rn((float)k, P.eps32);
                const float gx = __fmaf_rn(d, rgx, cgx), gy = __fmaf_rn(d, rgy, cgy), gz = __fmaf_rn(d, rgz, cgz);
                if (!(gx >= -0.5f && gx < hx && gy >= -0.5f && gy < hy && gz >= -0.5f && gz < hz)) break;
                const Cell8 c = cell8(P, gx, gy, gz);
                if (!PRISM_IN_RANGE(P, CHK_BWD_CORNER, (long long)c.base + P.pxy + P.px + 1, P.npad)) break;
                float vv[8], gg[3];
                corners<BF16>(P, M.occ, c, vv);
                if (tri_value_grad(vv, c.fx, c.fy, c.fz, gg) > P.tau32) { hit = true; break; }
            }
            if (hit && k >= 2) {
                Cell8 cs[2];
                float ds[2];
                for (int s = 0; s < 2; ++s) {
                    ds[s] = __fmul_rn((float)(k - 1 + s), P.eps32);
                    cs[s] = cell8(P, __fmaf_rn(ds[s], rgx, cgx), __fmaf_rn(ds[s], rgy, cgy),
                                  __fmaf_rn(ds[s], rgz, cgz));
                }
                if (PRISM_IN_RANGE(P, CHK_BWD_CORNER, (long long)cs[0].base + P.pxy + P.px + 1, P.npad) &&
                    PRISM_IN_RANGE(P, CHK_BWD_CORNER, (long long)cs[1].base + P.pxy + P.px + 1, P.npad)) {
                    float vo[2][8], go[2][3], f[2];
                    for (int s = 0; s < 2; ++s) {
                        corners<BF16>(P, M.occ, cs[s], vo[s]);
                        f[s] = tri_value_grad(vo[s], cs[s].fx, cs[s].fy, cs[s].fz, go[s]);
                    }
                    const float alpha = (P.tau32 - f[0]) / (f[1] - f[0]);
                    const void* planes[3] = {M.r, M.g, M.b};
                    float col[2][3], gcol[2][3][3];
                    for (int ch = 0; ch < 3; ++ch)
                        for (int s = 0; s < 2; ++s) {
                            float vc[8];
                            corners<BF16>(P, planes[ch], cs[s], vc);
                            col[s][ch] = tri_value_grad(vc, cs[s].fx, cs[s].fy, cs[s].fz, gcol[s][ch]);
                        }
                    float gA = gd * (ds[1] - ds[0]) * inv_n;
                    for (int ch = 0; ch < 3; ++ch) gA += gc[ch] * (col[1][ch] - col[0][ch]);
                    const float inv_df = 1.0f / (f[1] - f[0]);
                    const float gf[2] = {gA * (alpha - 1.0f) * inv_df, -gA * alpha * inv_df};
                    const float wa[2] = {1.0f - alpha, alpha};
                    const float r[3] = {r0, r1, r2};
                    for (int s = 0; s < 2; ++s) {
                        if (g_occ) scatter(P, g_occ, 1, 0, cs[s], gf[s]);
                        if (g_rgb)
                            for (int ch = 0; ch < 3; ++ch) scatter(P, g_rgb, 3, ch, cs[s], gc[ch] * wa[s]);
                        float gp[3];
                        for (int a = 0; a < 3; ++a) {
                            gp[a] = gf[s] * go[s][a];
                            for (int ch = 0; ch < 3; ++ch) gp[a] += gc[ch] * wa[s] * gcol[s][ch][a];
                            gp[a] *= P.inv_vs32;
                        }
                        // dL/dt += gp; dL/dtheta += d (r x gp)
                        gpose[0] += gp[0]; gpose[1] += gp[1]; gpose[2] += gp[2];
                        gpose[3] += ds[s] * (r[1] * gp[2] - r[2] * gp[1]);
                        gpose[4] += ds[s] * (r[2] * gp[0] - r[0] * gp[2]);
                        gpose[5] += ds[s] * (r[0] * gp[1] - r[1] * gp[0]);
                    }
                }
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        const float sum = warp_sum(gpose[i]);
        if (lane == 0) sred[warp][i] = sum;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const double s = (double)sred[0][threadIdx.x] + sred[1][threadIdx.x] + sred[2][threadIdx.x] +
                         sred[3][threadIdx.x];
        if (s != 0.0) atomicAdd(&dev->grad_pose[threadIdx.x], s);
    }
}

cudaError_t launch_render_bwd(const KParams& P, const float* mats, const MapPlanes& M, const float* grad_depth,
                              const float* grad_rgb, float* grad_occ, float* grad_rgb_map, DevState* dev,
                              cudaStream_t s) {
    dim3 grid((P.W + 15) / 16, (P.H + 7) / 8), block(128);
    if (P.bf16)
        launch_pdl(k_render_bwd<true>, grid, block, s, P, mats, M, grad_depth, grad_rgb, grad_occ, grad_rgb_map, dev);
    else
        launch_pdl(k_render_bwd<false>, grid, block, s, P, mats, M, grad_depth, grad_rgb, grad_occ, grad_rgb_map, dev);
    return cudaGetLastError();
}

}  // namespace prism
