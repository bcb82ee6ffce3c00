// mapping.cu — gradient-descent mapping, the alternative to the closed-form
// map update that the paper compares against (Sec. 4.4, Fig. sdfvsvi): a
// rendering loss over frames with known poses, carried to the map means by
// the render adjoint (render_bwd.cu), and plain descent steps on the means.
#include "kernels.h"
#include "prism_dev.cuh"

namespace prism {

// Per pixel of one rendered frame: where the render hit (mask) and the
// observed depth is valid (finite, > 0), the loss gradients
// g_d = (d - D) / sd^2 and g_c = (c - C) / sc^2 replace the rendered depth
// and colour (0 elsewhere), and the loss terms (d - D)^2 / (2 sd^2) +
// |c - C|^2 / (2 sc^2) are added to *loss (FP64, one atomic a block).
__global__ void __launch_bounds__(256) k_map_loss(int npix, float* __restrict__ depth, float* __restrict__ rgb,
                                                  const uint8_t* __restrict__ mask, const float* __restrict__ obs_d,
                                                  const float* __restrict__ obs_c, float inv_sd2, float inv_sc2,
                                                  double half_inv_sd2, double half_inv_sc2, double* loss) {
    pdl_enter();
    __shared__ double part[8];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < npix) {
        const float D = obs_d[p];
        const bool v = mask[p] != 0 && isfinite(D) && D > 0.0f;
        float gd = 0.0f, gc[3] = {0.0f, 0.0f, 0.0f};
        if (v) {
            const float rd = depth[p] - D;
            gd = rd * inv_sd2;
            double lc = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float rc = rgb[3 * p + c] - obs_c[3 * p + c];
                gc[c] = rc * inv_sc2;
                lc += (double)rc * (double)rc;
            }
            l = (double)rd * (double)rd * half_inv_sd2 + lc * half_inv_sc2;
        }
        depth[p] = gd;
#pragma unroll
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = gc[c];
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        if (s != 0.0) atomicAdd(loss, s);
    }
}

// The descent step on every padded element (ghosts included, each from the
// voxel it clamps to, as the map load fills them):
//   mu <- mu - lr (g + (mu - mu0) / prior_var)
// for occupancy (g_occ, lr_occ, mu0_occ) and the three colour planes (g_rgb,
// lr_rgb, mu0_rgb).  The prior term of the loss, sum (mu - mu0)^2 /
// (2 prior_var) over the voxels before the step, is added to *loss.
template <bool BF16>
__global__ void __launch_bounds__(256) k_map_step(KParams P, MapPlanes M, const float* __restrict__ g_occ,
                                                  const float* __restrict__ g_rgb, float lr_occ, float lr_rgb,
                                                  float mu0_occ, float mu0_rgb, float inv_v0, double half_inv_v0,
                                                  double* loss, uint32_t n) {
    pdl_enter();
    __shared__ double part[8];
    double l = 0.0;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int gx = (int)(e % P.px) - 1, gy = (int)((e / P.px) % P.py) - 1, gz = (int)(e / P.pxy) - 1;
        const int x = min(max(gx, 0), P.nx - 1), y = min(max(gy, 0), P.ny - 1), z = min(max(gz, 0), P.nz - 1);
        const bool interior = gx == x && gy == y && gz == z;
        const size_t i = ((size_t)z * P.ny + y) * P.nx + x;
        {
            const float m = map_load_rw<BF16>(M.occ, e);
            const float dm = m - mu0_occ;
            if (interior) l += (double)dm * (double)dm;
            map_store<BF16>(M.occ, e, m - lr_occ * (g_occ[i] + dm * inv_v0));
        }
        void* planes[3] = {M.r, M.g, M.b};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float m = map_load_rw<BF16>(planes[c], e);
            const float dm = m - mu0_rgb;
            if (interior) l += (double)dm * (double)dm;
            map_store<BF16>(planes[c], e, m - lr_rgb * (g_rgb[3 * i + c] + dm * inv_v0));
        }
    }
    l *= half_inv_v0;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(loss, s);
    }
}

cudaError_t launch_map_loss(const KParams& P, float* depth, float* rgb, const uint8_t* mask, const float* obs_d,
                            const float* obs_c, double sd, double sc, double* loss, cudaStream_t s) {
    const int npix = P.W * P.H;
    return launch_pdl(k_map_loss, (npix + 255) / 256, 256, s, npix, depth, rgb, mask, obs_d, obs_c,
                      (float)(1.0 / (sd * sd)), (float)(1.0 / (sc * sc)), 0.5 / (sd * sd), 0.5 / (sc * sc), loss);
}

cudaError_t launch_map_step(const KParams& P, const MapPlanes& M, const float* g_occ, const float* g_rgb,
                            double lr_occ, double lr_rgb, double mu0_occ, double mu0_rgb, double prior_var,
                            double* loss, cudaStream_t s) {
    const uint32_t n = P.npad;
    uint32_t g = (n + 255) / 256;
    g = g > 152u * 32u ? 152u * 32u : g;
    const float inv_v0 = (float)(1.0 / prior_var);
    if (P.bf16)
        return launch_pdl(k_map_step<true>, g, 256, s, P, M, g_occ, g_rgb, (float)lr_occ, (float)lr_rgb,
                          (float)mu0_occ, (float)mu0_rgb, inv_v0, 0.5 / prior_var, loss, n);
    return launch_pdl(k_map_step<false>, g, 256, s, P, M, g_occ, g_rgb, (float)lr_occ, (float)lr_rgb,
                      (float)mu0_occ, (float)mu0_rgb, inv_v0, 0.5 / prior_var, loss, n);
}

}  // namespace prism
