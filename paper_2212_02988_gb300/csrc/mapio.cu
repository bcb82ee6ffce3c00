// mapio.cu — map initialisation and conversion between the caller's linear
// layout (z-major, x fastest, colour interleaved) and the padded planes
// (a ghost border holding copies of the edge voxels, prism_dev.cuh).
#include "kernels.h"
#include "prism_dev.cuh"
#include "render_dev.cuh"

namespace prism {

template <bool BF16>
__global__ void k_map_fill(KParams P, MapPlanes M, float occ, float rgb, float var, uint32_t n) {
    pdl_enter();
    // n = padded elements per plane; ghosts get the same prior values
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        map_store<BF16>(M.occ, i, occ);
        map_store<BF16>(M.r, i, rgb);
        map_store<BF16>(M.g, i, rgb);
        map_store<BF16>(M.b, i, rgb);
        map_store<BF16>(M.var_occ, i, var);
        map_store<BF16>(M.var_rgb, i, var);
    }
}

// Every padded element (ghosts included) takes the caller's value of the
// voxel it clamps to.
template <bool BF16>
__global__ void k_map_load(KParams P, MapPlanes M, const float* __restrict__ occ, const float* __restrict__ rgb,
                           const float* __restrict__ vo, const float* __restrict__ vr, uint32_t n) {
    pdl_enter();
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int gx = (int)(e % P.px) - 1, gy = (int)((e / P.px) % P.py) - 1, gz = (int)(e / P.pxy) - 1;
        const int x = min(max(gx, 0), P.nx - 1), y = min(max(gy, 0), P.ny - 1), z = min(max(gz, 0), P.nz - 1);
        const size_t i = ((size_t)z * P.ny + y) * P.nx + x;
        if (occ) map_store<BF16>(M.occ, e, occ[i]);
        if (rgb) {
            map_store<BF16>(M.r, e, rgb[3 * i]);
            map_store<BF16>(M.g, e, rgb[3 * i + 1]);
            map_store<BF16>(M.b, e, rgb[3 * i + 2]);
        }
        if (vo) map_store<BF16>(M.var_occ, e, vo[i]);
        if (vr) map_store<BF16>(M.var_rgb, e, vr[i]);
    }
}

template <bool BF16>
__global__ void k_map_store(KParams P, MapPlanes M, float* __restrict__ occ, float* __restrict__ rgb,
                            float* __restrict__ vo, float* __restrict__ vr, uint32_t n) {
    pdl_enter();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % P.nx, y = (i / P.nx) % P.ny, z = i / (P.nx * P.ny);
        const uint32_t b = pad_index(P, x, y, z);
        if (occ) occ[i] = map_load_rw<BF16>(M.occ, b);
        if (rgb) {
            rgb[3 * (size_t)i] = map_load_rw<BF16>(M.r, b);
            rgb[3 * (size_t)i + 1] = map_load_rw<BF16>(M.g, b);
            rgb[3 * (size_t)i + 2] = map_load_rw<BF16>(M.b, b);
        }
        if (vo) vo[i] = map_load_rw<BF16>(M.var_occ, b);
        if (vr) vr[i] = map_load_rw<BF16>(M.var_rgb, b);
    }
}

// One block per 8^3 tile: (max, max |.|) of the occupancy means of each of
// its 4^3 sub-tiles.
template <bool BF16>
__global__ void __launch_bounds__(256) k_tile_bounds(KParams P, MapPlanes M) {
    pdl_enter();
    const uint32_t tile = blockIdx.x;
    const int bx = tile % P.nbx, by = (tile / P.nbx) % P.nby, bz = tile / (P.nbx * P.nby);
    float m[2], a[2];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int within = threadIdx.x + 256 * half;
        m[half] = map_load<BF16>(M.occ, pad_index(P, bx * 8 + (within & 7), by * 8 + ((within >> 3) & 7),
                                                  bz * 8 + (within >> 6)));
        a[half] = fabsf(m[half]);
    }
    subtile_bounds_store(P, M.tb, bx, by, bz, m, a);
}

// One block per top-level brick: the brick bounds of every level below it
// (render_dev.cuh).
__global__ void __launch_bounds__(512) k_brick_bounds(KParams P, MapPlanes M) {
    pdl_enter();
    render_detail::brick_pyramid_block(P, M, blockIdx.x);
}

static unsigned int io_grid(uint32_t n) {
    uint32_t g = (n + 255) / 256;
    return g > 152u * 64u ? 152u * 64u : (g ? g : 1u);
}

cudaError_t launch_map_fill(const KParams& P, const MapPlanes& M, float occ, float rgb, float var, cudaStream_t s) {
    uint32_t n = P.npad;
    if (P.bf16) launch_pdl(k_map_fill<true>, io_grid(n), 256, s, P, M, occ, rgb, var, n);
    else launch_pdl(k_map_fill<false>, io_grid(n), 256, s, P, M, occ, rgb, var, n);
    return cudaGetLastError();
}

cudaError_t launch_map_load(const KParams& P, const MapPlanes& M, const float* occ, const float* rgb,
                            const float* var_occ, const float* var_rgb, cudaStream_t s) {
    uint32_t n = P.npad;
    if (P.bf16) launch_pdl(k_map_load<true>, io_grid(n), 256, s, P, M, occ, rgb, var_occ, var_rgb, n);
    else launch_pdl(k_map_load<false>, io_grid(n), 256, s, P, M, occ, rgb, var_occ, var_rgb, n);
    return cudaGetLastError();
}

cudaError_t launch_map_store(const KParams& P, const MapPlanes& M, float* occ, float* rgb, float* var_occ,
                             float* var_rgb, cudaStream_t s) {
    uint32_t n = (uint32_t)P.nx * P.ny * P.nz;
    if (P.bf16) launch_pdl(k_map_store<true>, io_grid(n), 256, s, P, M, occ, rgb, var_occ, var_rgb, n);
    else launch_pdl(k_map_store<false>, io_grid(n), 256, s, P, M, occ, rgb, var_occ, var_rgb, n);
    return cudaGetLastError();
}

// A frame in pinned host memory that the device maps (s0, s1: device views of
// it) copied by the SMs' own loads: n0 floats s0 -> d0, n1 floats s1 -> d1.
// Each thread has four 16-byte loads in flight per round (the host memory's
// latency is the bound); single floats where an address is not 16-byte
// aligned, and for the tail.
__global__ void __launch_bounds__(256) k_frame_upload(const float* __restrict__ s0, float* __restrict__ d0,
                                                      size_t n0, const float* __restrict__ s1,
                                                      float* __restrict__ d1, size_t n1) {
    pdl_enter();
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const float* src[2] = {s0, s1};
    float* dst[2] = {d0, d1};
    const size_t cnt[2] = {n0, n1};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float* s = src[a];
        float* d = dst[a];
        const size_t n = cnt[a];
        size_t done = 0;
        if (((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(d)) & 15) == 0) {
            const size_t nv = n / 4;
            const float4* s4 = reinterpret_cast<const float4*>(s);
            float4* d4 = reinterpret_cast<float4*>(d);
            size_t i = tid;
            for (; i + 3 * stride < nv; i += 4 * stride) {
                const float4 x0 = s4[i], x1 = s4[i + stride], x2 = s4[i + 2 * stride], x3 = s4[i + 3 * stride];
                d4[i] = x0;
                d4[i + stride] = x1;
                d4[i + 2 * stride] = x2;
                d4[i + 3 * stride] = x3;
            }
            for (; i < nv; i += stride) d4[i] = s4[i];
            done = nv * 4;
        }
        for (size_t i = done + tid; i < n; i += stride) d[i] = s[i];
    }
}

cudaError_t launch_frame_upload(const float* s0, float* d0, size_t n0, const float* s1, float* d1, size_t n1,
                                int blocks, cudaStream_t s) {
    k_frame_upload<<<blocks, 256, 0, s>>>(s0, d0, n0, s1, d1, n1);
    return cudaGetLastError();
}

cudaError_t launch_tile_bounds(const KParams& P, const MapPlanes& M, cudaStream_t s) {
    const unsigned int tiles = (unsigned int)(P.nbx * P.nby * P.nbz);
    if (P.bf16) launch_pdl(k_tile_bounds<true>, tiles, 256, s, P, M);
    else launch_pdl(k_tile_bounds<false>, tiles, 256, s, P, M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_brick_bounds(P, M, s);
}

cudaError_t launch_brick_bounds(const KParams& P, const MapPlanes& M, cudaStream_t s) {
    const unsigned int top = (unsigned int)(P.bb_len - P.bb_off[P.nlev]);
    return launch_pdl(k_brick_bounds, top, 512, s, P, M);
}

}  // namespace prism
