// Device check of the FP64 helpers of linalg64.cuh used by the localisation
// finish: rcp64 against CUDA's correctly rounded 1.0 / d, and
// warp_ldlt6_solve on given 6x6 systems.  Reads from stdin:
//   n_rcp, then n_rcp doubles (hex bit patterns);
//   n_sys, then per system 21 doubles of A's lower triangle (row-major,
//   entry (i, j) at i (i + 1) / 2 + j) and 6 of b.
// Writes to stdout: per double "rcp <bits of rcp64(d)> <bits of 1.0 / d>",
// per system "x <6 bit patterns> <pd>".
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

#include "linalg64.cuh"

using namespace prism;

__global__ void k_rcp(const double* d, double* a, double* b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        a[i] = rcp64(d[i]);
        b[i] = 1.0 / d[i];
    }
}

// one warp a system: lane e < 21 takes A's packed entry e, lane 21 + i takes b_i
__global__ void k_solve(const double* sys, double* x, int* pd, int n) {
    const int s = blockIdx.x;
    if (s >= n) return;
    const int lane = threadIdx.x;
    const double a = lane < 27 ? sys[27 * s + lane] : 0.0;
    bool ok;
    const double r = warp_ldlt6_solve(a, &ok);
    if (lane >= 21 && lane < 27) x[6 * s + lane - 21] = r;
    if (lane == 0) pd[s] = ok ? 1 : 0;
}

static uint64_t bits(double v) { uint64_t u; std::memcpy(&u, &v, 8); return u; }
static double of_bits(uint64_t u) { double v; std::memcpy(&v, &u, 8); return v; }

int main() {
    int n = 0;
    if (std::scanf("%d", &n) != 1 || n < 0 || n > (1 << 22)) return 2;
    std::vector<double> h(n), ha(n), hb(n);
    for (int i = 0; i < n; ++i) {
        unsigned long long u;
        if (std::scanf("%llx", &u) != 1) return 2;
        h[i] = of_bits(u);
    }
    int m = 0;
    if (std::scanf("%d", &m) != 1 || m < 0 || m > (1 << 20)) return 2;
    std::vector<double> hs(27 * (size_t)m), hx(6 * (size_t)m);
    std::vector<int> hpd(m);
    for (size_t i = 0; i < hs.size(); ++i) {
        unsigned long long u;
        if (std::scanf("%llx", &u) != 1) return 2;
        hs[i] = of_bits(u);
    }
    double *dd, *da, *db, *ds, *dx;
    int* dpd;
    if (cudaMalloc(&dd, 8 * (n + 1)) || cudaMalloc(&da, 8 * (n + 1)) || cudaMalloc(&db, 8 * (n + 1)) ||
        cudaMalloc(&ds, 8 * (hs.size() + 1)) || cudaMalloc(&dx, 8 * (hx.size() + 1)) || cudaMalloc(&dpd, 4 * (m + 1)))
        return 3;
    cudaMemcpy(dd, h.data(), 8 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(ds, hs.data(), 8 * hs.size(), cudaMemcpyHostToDevice);
    if (n) k_rcp<<<(n + 255) / 256, 256>>>(dd, da, db, n);
    if (m) k_solve<<<m, 32>>>(ds, dx, dpd, m);
    if (cudaDeviceSynchronize() != cudaSuccess) return 4;
    cudaMemcpy(ha.data(), da, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(hb.data(), db, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(hx.data(), dx, 8 * hx.size(), cudaMemcpyDeviceToHost);
    cudaMemcpy(hpd.data(), dpd, 4 * m, cudaMemcpyDeviceToHost);
    for (int i = 0; i < n; ++i)
        std::printf("rcp %016llx %016llx\n", (unsigned long long)bits(ha[i]), (unsigned long long)bits(hb[i]));
    for (int s = 0; s < m; ++s) {
        std::printf("x");
        for (int k = 0; k < 6; ++k) std::printf(" %016llx", (unsigned long long)bits(hx[6 * s + k]));
        std::printf(" %d\n", hpd[s]);
    }
    return 0;
}
