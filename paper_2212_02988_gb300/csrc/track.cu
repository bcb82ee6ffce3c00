// track.cu — single-stream launches of the localisation passes; the device
// body is in track_dev.cuh.
#include "track_dev.cuh"

namespace prism {

// Two blocks per SM for the passes of every step (at most 128 registers).
// MASKGEN: the pass also evaluates the observation's depth validity and
// writes it to om_out (the first Gauss-Newton pass of a localisation).
template <int MODE, bool MASKGEN = false>
__global__ void __launch_bounds__(Block<MODE>::threads, 1)
    k_track(KParams P, const float* __restrict__ od, const float* __restrict__ orgb, const uint8_t* __restrict__ om,
            const float4* __restrict__ a0, const float4* __restrict__ a1, DevState* dev,
            float* __restrict__ partials, int pstride, unsigned int* __restrict__ counter,
            DevStats* __restrict__ stats, uint8_t* __restrict__ om_out) {
    pdl_enter();
    track_item<MODE, MASKGEN>(P, od, orgb, om, a0, a1, dev, partials, pstride, counter, stats, blockIdx.x, gridDim.x,
                              om_out);
}

// Gauss-Newton passes in one cooperative launch: the blocks stay resident
// from pass to pass (track_item's COOP); a pass that stops (a system not
// positive definite, a barrier timeout) stops every block, in the same pass.
__global__ void __launch_bounds__(Block<TRACK_GN>::threads, 1)
    k_track_coop(KParams P, const float* __restrict__ od, const float* __restrict__ orgb,
                 const uint8_t* __restrict__ om, const float4* __restrict__ a0, const float4* __restrict__ a1,
                 DevState* dev, float* __restrict__ partials, int pstride, unsigned int* __restrict__ barrier,
                 DevStats* __restrict__ stats, int passes) {
    pdl_enter();
    for (int pass = 0; pass < passes; ++pass)
        if (!track_item<TRACK_GN, false, true>(P, od, orgb, om, a0, a1, dev, partials, pstride, barrier, stats,
                                               blockIdx.x, gridDim.x, nullptr, pass))
            break;
}

// One wave: as many blocks as fit on the device at once (fewer partials for
// the last block to add), never more than the pixels need.
template <int MODE>
static int wave_blocks() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_track<MODE>, Block<MODE>::threads, 0);
        cached = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
    }
    return cached;
}

int track_grid(const KParams& P, int mode, int max_blocks) {
    const int threads = mode == TRACK_EXPORT ? Block<TRACK_EXPORT>::threads : Block<TRACK_GN>::threads;
    int need = (P.W * P.H + threads - 1) / threads;
    int cap = max_blocks < 32 * kMaxPerLane ? max_blocks : 32 * kMaxPerLane;
    int g = need < cap ? need : cap;
    return g > 0 ? g : 1;
}

int track_launch_grid(const KParams& P, int mode, int max_blocks) {
    const int grid = track_grid(P, mode, max_blocks);
    const int wave = mode == TRACK_GN ? wave_blocks<TRACK_GN>()
                                      : (mode == TRACK_LAPLACE ? wave_blocks<TRACK_LAPLACE>() : wave_blocks<TRACK_EXPORT>());
    return grid < wave ? grid : wave;
}

cudaError_t launch_track_coop(const KParams& P, const float* o_depth, const float* o_rgb, const uint8_t* o_mask,
                              const float4* a0, const float4* a1, DevState* dev, float* partials,
                              unsigned int* barrier, int max_blocks, DevStats* stats, int passes, cudaStream_t s) {
    static int resident = 0;   // blocks of k_track_coop the device holds at once
    if (!resident) {
        int d = 0, sms = 0, per = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_track_coop, Block<TRACK_GN>::threads, 0);
        resident = sms * per;
    }
    const int grid = track_launch_grid(P, TRACK_GN, max_blocks);
    if (grid > resident) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(Block<TRACK_GN>::threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_track_coop, P, o_depth, o_rgb, o_mask, a0, a1, dev, partials, max_blocks, barrier,
                              stats, passes);
}

cudaError_t launch_track(const KParams& P, int mode, const float* o_depth,
                         const float* o_rgb, const uint8_t* o_mask, const float4* a0, const float4* a1,
                         DevState* dev, float* partials, unsigned int* counter, int max_blocks,
                         DevStats* stats, cudaStream_t s, bool pdl, uint8_t* mask_out) {
    // the Laplace pass takes the Gauss-Newton passes' grid, so that its sums
    // see the pixels in the same order after either launch form of those
    // passes (prism_set_cooperative)
    const int grid = track_launch_grid(P, mode == TRACK_LAPLACE ? TRACK_GN : mode, max_blocks);
    if (mode == TRACK_GN && mask_out) {
        if (!pdl) {
            k_track<TRACK_GN, true><<<grid, Block<TRACK_GN>::threads, 0, s>>>(P, o_depth, o_rgb, o_mask, a0, a1, dev, partials,
                                                              max_blocks, counter, stats, mask_out);
            return cudaGetLastError();
        }
        return launch_pdl(k_track<TRACK_GN, true>, grid, Block<TRACK_GN>::threads, s, P, o_depth, o_rgb, o_mask, a0, a1, dev,
                          partials, max_blocks, counter, stats, mask_out);
    }
    switch (mode) {
        case TRACK_GN:
            if (!pdl) {
                k_track<TRACK_GN><<<grid, Block<TRACK_GN>::threads, 0, s>>>(P, o_depth, o_rgb, o_mask, a0, a1, dev, partials,
                                                            max_blocks, counter, stats, nullptr);
                break;
            }
            launch_pdl(k_track<TRACK_GN>, grid, Block<TRACK_GN>::threads, s, P, o_depth, o_rgb, o_mask, a0, a1, dev, partials,
                       max_blocks, counter, stats, (uint8_t*)nullptr);
            break;
        case TRACK_LAPLACE:
            launch_pdl(k_track<TRACK_LAPLACE>, grid, Block<TRACK_LAPLACE>::threads, s, P, o_depth, o_rgb, o_mask, a0, a1, dev, partials,
                       max_blocks, counter, stats, (uint8_t*)nullptr);
            break;
        default:
            launch_pdl(k_track<TRACK_EXPORT>, grid, Block<TRACK_EXPORT>::threads, s, P, o_depth, o_rgb, o_mask, a0, a1, dev, partials,
                       max_blocks, counter, stats, (uint8_t*)nullptr);
    }
    return cudaGetLastError();
}

}  // namespace prism
