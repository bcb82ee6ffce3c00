// noalloc.cu — prism_normal_equations_noalloc: one evaluation of the
// localisation normal equations for callers that cannot allocate device
// memory (for example code running where cudaMalloc is not allowed, or a
// host that must not grow its device footprint after start-up).
//
// It runs the same kernels as prism_anchor_load + prism_normal_equations
// (depth validity, anchor packing, pose matrices, the reduction pass), but
// every buffer those kernels need beyond the caller's inputs and outputs —
// the packed anchor, the observation's validity mask, the per-block partial
// sums, the ticket counter, the device state — lives in one file-scope static device
// array, g_noalloc_scratch, of PRISM_NOALLOC_SCRATCH_BYTES.  Each GPU that
// loads the library holds that array until the process exits.
//
// Host code may not hand the array's name to a kernel: on the host it only
// stands in for the symbol.  The device address is obtained once per device,
// with that device current, by cudaGetSymbolAddress on the first call made on
// that device, and cached for the life of the process.  A device reset
// (cudaDeviceReset) destroys the context that address belongs to; the entry
// point must not be called on that device after one.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "host_util.h"
#include "kernels.h"
#include "prism.h"
#include "prism_dev.cuh"

using namespace prism;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr int kMaxBlocks = 512;   // the reduction pass never uses more blocks than this
constexpr size_t kPix = PRISM_NOALLOC_MAX_PIXELS;

// Scratch layout (offsets in bytes, each 256-byte aligned).
constexpr size_t kOffState = 0;
constexpr size_t kOffCounter = align_up(kOffState + sizeof(DevState));
constexpr size_t kOffPartials = align_up(kOffCounter + sizeof(unsigned int));
constexpr size_t kOffA0 = align_up(kOffPartials + sizeof(float) * TRACK_NV_MAX * kMaxBlocks);
constexpr size_t kOffA1 = align_up(kOffA0 + 16 * kPix);
constexpr size_t kOffOMask = align_up(kOffA1 + 16 * kPix);
constexpr size_t kScratchBytes = align_up(kOffOMask + kPix);
static_assert(kScratchBytes <= PRISM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PRISM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

thread_local std::string g_noalloc_err;

prism_status fail(prism_status st, const std::string& m) {
    g_noalloc_err = m;
    return st;
}

// Device address of the scratch array on the current device (set up once).
prism_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(PRISM_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(PRISM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return PRISM_OK;
}

#define NA_CK(call, what)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(PRISM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

prism_status prism_normal_equations_noalloc(const prism_config* cfg, const double* anchor_pose7,
                                            const float* anchor_depth, const float* anchor_rgb,
                                            const double* pose7, const float* depth, const float* rgb,
                                            void* stream, double* out) {
    if (!cfg || !anchor_pose7 || !anchor_depth || !anchor_rgb || !pose7 || !depth || !rgb || !out)
        return fail(PRISM_EINVAL, "NULL argument");
    std::string why;
    if (!valid_track_config(cfg, why)) return fail(PRISM_EINVAL, "invalid config: " + why);
    if ((double)cfg->width * cfg->height > (double)kPix)
        return fail(PRISM_EINVAL, "image has " + std::to_string((long long)cfg->width * cfg->height) +
                                      " pixels; the allocation-free entry point supports at most " +
                                      std::to_string((long long)kPix));
    if (!finite_pose(anchor_pose7) || !finite_pose(pose7)) return fail(PRISM_EINVAL, "pose is not finite");
    int dev = 0;
    NA_CK(cudaGetDevice(&dev), "cudaGetDevice");
    unsigned char* base = nullptr;
    prism_status st = scratch_address(dev, &base);
    if (st != PRISM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    KParams P;
    fill_kparams(cfg, P);
    DevState* ds = (DevState*)(base + kOffState);
    unsigned int* counter = (unsigned int*)(base + kOffCounter);
    float* partials = (float*)(base + kOffPartials);
    float4* a0 = (float4*)(base + kOffA0);
    float4* a1 = (float4*)(base + kOffA1);
    uint8_t* o_mask = base + kOffOMask;
    // the ticket counter must start at zero; the rest is fully overwritten
    NA_CK(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s), "clear counter");
    double anc[7];
    normalise_pose(anchor_pose7, anc);
    NA_CK(cudaMemcpyAsync(ds->anchor_pose, anc, sizeof(anc), cudaMemcpyHostToDevice, s), "anchor pose");
    NA_CK(launch_anchor_pack(P, anchor_depth, anchor_rgb, a0, a1, s), "anchor pack");
    NA_CK(launch_depth_mask(P, depth, o_mask, s), "observation mask");
    PoseArg pa{};
    normalise_pose(pose7, pa.p);
    NA_CK(launch_prep(ds, PREP_AUX_REL, pa, s), "pose matrices");
    NA_CK(launch_track(P, TRACK_EXPORT, depth, rgb, o_mask, a0, a1, ds, partials, counter, kMaxBlocks, nullptr, s),
          "normal equations");
    NA_CK(cudaStreamSynchronize(s), "stream synchronize");
    NA_CK(cudaMemcpy(out, ds->ne_out, 80 * sizeof(double), cudaMemcpyDeviceToHost), "read normal equations");
    return PRISM_OK;
}

const char* prism_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

}  // extern "C"
