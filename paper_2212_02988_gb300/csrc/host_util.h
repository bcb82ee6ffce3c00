// host_util.h — host-side helpers shared by the single-stream ABI
// (prism_abi.cu) and the serving runtime (serve.cu).
#pragma once

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "prism.h"
#include "prism_dev.cuh"

namespace prism {

// An NVTX range over a scope of the host thread that enqueues the work (a
// no-op unless a tool such as Nsight Systems is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Checks a configuration; on failure `why` says what is wrong.
bool valid_config(const prism_config* c, std::string& why);
// Checks only the fields the localisation objective reads (image size,
// intrinsics, gates, Laplace scales, IRLS floors, discontinuity threshold);
// valid_config includes these checks.
bool valid_track_config(const prism_config* c, std::string& why);
// The kernels' parameter block of a configuration (FP32 copies are single
// roundings of the FP64 values).
void fill_kparams(const prism_config* c, KParams& k);
// q / sqrt(((w*w + x*x) + y*y) + z*z) with exactly these FP64 operations.
void normalise_pose(const double* in, double* out);
// All 7 values finite and a quaternion norm above 1e-10.
bool finite_pose(const double* p);

}  // namespace prism
