// serve.h — device tables and launcher of the batched filter step used by the
// serving runtime (serve.cu; public interface include/prism_serve.h).
//
// A batch is a set of streams, one pending request each.  Every kernel of
// the batched step is one persistent launch that walks the work items of all
// members — 16x8 render tiles, 256-pixel blocks, 8^3 voxel tiles, virtual
// blocks of the localisation passes — through prefix sums over the members,
// and runs on each item the same device body as the single-stream kernel
// (render_dev.cuh, track_dev.cuh, fuse_dev.cuh, state_dev.cuh).  The
// localisation passes of a member use the virtual grid its single-stream
// launch would use, so its partial sums, their order and hence its result
// are those of prism_step, whatever else shares the batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "prism_dev.cuh"

namespace prism {

constexpr int kServeMaxSlots = 64;
constexpr int kServeMaxCounters = 64;   // dynamic work counters per batch (n_gn + 2 used)

// One resident stream: parameters and device buffers (written once at
// admission into the device slot table).
struct SlotDesc {
    KParams P;
    MapPlanes M;
    DevState* dev;
    DevStats* stats;
    float* depth;              // frame staging of the current request (W x H)
    float* rgb;                // (W x H x 3)
    uint8_t* o_mask;
    float* a_depth;
    float* a_rgb;
    float4* a0;
    float4* a1;
    float* partials;           // localisation partials, value-major with stride pstride
    unsigned int* counter;     // ticket of the localisation passes
    int pstride;
    int grid_gn, grid_lap;     // virtual grids of the Gauss-Newton and Laplace passes
    int px_spec;               // render stride specialisation (render_px_specialisation)
    int tiles_x;               // render tiles along x
    int pad[3];
};

struct BatchMember {
    int slot;
    int localise;              // 0: the stream's first request (fuse and render only)
    int imu_off;               // offset of its IMU rows (x 7 doubles) in the batch's IMU array
    int n_imu;
    double dt;
};

// The batch, uploaded before each batched step (the counters start at 0).
struct BatchDesc {
    int n;                                  // members
    int n_loc;                              // members that localise
    int loc[kServeMaxSlots];                // their member indices
    int tiles_off[kServeMaxSlots + 1];      // prefix sums over members: render tiles
    int pix_off[kServeMaxSlots + 1];        // 256-pixel blocks
    int fuse_off[kServeMaxSlots + 1];       // 8^3 voxel tiles
    int brick_off[kServeMaxSlots + 1];      // top-level bricks
    int gn_off[kServeMaxSlots + 1];         // over localising members: Gauss-Newton virtual blocks
    int lap_off[kServeMaxSlots + 1];        // Laplace virtual blocks
    BatchMember m[kServeMaxSlots];
    unsigned int ctr[kServeMaxCounters];
};

// Per-member result, copied to the host after the step.
struct ServeOut {
    double t[3], q[4], v[3], w[3];
    double cov[144];
    int n_localised;
    int flags;
};

// Persistent grid sizes of the batched kernels (blocks), from the occupancy
// calculator at server creation.
struct BatchGrids {
    int pix, track_gn, track_lap, fuse, render, bricks;
};

cudaError_t batch_grids(bool bf16, BatchGrids* g);

// Enqueues the batched step (8 + n_gn kernels) on s.
cudaError_t launch_batch_step(const SlotDesc* slots, BatchDesc* batch, const double* imu, ServeOut* out, int n_gn,
                              bool bf16, const BatchGrids& g, cudaStream_t s);

}  // namespace prism
