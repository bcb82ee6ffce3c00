// kernels.h — host-callable launchers of the PRISM kernels (internal to the
// library; the public boundary is include/prism.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace prism {

struct KParams;
struct DevState;
struct DevStats;

// A pose given either by value (host-supplied) or by a device pointer to 7 doubles.
struct PoseArg {
    double p[7];
    const double* dev;
};

// Which FP32 matrices k_prep derives from an FP64 pose.
enum PrepKind : int {
    PREP_STATE = 0,   // c2w and w2c of the state mean
    PREP_AUX_C2W = 1, // aux = camera-to-world of the pose argument
    PREP_AUX_REL = 2, // aux = pose argument -> anchor camera
    PREP_REL = 3,     // rel = Gauss-Newton pose -> anchor camera
    PREP_REL_NEXT = 4 // as PREP_REL with the state mean's pose as the anchor's (the
                      // anchor rendered at the current mean, which may still be in flight)
};

// The six map planes (f32 or bf16 elements), each linear with a ghost border.
struct MapPlanes {
    void* occ;
    void* r;
    void* g;
    void* b;
    void* var_occ;
    void* var_rgb;
    // per 4^3 sub-tile: (max occupancy mean, max |occupancy mean|) over its
    // voxels, kept current by the fuse and by map fill / load; per 4^3 brick b
    // (the cells whose lower corner lies in sub-tile b): the same over
    // sub-tiles b + {0, 1}^3, derived from tb by launch_brick_bounds
    // (render_dev.cuh)
    float2* tb;
    float2* bb;
};

// The tile order of an anchor render and what the next one is planned from
// (render_plan_block, render_dev.cuh); tiles are 16x8 pixels, row-major.
struct RenderPlan {
    const int* order = nullptr;   // the tiles in launch order (a permutation), or null for row-major
    uint32_t* cost = nullptr;     // out, per tile: the sum over its warps of the largest march-step count
    float* rot = nullptr;         // out: this render's camera-to-world rotation and centre (12 floats)
};
struct RenderPlanIn {
    const uint32_t* cost;   // the last anchor render's RenderPlan::cost
    const float* rot_last;  // and its rotation and centre
    const float* depth_last;  // and its depth image (null: directions only)
    const float* c2w;       // the next anchor render's mats
    uint32_t* key;          // scratch, one word per tile
    int* order;             // out
};

// render.cu — mats: 12 FP32 values on the device (DevState::c2w or ::aux);
// anchor_src/anchor_dst: when given, block 0 copies the 7 pose doubles
// (the anchor's pose) from src to dst.
cudaError_t launch_render(const KParams& P, const float* mats, const MapPlanes& M, float* depth, float* rgb,
                          uint8_t* mask, int32_t* hitk, DevStats* stats, const double* anchor_src,
                          double* anchor_dst, bool detail, cudaStream_t s, const RenderPlan& plan = RenderPlan{});
// The next anchor render's tile order (one block).
cudaError_t launch_render_plan(const KParams& P, const RenderPlanIn& in, cudaStream_t s);
cudaError_t launch_depth_mask(const KParams& P, const float* depth, uint8_t* mask, cudaStream_t s);
// The render's compile-time plane-stride specialisation for P (0: none).
int render_px_specialisation(const KParams& P);
// The anchor's depth validity and packing in one pass.
cudaError_t launch_anchor_pack(const KParams& P, const float* depth, const float* rgb, float4* a0, float4* a1,
                               cudaStream_t s);

// track.cu — normal-equation passes of the localisation.
enum TrackMode : int { TRACK_EXPORT = 0, TRACK_GN = 1, TRACK_LAPLACE = 2, TRACK_ADAM = 3 };
// Evaluate the objective with the relative transform dev->rel (GN, Laplace)
// or dev->aux (export) against the packed anchor; the last block reduces
// the per-block partials in a fixed order and runs the mode's FP64 finish.
cudaError_t launch_track(const KParams& P, int mode, const float* o_depth,
                         const float* o_rgb, const uint8_t* o_mask, const float4* a0, const float4* a1,
                         DevState* dev, float* partials, unsigned int* counter, int max_blocks,
                         DevStats* stats, cudaStream_t s, bool pdl = true, uint8_t* mask_out = nullptr);
// Gauss-Newton passes 1 .. passes of a localisation in one cooperative
// launch (every block resident; a grid barrier between passes, the FP64
// finish in every block; track_item's COOP).  partials: two buffers of
// TRACK_NV_MAX x max_blocks floats; barrier: a counter this launch starts
// from zero (the caller clears it on the stream first).  Returns
// cudaErrorCooperativeLaunchTooLarge (launching nothing) when the grid
// cannot be resident at once.
cudaError_t launch_track_coop(const KParams& P, const float* o_depth, const float* o_rgb, const uint8_t* o_mask,
                              const float4* a0, const float4* a1, DevState* dev, float* partials,
                              unsigned int* barrier, int max_blocks, DevStats* stats, int passes, cudaStream_t s);
int track_grid(const KParams& P, int mode, int max_blocks);
// The grid launch_track uses for `mode` (one wave of the device at most).
int track_launch_grid(const KParams& P, int mode, int max_blocks);
constexpr int TRACK_NV_MAX = 50;   // FP32 values per block partial

// adam.cu — the paper's pose optimiser (App. F.2): Adam with momentum off on
// tangent coordinates xi at the prior mean, `steps` steps of `pixels` pixels
// (<= 256) drawn uniformly with SplitMix64 from `seed` (draws numbered from
// n_localised x steps x pixels); leaves dev->xi, dev->cur_pose and dev->rel
// for the Laplace pass.  One block.
struct AdamArgs {
    int steps, pixels;
    unsigned long long seed;
    double lr_t, lr_r, beta2, eps;
};
cudaError_t launch_adam(const KParams& P, const float* o_depth, const float* o_rgb, const uint8_t* o_mask,
                        const float4* a0, const float4* a1, DevState* dev, const AdamArgs& A, cudaStream_t s);

// state.cu — FP64 prediction and GN start; the FP32 matrices of a pose.
// pdl = false: a plain launch (for a kernel that follows an event wait, whose
// dependency must not be relaxed to the previous kernel of the stream).
cudaError_t launch_predict(const KParams& P, DevState* dev, const double* imu, int n, double dt,
                           cudaStream_t s, bool pdl = true);
cudaError_t launch_prep(DevState* dev, int kind, const PoseArg& pose, cudaStream_t s, bool pdl = true);
// The prediction followed, in the same block, by the PREP_REL_NEXT matrices of
// the prior's mean (a plain launch).
cudaError_t launch_predict_prep(const KParams& P, DevState* dev, const double* imu, int n, double dt,
                                cudaStream_t s);

// fuse.cu — the per-voxel map update with the world-to-camera matrices
// `w2c` (12 FP32 on the device, DevState::w2c).
cudaError_t launch_fuse(const KParams& P, const MapPlanes& M, const float* w2c, const float* depth,
                        const float* rgb, const uint8_t* mask, DevStats* stats, cudaStream_t s);
// The same update in two launches: the frustum test of every tile appends
// the tiles in view to `list` (ntiles ints), then a persistent grid updates
// only those; ctr (2 uints, zero between calls) counts them.  rejected
// (device int, nullable; DevState::rejected): nonzero lists no tile.
cudaError_t launch_fuse_listed(const KParams& P, const MapPlanes& M, const float* w2c, const float* depth,
                               const float* rgb, const uint8_t* mask, DevStats* stats, int* list, unsigned int* ctr,
                               const int* rejected, cudaStream_t s);

// mapio.cu — fill with the prior, and conversion between the caller's dense
// layout and the padded (ghost-bordered) device layout.
cudaError_t launch_map_fill(const KParams& P, const MapPlanes& M, float occ, float rgb, float var,
                            cudaStream_t s);
cudaError_t launch_map_load(const KParams& P, const MapPlanes& M, const float* occ, const float* rgb,
                            const float* var_occ, const float* var_rgb, cudaStream_t s);
cudaError_t launch_map_store(const KParams& P, const MapPlanes& M, float* occ, float* rgb, float* var_occ,
                             float* var_rgb, cudaStream_t s);
// A frame in mapped pinned host memory (s0, s1: its device views) copied to
// d0, d1 (n0, n1 floats) by the SMs' loads; a plain launch of `blocks`.
cudaError_t launch_frame_upload(const float* s0, float* d0, size_t n0, const float* s1, float* d1, size_t n1,
                                int blocks, cudaStream_t s);
// The tile bounds M.tb of the whole map (after a fill or a load), and the
// brick bounds M.bb derived from them (after any change of M.tb).
cudaError_t launch_tile_bounds(const KParams& P, const MapPlanes& M, cudaStream_t s);
cudaError_t launch_brick_bounds(const KParams& P, const MapPlanes& M, cudaStream_t s);

// rollout.cu — predictive rollouts (App. I): per candidate sequence one block
// chains k predictions (App. E.1/E.2) from the posterior of `src` on its own
// scratch state, each prior becoming the next state.  Frame f = seq k + i
// reads IMU rows row0[f] .. row0[f] + counts[f] - 1 and interval dts[f], and
// writes its state to out[f] and the FP32 camera-to-world matrices of its
// normalised pose mean to mats[12 f ..].  RollOut has prism_state's layout.
struct RollOut {
    double t[3], q[4], v[3], w[3];
    double cov[144];
    int32_t n_localised;
    int32_t flags;   // FLAG_PRIOR_NOTPD when the frame's pose prior was not PD
};
cudaError_t launch_rollout_states(const KParams& P, const DevState* src, DevState* scratch, int n_seq, int k,
                                  const double* imu, const long long* row0, const int* counts, const double* dts,
                                  RollOut* out, float* mats, cudaStream_t s);
// The render of `frames` poses in one launch (grid z = frame):
// frame f reads mats[12 f ..] and writes depth / rgb / hitk at f H W
// (f H W 3 for rgb); each output may be NULL.  frames <= 65535.
cudaError_t launch_render_frames(const KParams& P, const float* mats, int frames, const MapPlanes& M, float* depth,
                                 float* rgb, int32_t* hitk, DevStats* stats, cudaStream_t s);

// mapping.cu — gradient-descent mapping (the alternative to the closed-form
// update).  launch_map_loss: over one rendered frame (depth, rgb, hit mask of
// the render), where the render hit and obs_d is valid, the loss gradients
// (d - D) / sd^2 and (c - C) / sc^2 replace depth and rgb (0 elsewhere) and
// the loss terms are added to *loss.  launch_map_step: mu <- mu - lr (g +
// (mu - mu0) / prior_var) on every padded element of the occupancy (g_occ, N
// floats) and colour (g_rgb, 3N floats, linear layout) planes, the prior
// term of the loss added to *loss; the tile and brick bounds are left to the
// caller.
cudaError_t launch_map_loss(const KParams& P, float* depth, float* rgb, const uint8_t* mask, const float* obs_d,
                            const float* obs_c, double sd, double sc, double* loss, cudaStream_t s);
cudaError_t launch_map_step(const KParams& P, const MapPlanes& M, const float* g_occ, const float* g_rgb,
                            double lr_occ, double lr_rgb, double mu0_occ, double mu0_rgb, double prior_var,
                            double* loss, cudaStream_t s);

// render_bwd.cu — adjoint of the render at the pose whose matrices are in
// `mats` (DevState::aux); adds the pose gradient to dev->grad_pose.
cudaError_t launch_render_bwd(const KParams& P, const float* mats, const MapPlanes& M, const float* grad_depth,
                              const float* grad_rgb, float* grad_occ, float* grad_rgb_map, DevState* dev,
                              cudaStream_t s);

}  // namespace prism
