/* prism.h — C ABI of the GB300 (sm_103a) PRISM filter hot path.
 *
 * PRISM (arXiv 2212.02988) filters a dense Gaussian voxel map and a 12-D
 * agent state from RGB-D frames and IMU readings.  One filter step for
 * frame t is (Sec. 3.3, App. F):
 *     prism_predict      state propagation from the IMU window   (App. E.1/E.2)
 *     prism_localise     MAP pose + Laplace covariance + velocity (App. E.3, Sec. 4.1, Sec. 3.3.2)
 *     prism_update_map   per-voxel Gaussian map update           (App. D, Eq. mapupdategauss)
 *     prism_render       render of the map mean = next anchor    (App. B)
 * (frame 1 only fuses and renders: the first state is given, Eq. 1).
 * prism_step runs the four in order as one stream of kernels.
 *
 * Conventions
 *   - World frame z up; camera frame +x right, +y down, +z forward.
 *   - A pose is 7 doubles (t_x, t_y, t_z, q_w, q_x, q_y, q_z): X_w = R(q) X_c + t.
 *     q need not be normalised; it is normalised before use.
 *   - Images are row-major, pixel (u, v) at index v * width + u; depth is
 *     camera z-depth in metres (<= 0 or non-finite = no return); colour is
 *     3 interleaved floats per pixel.
 *   - Map arrays exchanged with the caller are linear, z-major, x fastest:
 *     voxel (i, j, k) at index (k * ny + j) * nx + i; colour 3 interleaved
 *     floats per voxel.  Voxel (i, j, k) covers [o + i vs, o + (i + 1) vs).
 *   - "Device pointer" = memory of the handle's CUDA device (e.g. a torch
 *     tensor's data_ptr()); "host pointer" = ordinary CPU memory.
 *
 * Ownership and concurrency
 *   The library owns the map, the state, the anchor and its scratch buffers
 *   (allocated in prism_create_map, freed in prism_destroy).  It never frees
 *   caller memory and keeps no caller pointer after a call returns.  Every
 *   call enqueues work on the handle's CUDA stream and returns without
 *   waiting, unless it writes a host output (documented per call), in which
 *   case it synchronises the stream first.  Device buffers passed in must
 *   stay valid until the stream has passed the call.  A handle must not be
 *   used from two host threads at once; distinct handles are independent.
 *
 * Errors
 *   Every call returns a prism_status.  On a negative status the handle's
 *   state is unchanged where the error is detected on the host, and
 *   prism_last_error(h) describes it.  Failures found on the device (a
 *   normal-equation matrix that is not positive definite) leave the state
 *   unchanged and are reported by the next call that synchronises.  No call
 *   traps, asserts or aborts on the device.
 */
#ifndef PRISM_H
#define PRISM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PRISM_ABI_VERSION 1

typedef struct prism_ctx* prism_handle;

typedef enum {
    PRISM_OK = 0,
    PRISM_EINVAL = -1,    /* bad argument: NULL, size, shape, alignment */
    PRISM_ENOMEM = -2,    /* device or host allocation failed */
    PRISM_ECUDA = -3,     /* a CUDA runtime call failed */
    PRISM_ENOTPD = -4,    /* a normal-equation / covariance matrix was not positive definite */
    PRISM_ESTATE = -5     /* call out of order (e.g. localise before any anchor) */
} prism_status;

enum { PRISM_STORAGE_F32 = 0, PRISM_STORAGE_BF16 = 1 };

/* Pose optimiser of the localisation: Gauss-Newton on the IRLS form of the
 * objective (n_gn passes, the default), or the paper's Adam (App. F.2, "Pose
 * optimisation": momentum off, adam_steps steps of adam_pixels pixels drawn
 * uniformly, step sizes adam_lr_t / adam_lr_r). */
enum { PRISM_OPT_GAUSS_NEWTON = 0, PRISM_OPT_ADAM = 1 };

/* Filter configuration.  prism_config_default() fills the paper's values
 * (App. F.2, Tbl. transscales) for a cubic grid and an image size. */
typedef struct {
    int32_t nx, ny, nz;          /* voxels per axis, each a positive multiple of 8 */
    int32_t storage;             /* PRISM_STORAGE_F32 or PRISM_STORAGE_BF16 (map means and variances) */
    int32_t width, height;       /* frame size, pixels (>= 3 each) */
    int32_t n_gn;                /* Gauss-Newton iterations per frame (>= 1) */
    int32_t skip_empty;          /* 1: rays skip 4^3 bricks whose occupancy bound stays below tau
                                    (same outputs, fewer samples); 0: every sample is evaluated */
    double voxel;                /* voxel edge length vs, metres */
    double origin[3];            /* world position of the grid's minimum corner */
    double fx, fy, cx, cy;       /* pinhole intrinsics, pixel centres at integers */
    double eps;                  /* ray step (App. F.2: 0.4 vs) */
    double tau;                  /* hit threshold on occupancy (App. F.2: 0) */
    double max_depth;            /* longest ray distance, metres; <= 0: the grid bounds the ray */
    double trunc;                /* truncation distance (App. F.2: 2 vs) */
    double prior_var;            /* prior variance of every channel (App. B: sigma >> 1; 1e4) */
    double init_occ;             /* initial occupancy mean (App. F.2: -0.001) */
    double init_rgb;             /* initial colour mean (App. F.2: 0) */
    double update_var;           /* sigma_update^2 (App. F.2: 1) */
    double sigma_vel[2];         /* velocity transition scales, translation / rotation (0.03, 0.03) */
    double sigma_pose[2];        /* pose transition scales, translation / rotation (0.05, 0.02) */
    double b_geo, b_rgb;         /* Laplace scales of the objective (0.02 m, 0.1) */
    double gate_geo, gate_rgb;   /* residual gates (0.45, 0.15) */
    double floor_geo, floor_rgb; /* IRLS floor on |r| (1e-3 m, 1e-2) */
    double ema;                  /* Laplace covariance EMA coefficient (0.8) */
    double disc;                 /* depth discontinuity threshold, metres (0.1) */
    double gravity;              /* m/s^2 along world -z (9.81) */
    int32_t optimiser;           /* PRISM_OPT_GAUSS_NEWTON (default) or PRISM_OPT_ADAM */
    int32_t adam_steps;          /* Adam steps per frame (App. F.2: 1000) */
    int32_t adam_pixels;         /* pixels drawn per step, 1..256 (App. F.2: 200) */
    int32_t adam_reserved;       /* 0 */
    uint64_t adam_seed;          /* seed of the SplitMix64 pixel draws (draws numbered across frames) */
    double adam_lr_t, adam_lr_r; /* step sizes, translation / rotation (App. F.2: 1e-3, 3.6e-4) */
    double adam_beta2, adam_eps; /* second-moment decay and epsilon (unstated: Adam's 0.999, 1e-8) */
} prism_config;

/* Filter state (host copy).  cov is 12x12 row-major over the error state
 * (dt, dtheta, dv, dw), the rotation error applied on the left:
 * R = Exp(dtheta) R_mean; velocities (v linear, w angular) in the world frame. */
typedef struct {
    double t[3], q[4], v[3], w[3];
    double cov[144];
    int32_t n_localised;         /* frames localised so far (the EMA starts at the first) */
    int32_t reserved;
} prism_state;

/* Cumulative counters of the work done by a handle's kernels. */
typedef struct {
    int64_t render_rays;         /* rays rendered */
    int64_t render_samples;      /* ray samples evaluated (8 occupancy corners each) */
    int64_t render_hits;         /* rays with a valid hit (colour read at 2 x 8 corners) */
    int64_t fuse_updates;        /* voxels whose occupancy was updated */
    int64_t fuse_colour_updates; /* voxels whose colour was updated */
    int64_t track_pixels;        /* pixel evaluations of the localisation objective */
    int64_t render_unique_corners; /* distinct occupancy corners per ray, summed (only while
                                      detail counters are on; see prism_set_detail_counters) */
    int64_t kernel_launches;     /* CUDA kernels this handle has launched */
} prism_stats;

/* Per-phase device time (CUDA events on the handle's stream), in ms,
 * accumulated since the last prism_timing_reset; enabled by prism_set_timing. */
typedef struct {
    double predict_ms, localise_ms, fuse_ms, render_ms, anchor_ms;
    int64_t predict_n, localise_n, fuse_n, render_n, anchor_n;
    double laplace_ms;   /* the Laplace pass alone (inside localise_ms) */
    int64_t laplace_n;
} prism_timing;

/* Paper defaults for an n^3 grid of edge `extent` metres centred on the
 * origin and a width x height camera with fx = fy = 70 width / 80. */
void prism_config_default(prism_config* cfg, int32_t n, double extent, int32_t width, int32_t height);

/* Create a filter on the current CUDA device.  Allocates the map (prior
 * values: occupancy init_occ, colour init_rgb, variances prior_var), the
 * state (s1, copied; NULL = identity pose, zero velocity, 1e-8 I covariance)
 * and the scratch buffers.  `stream` is a cudaStream_t (NULL = legacy
 * default stream) on which every later call of this handle enqueues work.
 * Returns PRISM_EINVAL for a bad configuration, PRISM_ENOMEM if the device
 * allocation fails (nothing is leaked).  App. B (prior), Eq. 1 (s_1 given). */
prism_status prism_create_map(const prism_config* cfg, const prism_state* s1, void* stream,
                              prism_handle* out);

/* Synchronise the stream and free everything the handle owns. */
prism_status prism_destroy(prism_handle h);

/* Propagate the state over one frame interval dt > 0 with the IMU samples
 * of that interval (App. E.1 transition, Eq. statepropagation, App. E.2
 * split into pose prior and velocity conditional).  imu: HOST pointer to n
 * rows of 7 doubles (t, acc_x, acc_y, acc_z, gyro_x, gyro_y, gyro_z), specific
 * force in m/s^2 and angular rate in rad/s in the camera frame; n = 0 means
 * no controls (constant velocity).  The rows are copied before returning. */
prism_status prism_predict(prism_handle h, const double* imu, int32_t n, double dt);

/* Localise frame t against the current anchor (App. E.3 objective with the
 * gates and scales of App. F.2, Gauss-Newton with IRLS weights, FP64 6x6
 * Cholesky; Sec. 4.1 Laplace covariance with the App. F.2 EMA; Sec. 3.3.2
 * recombination with the velocity conditional).  Needs a prior from
 * prism_predict since the last localisation and an anchor (PRISM_ESTATE).
 * depth: DEVICE pointer, H x W floats; rgb: DEVICE pointer, H x W x 3 floats.
 * out: HOST pointer or NULL; when given, the stream is synchronised and the
 * new state written (this also reports PRISM_ENOTPD found on the device).
 * Divergence guard: when the prior's pose covariance, a Gauss-Newton system
 * or the Laplace Hessian is not positive definite (or not finite), the
 * localisation is rejected: the state stays exactly as it was, a following
 * map update of the same prism_step fuses nothing, and the state read
 * reports PRISM_ENOTPD.  Each prediction clears the device flags, so a
 * report covers the latest step only. */
prism_status prism_localise(prism_handle h, const float* depth, const float* rgb, prism_state* out);

/* Fuse a frame into the map at the current state mean (App. D, Eq.
 * mapupdategauss; frustum and truncation rule of App. F.2).  depth, rgb:
 * DEVICE pointers as for prism_localise. */
prism_status prism_update_map(prism_handle h, const float* depth, const float* rgb);

/* Render the map mean at a pose (App. B: ray points d = k eps, trilinear
 * field, first occupancy above tau, alpha-interpolated depth and colour).
 * pose7: HOST pointer to a pose, or NULL for the current state mean — in
 * which case the result also becomes the anchor of the next localisation.
 * depth (H x W floats, z-depth, 0 = no hit), rgb (H x W x 3 floats),
 * mask (H x W bytes, 1 = hit), hitk (H x W int32: index k >= 2 of the hit
 * sample, 0 = none, -1 = hit at the first sample): DEVICE pointers, each
 * may be NULL (not written). */
prism_status prism_render(prism_handle h, const double* pose7, float* depth, float* rgb,
                          uint8_t* mask, int32_t* hitk);

/* One full filter step (R21): predict (skipped on the first step), localise
 * (skipped on the first step), update_map, render of the new anchor.  A
 * rejected localisation (see prism_localise) leaves state and map unchanged
 * and returns PRISM_ENOTPD when out is given.
 * Arguments as for the individual calls; out may be NULL.  With out, the call
 * returns as soon as the posterior is final: the map update and the anchor
 * render may still be running on the stream, and they read depth and rgb, so
 * write those buffers again only in stream order (or after a
 * synchronisation). */
prism_status prism_step(prism_handle h, const double* imu, int32_t n, double dt,
                        const float* depth, const float* rgb, prism_state* out);

/* prism_step with the frame in HOST memory: depth_host (H x W floats) and
 * rgb_host (H x W x 3 floats) are copied into device buffers the handle
 * owns (two, used in turn).  After the first step the copies run on a copy
 * stream of the handle beside the prediction, so that the upload of frame t
 * overlaps frame t-1's map update and anchor render; the buffer a step
 * writes was last read two steps before, which the posterior of the step
 * before has already waited for.  Pinned host memory that the device maps
 * (cudaMallocHost / cudaHostAlloc under unified addressing) is read by a
 * copy kernel; other host memory goes through cudaMemcpyAsync, which
 * stages pageable memory before the call returns.  With out given the copies are
 * complete when the call returns; with out NULL they may still be in flight,
 * so keep the host frames unchanged until the next call on the handle
 * returns (which waits for them).  Otherwise as prism_step.  The first call
 * allocates the two buffers (PRISM_ENOMEM if it cannot). */
prism_status prism_step_host(prism_handle h, const double* imu, int32_t n, double dt,
                             const float* depth_host, const float* rgb_host, prism_state* out);

/* Copy the state to HOST memory (synchronises the stream; reports
 * PRISM_ENOTPD while the latest step's flags are raised). */
prism_status prism_get_state(prism_handle h, prism_state* out);

/* Replace the state (HOST pointer); the pending prior is discarded. */
prism_status prism_set_state(prism_handle h, const prism_state* s);

/* Load / store the whole map in the linear caller layout (see Conventions):
 * occ (N floats), rgb (3N floats), var_occ (N floats), var_rgb (N floats),
 * N = nx*ny*nz; DEVICE pointers; for storage BF16 the values are rounded
 * to nearest-even on load.  Either call may be given NULL for any array,
 * which is then left unchanged (load) or not written (store). */
prism_status prism_map_load(prism_handle h, const float* occ, const float* rgb,
                            const float* var_occ, const float* var_rgb);
prism_status prism_map_store(prism_handle h, float* occ, float* rgb, float* var_occ, float* var_rgb);

/* Make an externally rendered observation the anchor (as prism_render with
 * pose7 = NULL does for its own output): pose7 HOST pointer, depth and rgb
 * DEVICE pointers in the image layout.  The anchor's validity mask (App.
 * F.3) and normals (App. E.3) are computed from depth. */
prism_status prism_anchor_load(prism_handle h, const double* pose7, const float* depth,
                               const float* rgb);

/* One evaluation of the localisation objective at a camera pose against the
 * current anchor (App. E.3), reduced on the device: out (HOST, 80 doubles)
 * = H (36, row-major, sum w J^T J), g (6, sum w J^T r), Ht (36, sum J^T J / b^2),
 * cost (sum |r| / b), kept pixel count; J is the derivative with respect to
 * a world-frame perturbation t' = t + dt, R' = Exp(dtheta) R.  Synchronises. */
prism_status prism_normal_equations(prism_handle h, const double* pose7, const float* depth,
                                    const float* rgb, double* out);

/* ---- Allocation-free evaluation of the normal equations ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (code that must not call cudaMalloc, or a
 * process whose device footprint is fixed after start-up).  It computes
 * what prism_anchor_load followed by prism_normal_equations computes, without
 * a handle: anchor_pose7 and pose7 are HOST poses, anchor_depth / anchor_rgb
 * (the rendered anchor) and depth / rgb (the observation) are DEVICE pointers
 * in the image layout, `stream` a cudaStream_t (NULL = legacy default), out
 * a HOST array of 80 doubles laid out as for prism_normal_equations.  Only
 * cfg's image size, intrinsics, gates, scales, floors and disc are used and
 * checked.
 *
 * All scratch (packed anchor, the observation's validity mask, per-block
 * partial sums, ticket counter, device state) lives in one static device
 * array of PRISM_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits; the call allocates and frees nothing.  Images
 * larger than PRISM_NOALLOC_MAX_PIXELS are rejected with PRISM_EINVAL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it for the
 * life of the process: make that first call before any stream capture, and
 * do not call the entry point on a device after a cudaDeviceReset of it
 * (the cached address belonged to the destroyed context).  The device is
 * the caller's current device; all four image pointers must be on it.  Calls share the array and it keeps
 * the last call's contents: two calls whose work overlaps on the GPU (other
 * streams, other host threads) race and give wrong results; serialise them.
 * The call synchronises `stream` before returning.  Errors: as elsewhere,
 * with the message in prism_noalloc_last_error(). */
#define PRISM_NOALLOC_MAX_PIXELS (640 * 480)
#define PRISM_NOALLOC_SCRATCH_BYTES (10u * 1024u * 1024u + 256u * 1024u)
prism_status prism_normal_equations_noalloc(const prism_config* cfg, const double* anchor_pose7,
                                            const float* anchor_depth, const float* anchor_rgb,
                                            const double* pose7, const float* depth, const float* rgb,
                                            void* stream, double* out);
const char* prism_noalloc_last_error(void);

/* Adjoint of prism_render at pose7 (App. B: the emission is
 * differentiable): gradients of L = sum grad_depth * depth + sum grad_rgb .
 * rgb for the render of the current map at pose7.  grad_depth (H x W) and
 * grad_rgb (H x W x 3): DEVICE pointers, either may be NULL (zero).  Each
 * ray is re-marched (nothing is stored by the forward) and the hit sample
 * held fixed.  grad_occ (N floats) and grad_rgb_map (3N floats): DEVICE
 * pointers in the linear map layout, ACCUMULATED into (zero them first;
 * atomics, so the summation order varies), either may be NULL.
 * grad_pose6: HOST, 6 doubles (dL/dt, dL/dtheta for the world-frame left
 * perturbation t' = t + dt, R' = Exp(dtheta) R) or NULL; grad_pose7: HOST,
 * 7 doubles, the same gradient with respect to (t, q) of pose7 as given
 * (before normalisation), or NULL.  Either host output synchronises. */
prism_status prism_render_backward(prism_handle h, const double* pose7, const float* grad_depth,
                                   const float* grad_rgb, float* grad_occ, float* grad_rgb_map,
                                   double* grad_pose6, double* grad_pose7);

/* Predictive rollouts from the filter belief (App. I, "Prediction and
 * Control"; Fig. 1).  From the current posterior q(s_t) and the map mean,
 * each of n_seq candidate control sequences of k frames propagates the state
 * belief with the transition of prism_predict (App. E.1/E.2) and no
 * observation: a frame's prior (mean, velocities and the full 12x12
 * covariance) becomes the next frame's state.  Each frame also renders the
 * map mean (App. B) at its predicted pose mean, normalised as prism_render
 * normalises a pose, all frames in one launch.  The filter's state, prior,
 * anchor and map are left as they were.  Frame f = s k + i is frame i of
 * sequence s.
 * imu: HOST, the IMU rows of frames 0, 1, ... one after another (7 doubles
 *      a row, as in prism_predict), NULL when every count is 0.
 * counts: HOST, n_seq k row counts (>= 0; 0 = no controls, constant velocity).
 * dt: HOST, n_seq k frame intervals (finite, > 0).
 * states: HOST, n_seq k records, or NULL; when given, the stream is
 *      synchronised and frame f's predicted state written to states[f].
 * depth (n_seq k H W floats), rgb (n_seq k H W 3 floats), hitk (n_seq k H W
 *      int32, the hit sample index as prism_render reports it): DEVICE
 *      pointers, frame-major, each may be NULL; with all three NULL nothing
 *      is rendered.  The render adds to the work counters but not to the
 *      detail counters.
 * The inputs are copied before the call returns.  Returns PRISM_EINVAL for
 * n_seq < 1, k < 1, n_seq k > 65535 or a bad count, interval or IMU value;
 * PRISM_ENOTPD when a predicted pose covariance was not positive definite
 * (reported only with states; the records are still written). */
prism_status prism_rollout(prism_handle h, int32_t n_seq, int32_t k, const double* imu, const int32_t* counts,
                           const double* dt, prism_state* states, float* depth, float* rgb, int32_t* hitk);

/* One step of gradient-descent mapping, the alternative to the closed-form
 * map update that the paper compares against (Sec. 4.4, Fig. sdfvsvi), over
 * n frames with known poses.  For each frame the map mean is rendered at its
 * pose (App. B); where the render hits and the observed depth is valid
 * (finite, > 0) the loss gains (d - D)^2 / (2 sd^2) + |c - C|^2 / (2 sc^2),
 * and the render adjoint carries its gradient to the occupancy and colour
 * means, summed over the frames.  With the App. B prior (mean init_occ /
 * init_rgb, variance prior_var) every mean then takes the step
 * mu <- mu - lr (g + (mu - mu0) / prior_var), lr_occ for occupancy and
 * lr_rgb for colour; variances are not changed.  The frames are those of
 * the map before the step (all frames first, then one update).
 * poses: HOST, n x 7 (t, q); depth (n x H x W floats) and rgb (n x H x W x 3
 * floats): DEVICE.  sd, sc > 0; lr_occ, lr_rgb >= 0.  loss: HOST, 1 double,
 * the loss before the step (data and prior terms), or NULL; when given the
 * stream is synchronised.  The first call allocates the gradient and render
 * buffers (PRISM_ENOMEM if it cannot).  PRISM_EINVAL for n < 1, a pose that
 * is not finite or has a zero quaternion, or a bad scale or step size. */
prism_status prism_map_descent(prism_handle h, int32_t n, const double* poses, const float* depth,
                               const float* rgb, double sd, double sc, double lr_occ, double lr_rgb,
                               double* loss);

/* Work counters and per-phase timing.  Detail counters (off by default)
 * make the render also count the distinct trilinear corners each ray
 * reads, at a few instructions per sample. */
prism_status prism_get_stats(prism_handle h, prism_stats* out);
prism_status prism_set_timing(prism_handle h, int32_t enabled);
prism_status prism_set_detail_counters(prism_handle h, int32_t enabled);
prism_status prism_get_timing(prism_handle h, prism_timing* out);   /* synchronises */
prism_status prism_timing_reset(prism_handle h);

/* The Gauss-Newton localisation's launch form.  enabled = 1 (the default):
 * the passes after the first run as one cooperative launch (every block
 * resident, a grid barrier between passes, each block repeating the FP64
 * finish), where the device holds that grid at once.  enabled = 0: one
 * launch per pass.  Both forms evaluate the same sums in the same order and
 * give the same bits. */
prism_status prism_set_cooperative(prism_handle h, int32_t enabled);

/* Bounds-check build.  libprism_checked.so is this library compiled with
 * PRISM_CHECKED: its kernels test the data-dependent index of every gather
 * and scatter (a trilinear cell's last corner in a map plane, a brick bound,
 * an anchor gather of the localisation, a block's partial column, a listed
 * fuse tile, a voxel and its nearest pixel in the map update, a corner of the
 * render adjoint, a tile of the anchor render's order) before the access, skip
 * any access outside its buffer, and keep the handle's first violation.
 * prism_checked_build returns 1 in that library, 0 in libprism.so.
 * prism_check_status synchronises the handle's stream and writes its first
 * violation to *word: 0 for none, else (site << 48) | (index & (2^48 - 1)),
 * site 1 render corner, 2 brick bound, 3 anchor gather, 4 partial column,
 * 5 fuse tile, 6 fuse voxel, 7 fuse pixel, 8 adjoint corner, 9 tile order;
 * always 0 in libprism.so, whose kernels carry no tests.  A violation means
 * a wrong result, never an access outside a buffer.  PRISM_EINVAL for a
 * NULL argument, PRISM_ECUDA if the read fails.  The allocation-free entry
 * point (prism_normal_equations_noalloc) runs without a word: its accesses
 * are tested and skipped but not recorded. */
int32_t prism_checked_build(void);
prism_status prism_check_status(prism_handle h, uint64_t* word);

/* Bytes of device memory the handle owns. */
int64_t prism_device_bytes(prism_handle h);

/* Human-readable description of the last error on h (never NULL), and of a status. */
const char* prism_last_error(prism_handle h);
const char* prism_status_string(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* PRISM_H */
