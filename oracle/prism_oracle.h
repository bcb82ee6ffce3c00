/* PRISM filter oracle — declarations.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow FP64 CPU restatement of
 * the PRISM filter step (arXiv 2212.02988): render (App. B), map update
 * (App. C/D, Eq. mapupdategauss), prediction-to-observation pose objective
 * (App. E.3, Eq. pointtoplanelaplace), Laplace approximation (Sec. 4.1),
 * state propagation and velocity conditional (App. E.1/E.2).  Only the test
 * suite, the package's smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code with the CUDA library.
 *
 * Precision: every value is computed in FP64.  Where a floating-point
 * comparison decides an integer (which voxel a sample falls in, whether a
 * sample is a hit, which pixel a point projects to, whether a residual is
 * gated), the decision is taken with the documented FP32 recipe that the
 * device kernels also follow, so the integers agree bit for bit; the FP64
 * value path then uses the decided indices.
 */
#ifndef PRISM_ORACLE_H
#define PRISM_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t nx, ny, nz;          /* voxels per axis */
    int32_t width, height;       /* image size, pixels */
    int32_t n_gn;                /* Gauss-Newton iterations per frame */
    double voxel;                /* voxel edge length, m */
    double origin[3];            /* world position of the grid's min corner */
    double fx, fy, cx, cy;       /* pinhole intrinsics, pixel centres at integers */
    double eps;                  /* ray step (App. F.2: 0.4 * voxel) */
    double tau;                  /* hit threshold (App. F.2: 0) */
    double max_depth;            /* longest ray distance, m; <= 0 means the grid bounds it */
    double trunc;                /* truncation distance (App. F.2: 2 * voxel) */
    double prior_var;            /* prior variance sigma^2 of every channel (App. B: sigma >> 1) */
    double init_occ;             /* first belief occupancy mean (App. F.2: -0.001) */
    double update_var;           /* sigma_update^2 (App. F.2: 1) */
    double sigma_vel[2];         /* transition scales, translation / rotation (Tbl. transscales) */
    double sigma_pose[2];
    double b_geo, b_rgb;         /* Laplace scales of the objective (App. F.2) */
    double gate_geo, gate_rgb;   /* residual gates (App. F.2) */
    double floor_geo, floor_rgb; /* IRLS floor on |r| (reading of the L1 objective) */
    double ema;                  /* Laplace covariance EMA coefficient (App. F.2: 0.8) */
    double disc;                 /* depth-discontinuity threshold, m (App. F.3) */
    double gravity;              /* m/s^2, world -z */
    /* pose optimiser: 0 Gauss-Newton on the IRLS form (n_gn iterations), 1 the
     * paper's Adam (App. F.2: momentum off, adam_steps steps of adam_pixels
     * uniformly sampled pixels, step sizes lr_t / lr_r; beta2 and eps unstated,
     * Adam's defaults) */
    int32_t optimiser;
    int32_t adam_steps;
    int32_t adam_pixels;
    int32_t adam_pad;
    uint64_t adam_seed;
    double adam_lr_t, adam_lr_r, adam_beta2, adam_eps;
} or_params;

/* Filter state s = (pose, velocity): pose (t, q), q = (w, x, y, z) maps
 * camera to world; velocity (v linear, w angular) in the world frame.
 * cov is 12x12 row-major over the error state (dt, dtheta, dv, dw) with the
 * rotation error applied on the left: R = Exp(dtheta) R_mean. */
typedef struct {
    double t[3], q[4], v[3], w[3];
    double cov[144];
    int32_t n_localised;         /* frames localised so far (EMA start) */
    int32_t pad;
} or_state;

/* Output of the prediction step (App. E.1/E.2). */
typedef struct {
    double t[3], q[4], v[3], w[3];  /* propagated mean */
    double cov[144];                /* propagated joint covariance */
    double cov_pp[36];              /* pose prior covariance */
    double prec_pp[36];             /* its inverse */
    double D[36];                   /* velocity conditional: E[dv | dp] = D dp */
    double cov_vel[36];             /* conditional covariance of v given p */
} or_prior;

/* Per-call diagnostics of the localisation. */
typedef struct {
    double cost;                 /* final objective: sum |r|/b over kept residuals */
    double n_pixels;             /* pixels kept at the final pose */
    double xi[6];                /* optimum in the prior's tangent coordinates */
} or_loc_diag;

#ifdef __cplusplus
extern "C" {
#endif
/* Worker threads of the per-ray, per-pixel and per-voxel loops (n <= 0:
 * every online processor, the default).  Results do not depend on it. */
void or_set_threads(int32_t n);
int32_t or_get_threads(void);
int or_render(const or_params* P, const double* occ, const double* rgb,
              const double pose[7], const int32_t* pix, int32_t npix,
              double* depth, double* rgb_out, uint8_t* mask, int32_t* hitk,
              int64_t* n_samples);
int or_render_backward(const or_params* P, const double* occ, const double* rgb, const double pose[7],
                       const double* gD, const double* gC, double* g_occ, double* g_rgb, double g_pose[6]);
void or_depth_mask(const or_params* P, const float* depth, uint8_t* mask);
void or_anchor_normals(const or_params* P, const float* depth, const uint8_t* mask,
                       double* n64, float* n32, uint8_t* nvalid);
int or_residuals(const or_params* P, const double anchor_pose[7], const float* a_depth,
                 const float* a_rgb, const double pose[7], const float* o_depth, const float* o_rgb,
                 double* r, double* J, int32_t* assoc, uint8_t* kept);
int or_normal_equations(const or_params* P, const double anchor_pose[7],
                        const float* a_depth, const float* a_rgb,
                        const double pose[7], const float* o_depth, const float* o_rgb,
                        double H[36], double g[6], double Ht[36], double stats[2]);
int or_predict(const or_params* P, const or_state* s, const double* imu, int32_t n_imu,
               double dt, or_prior* out);
int or_localise(const or_params* P, const or_prior* pr, const or_state* prev,
                const float* a_depth, const float* a_rgb,
                const float* o_depth, const float* o_rgb,
                or_state* out, or_loc_diag* diag);
int64_t or_fuse(const or_params* P, double* occ, double* rgb, double* var_occ, double* var_rgb,
                const double pose[7], const float* depth, const float* rgb_obs);
/* Output i (0-based) of SplitMix64 started at state `seed`, and the pixel
 * index it draws from n pixels (the high 32 bits times n, shifted down). */
uint64_t or_splitmix64(uint64_t seed, uint64_t i);
uint32_t or_sample_pixel(uint64_t seed, uint64_t i, uint32_t n);
/* The paper's pose optimiser on the objective of App. E.3 from xi = 0: Adam
 * steps s = 1 .. adam_steps on tangent coordinates xi at the prior mean;
 * pixels of step s are draws counter0 + (s - 1) adam_pixels + k.  xi_out: the
 * result; xi_trace (adam_steps x 6, may be NULL): xi after every step. */
int or_adam(const or_params* P, const or_prior* pr, const double anchor_pose[7], const float* a_depth,
            const float* a_rgb, const float* o_depth, const float* o_rgb, uint64_t counter0,
            double xi_out[6], double* xi_trace);
#ifdef __cplusplus
}
#endif
#endif
