// prism_abi.cu — the C ABI of include/prism.h: handle life cycle, argument
// checks, the order in which each entry enqueues its kernels on the
// handle's stream, and host-side state, counter and timing I/O.
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "prism.h"
#include "prism_dev.cuh"
#include "host_util.h"

using namespace prism;

namespace prism {

bool valid_track_config(const prism_config* c, std::string& why) {
    auto bad = [&](const char* m) { why = m; return false; };
    if (!c) return bad("config is NULL");
    if (c->width < 3 || c->height < 3 || (double)c->width * c->height > 1.0e8) return bad("image size out of range");
    if (!(c->fx > 0) || !(c->fy > 0)) return bad("fx, fy must be > 0");
    if (!(c->b_geo > 0) || !(c->b_rgb > 0) || !(c->floor_geo > 0) || !(c->floor_rgb > 0))
        return bad("Laplace scales and IRLS floors must be > 0");
    // gates and the discontinuity threshold may be +inf (no gate)
    if (!(c->gate_geo >= 0) || !(c->gate_rgb >= 0) || !(c->disc >= 0))
        return bad("gates and the discontinuity threshold must be >= 0");
    for (double x : {c->cx, c->cy, c->fx, c->fy, c->b_geo, c->b_rgb, c->floor_geo, c->floor_rgb})
        if (!std::isfinite(x)) return bad("non-finite configuration value");
    return true;
}

bool valid_config(const prism_config* c, std::string& why) {
    auto bad = [&](const char* m) { why = m; return false; };
    if (!c) return bad("config is NULL");
    if (!valid_track_config(c, why)) return false;
    if (c->nx <= 0 || c->ny <= 0 || c->nz <= 0 || (c->nx % 8) || (c->ny % 8) || (c->nz % 8))
        return bad("nx, ny, nz must be positive multiples of 8");
    if ((double)(c->nx + 2) * (c->ny + 2) * (c->nz + 2) > 2147483648.0) return bad("grid larger than 2^31 voxels");
    if (c->storage != PRISM_STORAGE_F32 && c->storage != PRISM_STORAGE_BF16) return bad("storage must be 0 or 1");
    if (c->n_gn < 1 || c->n_gn > 1000) return bad("n_gn must be in [1, 1000]");
    if (c->skip_empty != 0 && c->skip_empty != 1) return bad("skip_empty must be 0 or 1");
    if (!(c->voxel > 0) || !(c->eps > 0)) return bad("voxel and eps must be > 0");
    if (!(c->prior_var > 0) || !(c->update_var > 0) || !(c->trunc > 0)) return bad("variances and trunc must be > 0");
    if (!(c->ema >= 0 && c->ema <= 1)) return bad("ema must be in [0, 1]");
    if (c->optimiser != PRISM_OPT_GAUSS_NEWTON && c->optimiser != PRISM_OPT_ADAM)
        return bad("optimiser must be 0 (Gauss-Newton) or 1 (Adam)");
    if (c->optimiser == PRISM_OPT_ADAM) {
        if (c->adam_steps < 1 || c->adam_pixels < 1 || c->adam_pixels > 256)
            return bad("adam_steps must be >= 1 and adam_pixels in [1, 256]");
        if (!(c->adam_lr_t > 0) || !(c->adam_lr_r > 0) || !(c->adam_eps > 0) || !(c->adam_beta2 >= 0) ||
            !(c->adam_beta2 < 1))
            return bad("Adam step sizes and eps must be > 0 and beta2 in [0, 1)");
    }
    for (double x : {c->origin[0], c->origin[1], c->origin[2], c->tau, c->max_depth})
        if (!std::isfinite(x)) return bad("non-finite configuration value");
    return true;
}

void fill_kparams(const prism_config* c, KParams& k) {
    std::memset(&k, 0, sizeof(k));
    k.nx = c->nx; k.ny = c->ny; k.nz = c->nz;
    k.nbx = c->nx / 8; k.nby = c->ny / 8; k.nbz = c->nz / 8;
    k.px = (uint32_t)c->nx + 2; k.py = (uint32_t)c->ny + 2; k.pxy = k.px * k.py;
    k.npad = k.pxy * ((uint32_t)c->nz + 2);
    k.W = c->width; k.H = c->height;
    k.bf16 = c->storage == PRISM_STORAGE_BF16;
    k.skip = c->skip_empty;
    // brick levels: level l + 1 halves level l's brick counts while all three are even
    {
        int dx = c->nx / 4, dy = c->ny / 4, dz = c->nz / 4, off = 0;
        k.nlev = 0;
        for (int l = 0;; ++l) {
            k.bb_off[l] = off;
            off += dx * dy * dz;
            if (l == 3 || ((dx | dy | dz) & 1)) break;
            dx /= 2; dy /= 2; dz /= 2;
            k.nlev = l + 1;
        }
        k.bb_len = off;
    }
    // the march cannot take more than (nx + ny + nz) vs / eps in-grid samples
    double kcap = 2.0 * (c->nx + c->ny + c->nz) * c->voxel / c->eps + 2.0;
    double kuser = c->max_depth > 0 ? std::floor(c->max_depth / c->eps) : kcap;
    double km = kuser < kcap ? kuser : kcap;
    k.kmax = km > 2.0e9 ? 2000000000 : (int)km;
    for (int a = 0; a < 3; ++a) { k.o32[a] = (float)c->origin[a]; k.origin[a] = c->origin[a]; }
    k.vs32 = (float)c->voxel;
    k.inv_vs32 = (float)(1.0 / c->voxel);
    k.eps32 = (float)c->eps;
    k.tau32 = (float)c->tau;
    k.trunc32 = (float)c->trunc;
    k.disc32 = (float)c->disc;
    k.fx32 = (float)c->fx; k.fy32 = (float)c->fy; k.cx32 = (float)c->cx; k.cy32 = (float)c->cy;
    k.ifx32 = (float)(1.0 / c->fx); k.ify32 = (float)(1.0 / c->fy);
    k.gate_geo32 = (float)c->gate_geo; k.gate_rgb32 = (float)c->gate_rgb;
    k.b_geo32 = (float)c->b_geo; k.b_rgb32 = (float)c->b_rgb;
    k.floor_geo32 = (float)c->floor_geo; k.floor_rgb32 = (float)c->floor_rgb;
    k.upd_prec32 = (float)(1.0 / c->update_var);
    k.vs = c->voxel; k.eps = c->eps; k.tau = c->tau; k.trunc = c->trunc;
    k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy;
    for (int i = 0; i < 2; ++i) { k.sigma_vel[i] = c->sigma_vel[i]; k.sigma_pose[i] = c->sigma_pose[i]; }
    k.ema = c->ema; k.gravity = c->gravity; k.update_var = c->update_var;
}

// q / sqrt(((w*w + x*x) + y*y) + z*z): every pose given by the caller is
// normalised once, here, with exactly these FP64 operations (host code is
// compiled without floating-point contraction).
void normalise_pose(const double* in, double* out) {
    const double n = std::sqrt(((in[3] * in[3] + in[4] * in[4]) + in[5] * in[5]) + in[6] * in[6]);
    for (int a = 0; a < 3; ++a) out[a] = in[a];
    for (int a = 0; a < 4; ++a) out[3 + a] = in[3 + a] / n;
}

bool finite_pose(const double* p) {
    for (int i = 0; i < 7; ++i)
        if (!std::isfinite(p[i])) return false;
    double n = p[3] * p[3] + p[4] * p[4] + p[5] * p[5] + p[6] * p[6];
    return n > 1e-20;
}

}  // namespace prism


namespace {

enum Phase { PH_PREDICT = 0, PH_LOCALISE, PH_FUSE, PH_RENDER, PH_ANCHOR, PH_LAPLACE, PH_COUNT };
const char* const kPhaseName[PH_COUNT] = {"prism predict", "prism localise", "prism fuse",
                                          "prism render",  "prism anchor",   "prism laplace"};

struct TimedPair {
    int phase;
    cudaEvent_t a, b;
};

}  // namespace

struct prism_ctx {
    prism_config cfg{};
    KParams kp{};
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t nvox = 0;
    MapPlanes map{};
    void* map_block = nullptr;
    float* a_depth = nullptr;
    float* a_rgb = nullptr;
    float4* a0 = nullptr;
    float4* a1 = nullptr;
    uint8_t* o_mask = nullptr;
    DevState* dstate = nullptr;
    DevStats* dstats = nullptr;
    float* partials = nullptr;
    int* fuse_list = nullptr;
    unsigned int* fuse_ctr = nullptr;
    unsigned int* counter = nullptr;
    // the anchor render's tile order (render_plan_block): the last anchor
    // render's tile costs and rotation, the planned order and its scratch,
    // in one block; planned on its own stream once the posterior is final
    // (beside the map update), the render waits for ev_plan.  plan_ready: an
    // anchor render has recorded its costs; plan_fresh: the order was
    // planned for the next anchor render
    unsigned long long* check = nullptr;   // bounds-check build: the first index violation
    void* plan_block = nullptr;
    RenderPlanIn plan_in{};
    RenderPlan plan_out{};
    cudaStream_t plan_stream = nullptr;
    cudaEvent_t ev_plan = nullptr;
    bool plan_ready = false;
    bool plan_fresh = false;
    bool plan_waited = false;   // the main stream already waits for ev_plan
    DevState* h_state = nullptr;       // pinned host copy of the device state (read_state)
    int max_blocks = 0;
    double* d_imu = nullptr;
    int imu_cap = 0;
    // prism_step's prediction stream: the prior of step t + 1 needs only the
    // posterior of step t, so it runs beside step t's fuse and render
    cudaStream_t side = nullptr;
    cudaEvent_t ev_state = nullptr;   // main stream: the posterior is final
    cudaEvent_t ev_pred = nullptr;    // side stream: the prior is ready
    cudaEvent_t ev_read = nullptr;    // side stream: the posterior's host copy is done
    static constexpr int kImuRing = 4;
    double* h_imu[kImuRing] = {nullptr, nullptr, nullptr, nullptr};   // pinned IMU staging
    cudaEvent_t ev_imu[kImuRing] = {nullptr, nullptr, nullptr, nullptr};
    int h_imu_cap = 0;
    int imu_slot = 0;
    // prism_rollout's buffers: device scratch states, records, matrices and
    // inputs in one block; their pinned host staging, reused once ev_roll
    // (recorded after the upload) has passed
    void* roll_dev = nullptr;
    size_t roll_cap = 0;
    char* h_roll = nullptr;
    size_t h_roll_cap = 0;
    cudaEvent_t ev_roll = nullptr;
    // prism_map_descent's buffers: gradients (N + 3N floats), one rendered
    // frame (depth, colour, hit mask) and the loss, in one block
    void* md_dev = nullptr;
    // prism_step_host's device copies of the host frames, used in turn, and
    // the event after the last call's copies
    float* in_depth[2] = {nullptr, nullptr};
    float* in_rgb[2] = {nullptr, nullptr};
    int in_slot = 0;
    cudaStream_t copy = nullptr;      // their uploads, beside the prediction
    cudaEvent_t ev_in = nullptr;
    bool has_anchor = false;
    bool anchor_at_mean = false;   // the anchor was rendered at the current state mean
    bool has_prior = false;
    int64_t steps = 0;
    int64_t bytes = 0;
    std::string err;
    bool timing = false;
    bool detail = false;
    bool coop = true;   // the cooperative localisation launch (prism_set_cooperative)
    int64_t launches = 0;
    std::vector<TimedPair> pending;
    std::vector<cudaEvent_t> pool;
    double acc_ms[PH_COUNT] = {0, 0, 0, 0, 0, 0};
    int64_t acc_n[PH_COUNT] = {0, 0, 0, 0, 0, 0};
};

namespace {

thread_local std::string g_err;   // errors without a handle

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

prism_status fail(prism_handle h, prism_status st, const std::string& msg) {
    if (h) h->err = msg;
    else g_err = msg;
    return st;
}

prism_status cuda_fail(prism_handle h, cudaError_t e, const char* what) {
    return fail(h, PRISM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// A kernel launch: counted (prism_stats.kernel_launches), then checked.
#define LAUNCH(h, call, what)                              \
    do {                                                   \
        ++(h)->launches;                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

cudaEvent_t take_event(prism_handle h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// A phase's CUDA events (with prism_set_timing) and its NVTX range on the
// host thread that enqueues it (an NVTX call is a no-op unless a tool such
// as Nsight Systems is attached).
struct PhaseTimer {
    prism_handle h;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseTimer(prism_handle h_, int ph, cudaStream_t s_ = nullptr) : h(h_), phase(ph), s(s_ ? s_ : h_->stream) {
        nvtxRangePushA(kPhaseName[ph]);
        if (h->timing) {
            a = take_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseTimer() {
        if (a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, s);
            h->pending.push_back({phase, a, b});
        }
        nvtxRangePop();
    }
};

void collect_timing(prism_handle h) {
    for (auto& t : h->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            h->acc_ms[t.phase] += ms;
            h->acc_n[t.phase] += 1;
        }
        h->pool.push_back(t.a);
        h->pool.push_back(t.b);
    }
    h->pending.clear();
}

void free_all(prism_handle h) {
    void* ptrs[] = {h->map_block, h->a_depth, h->a_rgb, h->a0, h->a1, h->o_mask,
                    h->dstate, h->dstats, h->partials, h->counter, h->d_imu, h->fuse_list, h->fuse_ctr,
                    h->plan_block, h->check};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& t : h->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->plan_stream) {
        cudaStreamSynchronize(h->plan_stream);
        cudaStreamDestroy(h->plan_stream);
    }
    if (h->ev_plan) cudaEventDestroy(h->ev_plan);
    for (int k = 0; k < prism_ctx::kImuRing; ++k) {
        if (h->h_imu[k]) cudaFreeHost(h->h_imu[k]);
        if (h->ev_imu[k]) cudaEventDestroy(h->ev_imu[k]);
    }
    for (int b = 0; b < 2; ++b) {
        if (h->in_depth[b]) cudaFree(h->in_depth[b]);
        if (h->in_rgb[b]) cudaFree(h->in_rgb[b]);
    }
    if (h->copy) {
        cudaStreamSynchronize(h->copy);
        cudaStreamDestroy(h->copy);
    }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->md_dev) cudaFree(h->md_dev);
    if (h->roll_dev) cudaFree(h->roll_dev);
    if (h->h_roll) cudaFreeHost(h->h_roll);
    if (h->ev_roll) cudaEventDestroy(h->ev_roll);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->ev_state) cudaEventDestroy(h->ev_state);
    if (h->ev_pred) cudaEventDestroy(h->ev_pred);
    if (h->ev_read) cudaEventDestroy(h->ev_read);
}

template <class T>
cudaError_t dalloc(prism_handle h, T** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) h->bytes += (int64_t)bytes;
    return e;
}

// Reports the flags of a state copy just read (each prediction clears them
// on the device, so they are those of the latest step until the next one).
prism_status check_flags(prism_handle h, int flags) {
    if (flags) {
        std::string m = "device reported:";
        if (flags & FLAG_GN_NOTPD) m += " Gauss-Newton system not positive definite;";
        if (flags & FLAG_LAPLACE_NOTPD) m += " Laplace Hessian not positive definite;";
        if (flags & FLAG_PRIOR_NOTPD) m += " prior pose covariance not positive definite;";
        if (flags & FLAG_SYNC_TIMEOUT) {
            m += " a grid-wide wait of the localisation timed out; the step was rejected (state and map unchanged)";
            return fail(h, PRISM_ECUDA, m);
        }
        m += " the step was rejected (state and map unchanged)";
        return fail(h, PRISM_ENOTPD, m);
    }
    return PRISM_OK;
}

void fill_state(const DevState& s, prism_state* out) {
    std::memset(out, 0, sizeof(*out));
    std::memcpy(out->t, s.t, sizeof(s.t));
    std::memcpy(out->q, s.q, sizeof(s.q));
    std::memcpy(out->v, s.v, sizeof(s.v));
    std::memcpy(out->w, s.w, sizeof(s.w));
    std::memcpy(out->cov, s.cov, sizeof(s.cov));
    out->n_localised = s.n_localised;
}

// prism_step's read-back: the posterior is final at ev_state (after the
// Laplace pass), so its fields are copied on the side stream behind that
// event and only that copy is waited for; the map update and the anchor
// render go on on the main stream (they write none of these fields).
prism_status read_posterior(prism_handle h, prism_state* out) {
    DevState* d = h->dstate;
    DevState* hs = h->h_state;
    CK(h, cudaStreamWaitEvent(h->side, h->ev_state, 0), "wait for the posterior");
    // t, q, v, w, cov (contiguous at the start of DevState), then n_localised and flags
    const size_t head = offsetof(DevState, cov) + sizeof(d->cov);
    CK(h, cudaMemcpyAsync(hs, d, head, cudaMemcpyDeviceToHost, h->side), "read state");
    CK(h, cudaMemcpyAsync(&hs->n_localised, &d->n_localised, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->side),
       "read state");
    CK(h, cudaEventRecord(h->ev_read, h->side), "read event");
    CK(h, cudaEventSynchronize(h->ev_read), "wait for the state");
    fill_state(*hs, out);
    return check_flags(h, hs->flags);
}

prism_status read_state(prism_handle h, prism_state* out) {
    // one asynchronous copy behind the stream's work, then one wait
    CK(h, cudaMemcpyAsync(h->h_state, h->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream), "read state");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    const DevState& s = *h->h_state;
    fill_state(s, out);
    return check_flags(h, s.flags);
}

prism_status write_state(prism_handle h, const prism_state* s) {
    DevState d;
    std::memset(&d, 0, sizeof(d));
    double pin[7], pn[7];
    std::memcpy(pin, s->t, 3 * sizeof(double));
    std::memcpy(pin + 3, s->q, 4 * sizeof(double));
    normalise_pose(pin, pn);
    std::memcpy(d.t, pn, sizeof(d.t));
    std::memcpy(d.q, pn + 3, sizeof(d.q));
    std::memcpy(d.v, s->v, sizeof(d.v));
    std::memcpy(d.w, s->w, sizeof(d.w));
    std::memcpy(d.cov, s->cov, sizeof(d.cov));
    d.n_localised = s->n_localised;
    // keep the anchor pose already on the device
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    double anchor[7];
    CK(h, cudaMemcpy(anchor, h->dstate->anchor_pose, sizeof(anchor), cudaMemcpyDeviceToHost), "read anchor pose");
    std::memcpy(d.anchor_pose, anchor, sizeof(anchor));
    CK(h, cudaMemcpy(h->dstate, &d, sizeof(d), cudaMemcpyHostToDevice), "write state");
    PoseArg pa{};
    LAUNCH(h, launch_prep(h->dstate, PREP_STATE, pa, h->stream), "pose matrices");
    CK(h, cudaEventRecord(h->ev_state, h->stream), "state event");
    h->has_prior = false;
    h->anchor_at_mean = false;
    return PRISM_OK;
}

prism_status do_render_anchor(prism_handle h, uint8_t* mask = nullptr, int32_t* hitk = nullptr) {
    {
        PhaseTimer t(h, PH_RENDER);
        // t[3] and q[4] are contiguous: the state mean pose becomes the anchor's pose
        RenderPlan plan = h->plan_out;
        if (!h->plan_fresh) plan.order = nullptr;
        else if (!h->plan_waited) CK(h, cudaStreamWaitEvent(h->stream, h->ev_plan, 0), "wait for the tile order");
        LAUNCH(h, launch_render(h->kp, h->dstate->c2w, h->map, h->a_depth, h->a_rgb, mask, hitk, h->dstats,
                                h->dstate->t, h->dstate->anchor_pose, h->detail, h->stream, plan),
               "render");
        h->plan_ready = true;
        h->plan_fresh = false;
        h->plan_waited = false;
    }
    PhaseTimer t(h, PH_ANCHOR);
    LAUNCH(h, launch_anchor_pack(h->kp, h->a_depth, h->a_rgb, h->a0, h->a1, h->stream), "anchor pack");
    h->has_anchor = true;
    h->anchor_at_mean = true;
    return PRISM_OK;
}

// after_side: the prior was predicted on the side stream (prism_step) and the
// passes wait for it; prepped: that prediction also left the Gauss-Newton
// start matrices (the anchor is the one rendered at the state mean);
// wait_in: the frame is being uploaded on the copy stream (prism_step_host).
prism_status do_localise(prism_handle h, const float* depth, const float* rgb, bool after_side = false,
                         bool prepped = false, bool wait_in = false) {
    PhaseTimer t(h, PH_LOCALISE);
    PoseArg pa{};
    if (after_side) CK(h, cudaStreamWaitEvent(h->stream, h->ev_pred, 0), "wait for the prior");
    if (wait_in) CK(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0), "wait for the frame");
    if (!prepped) LAUNCH(h, launch_prep(h->dstate, PREP_REL, pa, h->stream, !after_side), "pose matrices");
    if (h->cfg.optimiser == PRISM_OPT_ADAM) {   // the paper's optimiser, then the Laplace pass
        LAUNCH(h, launch_depth_mask(h->kp, depth, h->o_mask, h->stream), "observation mask");
        AdamArgs A;
        A.steps = h->cfg.adam_steps;
        A.pixels = h->cfg.adam_pixels;
        A.seed = (unsigned long long)h->cfg.adam_seed;
        A.lr_t = h->cfg.adam_lr_t;
        A.lr_r = h->cfg.adam_lr_r;
        A.beta2 = h->cfg.adam_beta2;
        A.eps = h->cfg.adam_eps;
        LAUNCH(h, launch_adam(h->kp, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, A, h->stream), "Adam");
        LAUNCH(h, launch_track(h->kp, TRACK_LAPLACE, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, h->partials,
                               h->counter, h->max_blocks, h->dstats, h->stream),
               "Laplace pass");
        CK(h, cudaEventRecord(h->ev_state, h->stream), "state event");
        h->has_prior = false;
        h->anchor_at_mean = false;
        return PRISM_OK;
    }
    // the first pass also evaluates the observation's depth validity into o_mask
    // (read by the later passes and by the fuse), and clears the barrier of the
    // cooperative launch that runs the other passes (a pass per launch where
    // the device cannot hold that launch's grid at once, or with
    // prism_set_cooperative off)
    for (int it = 0; it < h->cfg.n_gn; ++it) {
        if (it == 1 && h->coop) {
            cudaError_t e = launch_track_coop(h->kp, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, h->partials,
                                              h->counter + 1, h->max_blocks, h->dstats, h->cfg.n_gn - 1, h->stream);
            if (e == cudaSuccess) {
                ++h->launches;
                break;
            }
            if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(h, e, "Gauss-Newton passes");
            cudaGetLastError();
        }
        LAUNCH(h, launch_track(h->kp, TRACK_GN, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, h->partials,
                           h->counter, h->max_blocks, h->dstats, h->stream, !(prepped && it == 0),
                           it == 0 ? h->o_mask : nullptr),
           "Gauss-Newton pass");
    }
    {
        PhaseTimer tl(h, PH_LAPLACE);
        LAUNCH(h, launch_track(h->kp, TRACK_LAPLACE, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, h->partials,
                           h->counter, h->max_blocks, h->dstats, h->stream),
           "Laplace pass");
    }
    CK(h, cudaEventRecord(h->ev_state, h->stream), "state event");
    h->has_prior = false;
    h->anchor_at_mean = false;
    return PRISM_OK;
}

prism_status do_fuse(prism_handle h, const float* depth, const float* rgb, bool mask_ready) {
    PhaseTimer t(h, PH_FUSE);
    if (!mask_ready) LAUNCH(h, launch_depth_mask(h->kp, depth, h->o_mask, h->stream), "observation mask");
    // after a localisation in the same step (mask_ready), a rejected step fuses nothing
    LAUNCH(h, launch_fuse_listed(h->kp, h->map, h->dstate->w2c, depth, rgb, h->o_mask, h->dstats, h->fuse_list,
                                 h->fuse_ctr, mask_ready ? &h->dstate->rejected : nullptr, h->stream),
           "fuse");
    ++h->launches;   // (two kernels: the frustum list and the update)
    if (h->kp.skip) {
        // the tile order is done long before (it started with the map update):
        // waiting here keeps the brick bounds and the render back to back
        if (h->plan_fresh && !h->plan_waited) {
            CK(h, cudaStreamWaitEvent(h->stream, h->ev_plan, 0), "wait for the tile order");
            h->plan_waited = true;
        }
        LAUNCH(h, launch_brick_bounds(h->kp, h->map, h->stream), "brick bounds");
    }
    return PRISM_OK;
}

// The tile order of the anchor render that follows at the posterior mean,
// planned on its own stream once the posterior is final (ev_state).
prism_status do_plan(prism_handle h) {
    if (!h->plan_ready) return PRISM_OK;
    CK(h, cudaStreamWaitEvent(h->plan_stream, h->ev_state, 0), "wait for the posterior");
    LAUNCH(h, launch_render_plan(h->kp, h->plan_in, h->plan_stream), "tile order");
    CK(h, cudaEventRecord(h->ev_plan, h->plan_stream), "tile-order event");
    h->plan_fresh = true;
    h->plan_waited = false;
    return PRISM_OK;
}

prism_status do_predict(prism_handle h, const double* imu, int32_t n, double dt) {
    if (n > h->imu_cap) {
        if (h->d_imu) {
            CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
            cudaFree(h->d_imu);
            h->bytes -= (int64_t)h->imu_cap * 7 * sizeof(double);
            h->d_imu = nullptr;
            h->imu_cap = 0;
        }
        int cap = n < 256 ? 256 : n;
        CK(h, dalloc(h, &h->d_imu, (size_t)cap * 7 * sizeof(double)), "IMU buffer");
        h->imu_cap = cap;
    }
    PhaseTimer t(h, PH_PREDICT);
    if (n > 0)
        CK(h, cudaMemcpyAsync(h->d_imu, imu, (size_t)n * 7 * sizeof(double), cudaMemcpyHostToDevice, h->stream),
           "IMU upload");
    LAUNCH(h, launch_predict(h->kp, h->dstate, h->d_imu, n, dt, h->stream), "predict");
    h->has_prior = true;
    return PRISM_OK;
}

// prism_step's prediction: on the side stream once the posterior is final
// (it then overlaps the previous step's fuse and render), the IMU window
// staged through a ring of pinned buffers so that the upload is asynchronous.
// prep: the same kernel also derives the Gauss-Newton start matrices against
// the state mean's camera (valid when the anchor is rendered there).
prism_status do_predict_side(prism_handle h, const double* imu, int32_t n, double dt, bool prep) {
    if (n > h->imu_cap || n > h->h_imu_cap) {
        CK(h, cudaStreamSynchronize(h->side), "stream synchronize");
        CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
        const int cap = n < 256 ? 256 : n;
        if (n > h->imu_cap) {
            if (h->d_imu) {
                cudaFree(h->d_imu);
                h->bytes -= (int64_t)h->imu_cap * 7 * sizeof(double);
                h->d_imu = nullptr;
                h->imu_cap = 0;
            }
            CK(h, dalloc(h, &h->d_imu, (size_t)cap * 7 * sizeof(double)), "IMU buffer");
            h->imu_cap = cap;
        }
        if (n > h->h_imu_cap) {
            for (int k = 0; k < prism_ctx::kImuRing; ++k) {
                if (h->h_imu[k]) cudaFreeHost(h->h_imu[k]);
                h->h_imu[k] = nullptr;
            }
            h->h_imu_cap = 0;
            for (int k = 0; k < prism_ctx::kImuRing; ++k)
                CK(h, cudaMallocHost(&h->h_imu[k], (size_t)cap * 7 * sizeof(double)), "IMU staging");
            h->h_imu_cap = cap;
        }
    }
    const int k = h->imu_slot;
    h->imu_slot = (k + 1) % prism_ctx::kImuRing;
    CK(h, cudaEventSynchronize(h->ev_imu[k]), "IMU staging reuse");   // its last upload has run
    if (n > 0) std::memcpy(h->h_imu[k], imu, (size_t)n * 7 * sizeof(double));
    CK(h, cudaStreamWaitEvent(h->side, h->ev_state, 0), "wait for the posterior");
    {
        PhaseTimer t(h, PH_PREDICT, h->side);
        if (n > 0)
            CK(h, cudaMemcpyAsync(h->d_imu, h->h_imu[k], (size_t)n * 7 * sizeof(double), cudaMemcpyHostToDevice,
                                  h->side),
               "IMU upload");
        CK(h, cudaEventRecord(h->ev_imu[k], h->side), "IMU event");
        if (prep) LAUNCH(h, launch_predict_prep(h->kp, h->dstate, h->d_imu, n, dt, h->side), "predict");
        else LAUNCH(h, launch_predict(h->kp, h->dstate, h->d_imu, n, dt, h->side, false), "predict");
    }
    CK(h, cudaEventRecord(h->ev_pred, h->side), "prior event");
    h->has_prior = true;
    return PRISM_OK;
}

bool imu_ok(const double* imu, int32_t n, double dt, std::string& why) {
    if (n < 0) { why = "n must be >= 0"; return false; }
    if (n > 0 && !imu) { why = "imu is NULL with n > 0"; return false; }
    if (!(dt > 0) || !std::isfinite(dt)) { why = "dt must be finite and > 0"; return false; }
    for (int i = 0; i < 7 * n; ++i)
        if (!std::isfinite(imu[i])) { why = "non-finite IMU value"; return false; }
    return true;
}

// The filter step after its argument checks (prism_step, prism_step_host).
prism_status step_checked(prism_handle h, const double* imu, int32_t n, double dt, const float* depth,
                          const float* rgb, prism_state* out, bool wait_in = false);

}  // namespace

extern "C" {

void prism_config_default(prism_config* c, int32_t n, double extent, int32_t width, int32_t height) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->nx = c->ny = c->nz = n;
    c->storage = PRISM_STORAGE_F32;
    c->width = width;
    c->height = height;
    c->n_gn = 10;
    c->skip_empty = 1;
    c->voxel = extent / n;
    for (int a = 0; a < 3; ++a) c->origin[a] = -0.5 * extent;
    c->fx = c->fy = 70.0 * width / 80.0;
    c->cx = 0.5 * (width - 1);
    c->cy = 0.5 * (height - 1);
    c->eps = 0.4 * c->voxel;
    c->tau = 0.0;
    c->max_depth = 0.0;
    c->trunc = 2.0 * c->voxel;
    c->prior_var = 1e4;
    c->init_occ = -0.001;
    c->init_rgb = 0.0;
    c->update_var = 1.0;
    c->sigma_vel[0] = 0.03; c->sigma_vel[1] = 0.03;
    c->sigma_pose[0] = 0.05; c->sigma_pose[1] = 0.02;
    c->b_geo = 0.02; c->b_rgb = 0.1;
    c->gate_geo = 0.45; c->gate_rgb = 0.15;
    c->floor_geo = 1e-3; c->floor_rgb = 1e-2;
    c->ema = 0.8;
    c->disc = 0.1;
    c->gravity = 9.81;
    c->optimiser = PRISM_OPT_GAUSS_NEWTON;
    c->adam_steps = 1000;
    c->adam_pixels = 200;
    c->adam_seed = 0x5EED2212ull;
    c->adam_lr_t = 1e-3;
    c->adam_lr_r = 3.6e-4;
    c->adam_beta2 = 0.999;
    c->adam_eps = 1e-8;
}

prism_status prism_create_map(const prism_config* cfg, const prism_state* s1, void* stream, prism_handle* out) {
    std::string why;
    if (!out) return fail(nullptr, PRISM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_config(cfg, why)) return fail(nullptr, PRISM_EINVAL, "invalid config: " + why);
    if (s1) {
        double p[7];
        std::memcpy(p, s1->t, 3 * sizeof(double));
        std::memcpy(p + 3, s1->q, 4 * sizeof(double));
        if (!finite_pose(p)) return fail(nullptr, PRISM_EINVAL, "initial state pose is not finite");
    }
    prism_ctx* h = new (std::nothrow) prism_ctx();
    if (!h) return fail(nullptr, PRISM_ENOMEM, "host allocation failed");
    h->cfg = *cfg;
    fill_kparams(cfg, h->kp);
    h->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->max_blocks = (sms > 0 ? sms : 152) * 4;
    h->nvox = (size_t)cfg->nx * cfg->ny * cfg->nz;
    const size_t es = cfg->storage == PRISM_STORAGE_BF16 ? 2 : 4;
    const size_t plane = (((size_t)h->kp.npad * es + 255) / 256) * 256;   // padded plane, 256-byte aligned
    const size_t npix = (size_t)cfg->width * cfg->height;
    auto cleanup = [&](prism_status st, const std::string& m) {
        free_all(h);
        delete h;
        return fail(nullptr, st, m);
    };
    const size_t tbytes = ((8 * (size_t)h->kp.nbx * h->kp.nby * h->kp.nbz * sizeof(float2) + 255) / 256) * 256;
    const size_t bbytes = (((size_t)h->kp.bb_len * sizeof(float2) + 255) / 256) * 256;
    if (dalloc(h, &h->map_block, 6 * plane + tbytes + bbytes) != cudaSuccess)
        return cleanup(PRISM_ENOMEM, "map allocation failed");
    char* base = (char*)h->map_block;
    h->map.tb = (float2*)(base + 6 * plane);
    h->map.bb = (float2*)(base + 6 * plane + tbytes);
    h->map.occ = base;
    h->map.r = base + plane;
    h->map.g = base + 2 * plane;
    h->map.b = base + 3 * plane;
    h->map.var_occ = base + 4 * plane;
    h->map.var_rgb = base + 5 * plane;
    if (dalloc(h, &h->a_depth, npix * 4) || dalloc(h, &h->a_rgb, npix * 12) ||
        dalloc(h, &h->a0, npix * 16) || dalloc(h, &h->a1, npix * 16) || dalloc(h, &h->o_mask, npix) ||
        dalloc(h, &h->dstate, sizeof(DevState)) || dalloc(h, &h->dstats, sizeof(DevStats)) ||
        dalloc(h, &h->partials, 2 * (size_t)h->max_blocks * TRACK_NV_MAX * sizeof(float)) ||
        dalloc(h, &h->counter, 2 * sizeof(unsigned int)) ||
        dalloc(h, &h->fuse_list, (size_t)h->kp.nbx * h->kp.nby * h->kp.nbz * sizeof(int)) ||
        dalloc(h, &h->fuse_ctr, 2 * sizeof(unsigned int)))
        return cleanup(PRISM_ENOMEM, "device allocation failed");
    {   // tile costs, order and scratch (one word each per 16x8 tile), the rotation
        const size_t nt = (size_t)((cfg->width + 15) / 16) * ((cfg->height + 7) / 8);
        const size_t words = ((nt + 63) / 64) * 64;
        if (dalloc(h, &h->plan_block, 3 * words * 4 + 64) != cudaSuccess)
            return cleanup(PRISM_ENOMEM, "device allocation failed");
        uint32_t* w = (uint32_t*)h->plan_block;
        float* rot = (float*)(w + 3 * words);
        h->plan_out = RenderPlan{(const int*)(w + words), w, rot};
        h->plan_in = RenderPlanIn{w, rot, h->a_depth, h->dstate->c2w, w + 2 * words, (int*)(w + words)};
    }
#ifdef PRISM_CHECKED
    if (dalloc(h, &h->check, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(h->check, 0, sizeof(unsigned long long)) != cudaSuccess)
        return cleanup(PRISM_ENOMEM, "device allocation failed");
    h->kp.check = h->check;
#endif
    if (cudaMallocHost(&h->h_state, sizeof(DevState)) != cudaSuccess)
        return cleanup(PRISM_ENOMEM, "host allocation failed");
    cudaGetLastError();
    {   // the prediction stream (high priority: its one block is scheduled ahead of waiting fuse tiles)
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if ((e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&h->plan_stream, cudaStreamNonBlocking, greatest)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_plan, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_state, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_pred, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_read, cudaEventDisableTiming)) != cudaSuccess)
            return cleanup(PRISM_ECUDA, std::string("streams: ") + cudaGetErrorString(e));
        for (int k = 0; k < prism_ctx::kImuRing; ++k)
            if ((e = cudaEventCreateWithFlags(&h->ev_imu[k], cudaEventDisableTiming)) != cudaSuccess)
                return cleanup(PRISM_ECUDA, std::string("events: ") + cudaGetErrorString(e));
    }
    if ((e = launch_map_fill(h->kp, h->map, (float)cfg->init_occ, (float)cfg->init_rgb, (float)cfg->prior_var,
                             h->stream)) != cudaSuccess ||
        (e = launch_tile_bounds(h->kp, h->map, h->stream)) != cudaSuccess)
        return cleanup(PRISM_ECUDA, std::string("map fill: ") + cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(h->dstats, 0, sizeof(DevStats), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->counter, 0, 2 * sizeof(unsigned int), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->fuse_ctr, 0, 2 * sizeof(unsigned int), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->dstate, 0, sizeof(DevState), h->stream)) != cudaSuccess)
        return cleanup(PRISM_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
    prism_state init;
    if (s1) {
        init = *s1;
    } else {
        std::memset(&init, 0, sizeof(init));
        init.q[0] = 1.0;
        for (int i = 0; i < 12; ++i) init.cov[13 * i] = 1e-8;
    }
    prism_status st = write_state(h, &init);
    if (st != PRISM_OK) return cleanup(st, h->err);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cleanup(PRISM_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    *out = h;
    return PRISM_OK;
}

prism_status prism_destroy(prism_handle h) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return PRISM_OK;
}

prism_status prism_predict(prism_handle h, const double* imu, int32_t n, double dt) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    std::string why;
    if (!imu_ok(imu, n, dt, why)) return fail(h, PRISM_EINVAL, why);
    DeviceGuard g(h->device);
    return do_predict(h, imu, n, dt);
}

prism_status prism_localise(prism_handle h, const float* depth, const float* rgb, prism_state* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!depth || !rgb) return fail(h, PRISM_EINVAL, "depth or rgb is NULL");
    if (!h->has_prior) return fail(h, PRISM_ESTATE, "localise needs prism_predict first");
    if (!h->has_anchor) return fail(h, PRISM_ESTATE, "localise needs an anchor (prism_render or prism_anchor_load)");
    DeviceGuard g(h->device);
    prism_status st = do_localise(h, depth, rgb);
    if (st != PRISM_OK || !out) return st;
    return read_state(h, out);
}

prism_status prism_update_map(prism_handle h, const float* depth, const float* rgb) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!depth || !rgb) return fail(h, PRISM_EINVAL, "depth or rgb is NULL");
    DeviceGuard g(h->device);
    return do_fuse(h, depth, rgb, false);
}

prism_status prism_render(prism_handle h, const double* pose7, float* depth, float* rgb, uint8_t* mask,
                          int32_t* hitk) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (pose7 && !finite_pose(pose7)) return fail(h, PRISM_EINVAL, "pose is not finite or has a zero quaternion");
    DeviceGuard g(h->device);
    const size_t npix = (size_t)h->cfg.width * h->cfg.height;
    if (pose7) {
        PhaseTimer t(h, PH_RENDER);
        PoseArg pa{};
        normalise_pose(pose7, pa.p);
        LAUNCH(h, launch_prep(h->dstate, PREP_AUX_C2W, pa, h->stream), "pose matrices");
        LAUNCH(h, launch_render(h->kp, h->dstate->aux, h->map, depth, rgb, mask, hitk, h->dstats, nullptr, nullptr,
                            h->detail, h->stream),
           "render");
        return PRISM_OK;
    }
    prism_status st = do_render_anchor(h, mask, hitk);
    if (st != PRISM_OK) return st;
    if (depth) CK(h, cudaMemcpyAsync(depth, h->a_depth, npix * 4, cudaMemcpyDeviceToDevice, h->stream), "copy depth");
    if (rgb) CK(h, cudaMemcpyAsync(rgb, h->a_rgb, npix * 12, cudaMemcpyDeviceToDevice, h->stream), "copy rgb");
    return PRISM_OK;
}

prism_status prism_step(prism_handle h, const double* imu, int32_t n, double dt, const float* depth,
                        const float* rgb, prism_state* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!depth || !rgb) return fail(h, PRISM_EINVAL, "depth or rgb is NULL");
    DeviceGuard g(h->device);
    if (h->steps > 0) {
        std::string why;
        if (!imu_ok(imu, n, dt, why)) return fail(h, PRISM_EINVAL, why);
        if (!h->has_anchor) return fail(h, PRISM_ESTATE, "no anchor");
    }
    return step_checked(h, imu, n, dt, depth, rgb, out);
}

prism_status prism_step_host(prism_handle h, const double* imu, int32_t n, double dt, const float* depth_host,
                             const float* rgb_host, prism_state* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!depth_host || !rgb_host) return fail(h, PRISM_EINVAL, "depth or rgb is NULL");
    DeviceGuard g(h->device);
    if (h->steps > 0) {
        std::string why;
        if (!imu_ok(imu, n, dt, why)) return fail(h, PRISM_EINVAL, why);
        if (!h->has_anchor) return fail(h, PRISM_ESTATE, "no anchor");
    }
    const size_t npix = (size_t)h->cfg.width * h->cfg.height;
    if (!h->ev_in || !h->copy) {   // first call (or one after a failed set-up): what is missing
        for (int b = 0; b < 2; ++b)
            if ((!h->in_depth[b] && dalloc(h, &h->in_depth[b], npix * 4) != cudaSuccess) ||
                (!h->in_rgb[b] && dalloc(h, &h->in_rgb[b], npix * 12) != cudaSuccess)) {
                cudaGetLastError();
                return fail(h, PRISM_ENOMEM, "host-frame buffers");
            }
        if (!h->ev_in) CK(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "host-frame event");
        if (!h->copy) {   // high priority: its upload blocks go ahead of the waiting fuse and render blocks
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            CK(h, cudaStreamCreateWithPriority(&h->copy, cudaStreamNonBlocking, greatest), "host-frame stream");
        }
    }
    CK(h, cudaEventSynchronize(h->ev_in), "previous host-frame copies");
    const int b = h->in_slot;
    h->in_slot ^= 1;
    // after the first step: on the copy stream beside the prediction, behind
    // the previous posterior (which follows the map update that last read
    // this buffer); the localisation waits for them before its first pass
    const bool later = h->steps > 0;
    cudaStream_t cs = later ? h->copy : h->stream;
    if (later) CK(h, cudaStreamWaitEvent(h->copy, h->ev_state, 0), "wait for the posterior");
    // pinned host memory the device maps: the SMs load it (faster over the
    // host link than the copy engines); anything else: the copy engines
    cudaPointerAttributes ad{}, ac{};
    const bool mapped = cudaPointerGetAttributes(&ad, depth_host) == cudaSuccess &&
                        cudaPointerGetAttributes(&ac, rgb_host) == cudaSuccess && ad.type == cudaMemoryTypeHost &&
                        ac.type == cudaMemoryTypeHost && ad.devicePointer && ac.devicePointer;
    cudaGetLastError();
    if (mapped) {
        LAUNCH(h, launch_frame_upload((const float*)ad.devicePointer, h->in_depth[b], npix,
                                      (const float*)ac.devicePointer, h->in_rgb[b], 3 * npix, h->max_blocks / 4, cs),
               "frame upload");
    } else {
        CK(h, cudaMemcpyAsync(h->in_depth[b], depth_host, npix * 4, cudaMemcpyHostToDevice, cs), "depth upload");
        CK(h, cudaMemcpyAsync(h->in_rgb[b], rgb_host, npix * 12, cudaMemcpyHostToDevice, cs), "rgb upload");
    }
    CK(h, cudaEventRecord(h->ev_in, cs), "host-frame event");
    return step_checked(h, imu, n, dt, h->in_depth[b], h->in_rgb[b], out, later);
}

}  // extern "C"

namespace {

prism_status step_checked(prism_handle h, const double* imu, int32_t n, double dt, const float* depth,
                          const float* rgb, prism_state* out, bool wait_in) {
    NvtxRange range("prism step");
    prism_status st;
    bool mask_ready = false;
    if (h->steps > 0) {
        const bool prep = h->anchor_at_mean;
        if ((st = do_predict_side(h, imu, n, dt, prep)) != PRISM_OK) return st;
        if ((st = do_localise(h, depth, rgb, true, prep, wait_in)) != PRISM_OK) return st;
        if ((st = do_plan(h)) != PRISM_OK) return st;
        mask_ready = true;
    }
    if ((st = do_fuse(h, depth, rgb, mask_ready)) != PRISM_OK) return st;
    if ((st = do_render_anchor(h)) != PRISM_OK) return st;
    h->steps += 1;
    if (!out) return PRISM_OK;
    return read_posterior(h, out);
}

}  // namespace

extern "C" {

int32_t prism_checked_build(void) {
#ifdef PRISM_CHECKED
    return 1;
#else
    return 0;
#endif
}

prism_status prism_check_status(prism_handle h, uint64_t* word) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!word) return fail(h, PRISM_EINVAL, "word is NULL");
    *word = 0;
    if (!h->check) return PRISM_OK;
    DeviceGuard g(h->device);
    unsigned long long v = 0;
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    CK(h, cudaMemcpy(&v, h->check, sizeof(v), cudaMemcpyDeviceToHost), "read check word");
    *word = v;
    return PRISM_OK;
}

prism_status prism_get_state(prism_handle h, prism_state* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!out) return fail(h, PRISM_EINVAL, "out is NULL");
    DeviceGuard g(h->device);
    return read_state(h, out);
}

prism_status prism_set_state(prism_handle h, const prism_state* s) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!s) return fail(h, PRISM_EINVAL, "state is NULL");
    double p[7];
    std::memcpy(p, s->t, 3 * sizeof(double));
    std::memcpy(p + 3, s->q, 4 * sizeof(double));
    if (!finite_pose(p)) return fail(h, PRISM_EINVAL, "state pose is not finite");
    DeviceGuard g(h->device);
    return write_state(h, s);
}

prism_status prism_map_load(prism_handle h, const float* occ, const float* rgb, const float* var_occ,
                            const float* var_rgb) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    LAUNCH(h, launch_map_load(h->kp, h->map, occ, rgb, var_occ, var_rgb, h->stream), "map load");
    if (occ) {
        LAUNCH(h, launch_tile_bounds(h->kp, h->map, h->stream), "tile bounds");
        ++h->launches;   // and the brick bounds derived from them
    }
    return PRISM_OK;
}

prism_status prism_render_backward(prism_handle h, const double* pose7, const float* grad_depth,
                                   const float* grad_rgb, float* grad_occ, float* grad_rgb_map,
                                   double* grad_pose6, double* grad_pose7) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!pose7) return fail(h, PRISM_EINVAL, "pose is NULL");
    if (!finite_pose(pose7)) return fail(h, PRISM_EINVAL, "pose is not finite or has a zero quaternion");
    DeviceGuard g(h->device);
    PoseArg pa{};
    normalise_pose(pose7, pa.p);
    LAUNCH(h, launch_prep(h->dstate, PREP_AUX_C2W, pa, h->stream), "pose matrices");
    CK(h, cudaMemsetAsync(h->dstate->grad_pose, 0, 6 * sizeof(double), h->stream), "clear pose gradient");
    LAUNCH(h, launch_render_bwd(h->kp, h->dstate->aux, h->map, grad_depth, grad_rgb, grad_occ, grad_rgb_map,
                                h->dstate, h->stream),
           "render adjoint");
    if (!grad_pose6 && !grad_pose7) return PRISM_OK;
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    double g6[6];
    CK(h, cudaMemcpy(g6, h->dstate->grad_pose, sizeof(g6), cudaMemcpyDeviceToHost), "read pose gradient");
    if (grad_pose6) std::memcpy(grad_pose6, g6, sizeof(g6));
    if (grad_pose7) {
        // d/dt as is.  For q (given unnormalised, |q| = n, q^ = q / n), a change dq
        // rotates by dtheta = 2 vec(dq^ (x) conj(q^)) with dq^ = (dq - q^ (q^ . dq)) / n,
        // so dL/dq = G / n with G = 2 (-g . q^_v, q^_w g - q^_v x g); G . q^ = 0.
        const double* gt = g6;
        const double* gth = g6 + 3;
        const double n = std::sqrt(((pose7[3] * pose7[3] + pose7[4] * pose7[4]) + pose7[5] * pose7[5]) +
                                   pose7[6] * pose7[6]);
        const double w = pa.p[3], x = pa.p[4], y = pa.p[5], z = pa.p[6];
        const double cx = y * gth[2] - z * gth[1], cy = z * gth[0] - x * gth[2], cz = x * gth[1] - y * gth[0];
        for (int a = 0; a < 3; ++a) grad_pose7[a] = gt[a];
        grad_pose7[3] = 2.0 * -(gth[0] * x + gth[1] * y + gth[2] * z) / n;
        grad_pose7[4] = 2.0 * (w * gth[0] - cx) / n;
        grad_pose7[5] = 2.0 * (w * gth[1] - cy) / n;
        grad_pose7[6] = 2.0 * (w * gth[2] - cz) / n;
    }
    return PRISM_OK;
}

prism_status prism_rollout(prism_handle h, int32_t n_seq, int32_t k, const double* imu, const int32_t* counts,
                           const double* dt, prism_state* states, float* depth, float* rgb, int32_t* hitk) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (n_seq < 1 || k < 1) return fail(h, PRISM_EINVAL, "n_seq and k must be >= 1");
    if ((int64_t)n_seq * k > 65535) return fail(h, PRISM_EINVAL, "n_seq * k must be <= 65535");
    if (!counts || !dt) return fail(h, PRISM_EINVAL, "counts or dt is NULL");
    const int frames = n_seq * k;
    int64_t rows = 0;
    for (int f = 0; f < frames; ++f) {
        if (counts[f] < 0) return fail(h, PRISM_EINVAL, "counts must be >= 0");
        if (counts[f] > 0 && !imu) return fail(h, PRISM_EINVAL, "imu is NULL with rows to read");
        std::string why;
        if (!imu_ok(imu ? imu + 7 * rows : nullptr, counts[f], dt[f], why)) return fail(h, PRISM_EINVAL, why);
        rows += counts[f];
    }
    DeviceGuard g(h->device);
    // one block: scratch states | records | matrices | row offsets | counts | dts | IMU rows
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_rec = up((size_t)n_seq * sizeof(DevState));
    const size_t o_mat = o_rec + up((size_t)frames * sizeof(RollOut));
    const size_t o_row = o_mat + up((size_t)frames * 12 * sizeof(float));
    const size_t o_cnt = o_row + up((size_t)frames * sizeof(long long));
    const size_t o_dt = o_cnt + up((size_t)frames * sizeof(int));
    const size_t o_imu = o_dt + up((size_t)frames * sizeof(double));
    const size_t total = o_imu + up((size_t)(rows > 0 ? rows : 1) * 7 * sizeof(double));
    const size_t staged = total - o_row;   // the inputs, uploaded in one copy
    if (!h->ev_roll) CK(h, cudaEventCreateWithFlags(&h->ev_roll, cudaEventDisableTiming), "rollout event");
    if (total > h->roll_cap) {
        CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
        if (h->roll_dev) {
            cudaFree(h->roll_dev);
            h->bytes -= (int64_t)h->roll_cap;
            h->roll_dev = nullptr;
            h->roll_cap = 0;
        }
        CK(h, dalloc(h, &h->roll_dev, total), "rollout buffers");
        h->roll_cap = total;
    }
    CK(h, cudaEventSynchronize(h->ev_roll), "rollout staging reuse");
    if (staged > h->h_roll_cap) {
        if (h->h_roll) cudaFreeHost(h->h_roll);
        h->h_roll = nullptr;
        h->h_roll_cap = 0;
        CK(h, cudaMallocHost((void**)&h->h_roll, staged), "rollout staging");
        h->h_roll_cap = staged;
    }
    char* hb = h->h_roll;
    long long* h_row = (long long*)hb;
    int* h_cnt = (int*)(hb + (o_cnt - o_row));
    double* h_dt = (double*)(hb + (o_dt - o_row));
    long long r = 0;
    for (int f = 0; f < frames; ++f) {
        h_row[f] = r;
        h_cnt[f] = counts[f];
        h_dt[f] = dt[f];
        r += counts[f];
    }
    if (rows > 0) std::memcpy(hb + (o_imu - o_row), imu, (size_t)rows * 7 * sizeof(double));
    char* db = (char*)h->roll_dev;
    CK(h, cudaMemcpyAsync(db + o_row, hb, staged, cudaMemcpyHostToDevice, h->stream), "rollout upload");
    CK(h, cudaEventRecord(h->ev_roll, h->stream), "rollout event");
    RollOut* d_rec = (RollOut*)(db + o_rec);
    float* d_mats = (float*)(db + o_mat);
    LAUNCH(h, launch_rollout_states(h->kp, h->dstate, (DevState*)db, n_seq, k, (const double*)(db + o_imu),
                                    (const long long*)(db + o_row), (const int*)(db + o_cnt),
                                    (const double*)(db + o_dt), d_rec, d_mats, h->stream),
           "rollout states");
    if (depth || rgb || hitk)
        LAUNCH(h, launch_render_frames(h->kp, d_mats, frames, h->map, depth, rgb, hitk, h->dstats, h->stream),
               "rollout render");
    if (!states) return PRISM_OK;
    static_assert(sizeof(RollOut) == sizeof(prism_state), "rollout record layout");
    CK(h, cudaMemcpyAsync(states, d_rec, (size_t)frames * sizeof(RollOut), cudaMemcpyDeviceToHost, h->stream),
       "read rollout states");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    bool notpd = false;
    for (int f = 0; f < frames; ++f) {
        notpd |= states[f].reserved != 0;
        states[f].reserved = 0;
    }
    if (notpd) return fail(h, PRISM_ENOTPD, "device reported: a predicted pose covariance not positive definite");
    return PRISM_OK;
}

prism_status prism_map_descent(prism_handle h, int32_t n, const double* poses, const float* depth,
                               const float* rgb, double sd, double sc, double lr_occ, double lr_rgb,
                               double* loss) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (n < 1 || !poses || !depth || !rgb) return fail(h, PRISM_EINVAL, "n < 1 or a NULL array");
    if (!(sd > 0) || !(sc > 0) || !std::isfinite(sd) || !std::isfinite(sc))
        return fail(h, PRISM_EINVAL, "sd and sc must be finite and > 0");
    if (!(lr_occ >= 0) || !(lr_rgb >= 0) || !std::isfinite(lr_occ) || !std::isfinite(lr_rgb))
        return fail(h, PRISM_EINVAL, "step sizes must be finite and >= 0");
    for (int j = 0; j < n; ++j)
        if (!finite_pose(poses + 7 * j)) return fail(h, PRISM_EINVAL, "pose is not finite or has a zero quaternion");
    DeviceGuard g(h->device);
    const size_t npix = (size_t)h->cfg.width * h->cfg.height;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_grgb = up(h->nvox * sizeof(float));
    const size_t o_rd = o_grgb + up(3 * h->nvox * sizeof(float));
    const size_t o_rc = o_rd + up(npix * sizeof(float));
    const size_t o_rm = o_rc + up(3 * npix * sizeof(float));
    const size_t o_loss = o_rm + up(npix);
    const size_t total = o_loss + 256;
    if (!h->md_dev) CK(h, dalloc(h, &h->md_dev, total), "descent buffers");
    char* b = (char*)h->md_dev;
    float* g_occ = (float*)b;
    float* g_rgb = (float*)(b + o_grgb);
    float* r_d = (float*)(b + o_rd);
    float* r_c = (float*)(b + o_rc);
    uint8_t* r_m = (uint8_t*)(b + o_rm);
    double* d_loss = (double*)(b + o_loss);
    CK(h, cudaMemsetAsync(g_occ, 0, o_rd, h->stream), "clear gradients");
    CK(h, cudaMemsetAsync(d_loss, 0, sizeof(double), h->stream), "clear loss");
    for (int j = 0; j < n; ++j) {
        PoseArg pa{};
        normalise_pose(poses + 7 * j, pa.p);
        LAUNCH(h, launch_prep(h->dstate, PREP_AUX_C2W, pa, h->stream), "pose matrices");
        LAUNCH(h, launch_render(h->kp, h->dstate->aux, h->map, r_d, r_c, r_m, nullptr, h->dstats, nullptr, nullptr,
                                h->detail, h->stream),
               "render");
        LAUNCH(h, launch_map_loss(h->kp, r_d, r_c, r_m, depth + npix * j, rgb + 3 * npix * j, sd, sc, d_loss,
                                  h->stream),
               "loss gradients");
        LAUNCH(h, launch_render_bwd(h->kp, h->dstate->aux, h->map, r_d, r_c, g_occ, g_rgb, h->dstate, h->stream),
               "render adjoint");
    }
    LAUNCH(h, launch_map_step(h->kp, h->map, g_occ, g_rgb, lr_occ, lr_rgb, h->cfg.init_occ, h->cfg.init_rgb,
                              h->cfg.prior_var, d_loss, h->stream),
           "descent step");
    LAUNCH(h, launch_tile_bounds(h->kp, h->map, h->stream), "tile bounds");
    ++h->launches;   // and the brick bounds derived from them
    if (!loss) return PRISM_OK;
    CK(h, cudaMemcpyAsync(loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read loss");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    return PRISM_OK;
}

prism_status prism_map_store(prism_handle h, float* occ, float* rgb, float* var_occ, float* var_rgb) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    LAUNCH(h, launch_map_store(h->kp, h->map, occ, rgb, var_occ, var_rgb, h->stream), "map store");
    return PRISM_OK;
}

prism_status prism_anchor_load(prism_handle h, const double* pose7, const float* depth, const float* rgb) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!pose7 || !depth || !rgb) return fail(h, PRISM_EINVAL, "pose, depth or rgb is NULL");
    if (!finite_pose(pose7)) return fail(h, PRISM_EINVAL, "pose is not finite");
    DeviceGuard g(h->device);
    const size_t npix = (size_t)h->cfg.width * h->cfg.height;
    CK(h, cudaMemcpyAsync(h->a_depth, depth, npix * 4, cudaMemcpyDeviceToDevice, h->stream), "copy depth");
    CK(h, cudaMemcpyAsync(h->a_rgb, rgb, npix * 12, cudaMemcpyDeviceToDevice, h->stream), "copy rgb");
    double pn[7];
    normalise_pose(pose7, pn);
    CK(h, cudaMemcpyAsync(h->dstate->anchor_pose, pn, 7 * sizeof(double), cudaMemcpyHostToDevice, h->stream),
       "anchor pose");
    PhaseTimer t(h, PH_ANCHOR);
    LAUNCH(h, launch_anchor_pack(h->kp, h->a_depth, h->a_rgb, h->a0, h->a1, h->stream), "anchor pack");
    h->has_anchor = true;
    h->anchor_at_mean = false;
    return PRISM_OK;
}

prism_status prism_normal_equations(prism_handle h, const double* pose7, const float* depth, const float* rgb,
                                    double* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!pose7 || !depth || !rgb || !out) return fail(h, PRISM_EINVAL, "NULL argument");
    if (!finite_pose(pose7)) return fail(h, PRISM_EINVAL, "pose is not finite");
    if (!h->has_anchor) return fail(h, PRISM_ESTATE, "no anchor");
    DeviceGuard g(h->device);
    LAUNCH(h, launch_depth_mask(h->kp, depth, h->o_mask, h->stream), "observation mask");
    PoseArg pa{};
    normalise_pose(pose7, pa.p);
    LAUNCH(h, launch_prep(h->dstate, PREP_AUX_REL, pa, h->stream), "pose matrices");
    LAUNCH(h, launch_track(h->kp, TRACK_EXPORT, depth, rgb, h->o_mask, h->a0, h->a1, h->dstate, h->partials,
                       h->counter, h->max_blocks, h->dstats, h->stream),
       "normal equations");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    CK(h, cudaMemcpy(out, h->dstate->ne_out, 80 * sizeof(double), cudaMemcpyDeviceToHost), "read normal equations");
    return PRISM_OK;
}

prism_status prism_get_stats(prism_handle h, prism_stats* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!out) return fail(h, PRISM_EINVAL, "out is NULL");
    DeviceGuard g(h->device);
    CK(h, cudaStreamSynchronize(h->side), "stream synchronize");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    DevStats s;
    CK(h, cudaMemcpy(&s, h->dstats, sizeof(s), cudaMemcpyDeviceToHost), "read stats");
    out->render_rays = (int64_t)s.render_rays;
    out->render_samples = (int64_t)s.render_samples;
    out->render_hits = (int64_t)s.render_hits;
    out->fuse_updates = (int64_t)s.fuse_updates;
    out->fuse_colour_updates = (int64_t)s.fuse_colour_updates;
    out->track_pixels = (int64_t)s.track_pixels;
    out->render_unique_corners = (int64_t)s.render_unique_corners;
    out->kernel_launches = h->launches;
    return PRISM_OK;
}

prism_status prism_set_timing(prism_handle h, int32_t enabled) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    h->timing = enabled != 0;
    return PRISM_OK;
}

prism_status prism_set_detail_counters(prism_handle h, int32_t enabled) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    h->detail = enabled != 0;
    return PRISM_OK;
}

prism_status prism_set_cooperative(prism_handle h, int32_t enabled) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    h->coop = enabled != 0;
    return PRISM_OK;
}

prism_status prism_get_timing(prism_handle h, prism_timing* out) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    if (!out) return fail(h, PRISM_EINVAL, "out is NULL");
    DeviceGuard g(h->device);
    CK(h, cudaStreamSynchronize(h->side), "stream synchronize");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    collect_timing(h);
    out->predict_ms = h->acc_ms[PH_PREDICT];
    out->localise_ms = h->acc_ms[PH_LOCALISE];
    out->fuse_ms = h->acc_ms[PH_FUSE];
    out->render_ms = h->acc_ms[PH_RENDER];
    out->anchor_ms = h->acc_ms[PH_ANCHOR];
    out->laplace_ms = h->acc_ms[PH_LAPLACE];
    out->laplace_n = h->acc_n[PH_LAPLACE];
    out->predict_n = h->acc_n[PH_PREDICT];
    out->localise_n = h->acc_n[PH_LOCALISE];
    out->fuse_n = h->acc_n[PH_FUSE];
    out->render_n = h->acc_n[PH_RENDER];
    out->anchor_n = h->acc_n[PH_ANCHOR];
    return PRISM_OK;
}

prism_status prism_timing_reset(prism_handle h) {
    if (!h) return fail(nullptr, PRISM_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    CK(h, cudaStreamSynchronize(h->side), "stream synchronize");
    CK(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    collect_timing(h);
    for (int i = 0; i < PH_COUNT; ++i) { h->acc_ms[i] = 0.0; h->acc_n[i] = 0; }
    return PRISM_OK;
}

int64_t prism_device_bytes(prism_handle h) { return h ? h->bytes : 0; }

const char* prism_last_error(prism_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

const char* prism_status_string(int32_t st) {
    switch (st) {
        case PRISM_OK: return "ok";
        case PRISM_EINVAL: return "invalid argument";
        case PRISM_ENOMEM: return "out of memory";
        case PRISM_ECUDA: return "CUDA error";
        case PRISM_ENOTPD: return "matrix not positive definite";
        case PRISM_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

}  // extern "C"
