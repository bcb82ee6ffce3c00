// serve.cu — the serving runtime of include/prism_serve.h: streams,
// admission by device-memory budget, the batching and completion threads,
// and the captured batched step (serve.h, serve_kernels.cu).
//
// Threads.  Client threads call open / submit / close / poll.  The batching
// thread is the only one that enqueues device work: it releases the memory
// of closed streams, admits waiting streams in FIFO order while slots and
// budget allow (allocation, prior fill, optional map load, first state,
// slot-table entry), and — while fewer than max_inflight batches are on the
// device — forms a batch from the oldest pending request of every resident
// stream, uploads its frames, IMU windows and descriptor, launches the step
// and the read-back of the results, and records an event.  The completion
// thread waits for the events in order, timestamps the batch and turns its
// read-back into results.  One mutex guards the host state; device work is
// enqueued outside it, on the server's own stream, so batches run in order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "host_util.h"
#include "kernels.h"
#include "prism.h"
#include "prism_dev.cuh"
#include "prism_serve.h"
#include "serve.h"

using namespace prism;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte layout of one stream's single device allocation.
struct StreamLayout {
    size_t plane, off_map, off_tb, off_bb, off_depth, off_rgb, off_omask, off_adepth, off_argb, off_a0, off_a1,
        off_dev, off_stats, off_partials, off_counter, total;
    int max_blocks;
};

int device_sms(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 152;
    return sms;
}

StreamLayout layout_of(const prism_config* c, int storage, int sms) {
    StreamLayout L{};
    const size_t es = storage == PRISM_STORAGE_BF16 ? 2 : 4;
    const size_t npad = (size_t)(c->nx + 2) * (c->ny + 2) * (c->nz + 2);
    const size_t npix = (size_t)c->width * c->height;
    L.max_blocks = sms * 4;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += align256(bytes); return at; };
    L.plane = align256(npad * es);
    L.off_map = take(6 * L.plane);
    L.off_tb = take((size_t)(c->nx / 4) * (c->ny / 4) * (c->nz / 4) * sizeof(float2));
    KParams kp;
    fill_kparams(c, kp);
    L.off_bb = take((size_t)kp.bb_len * sizeof(float2));
    L.off_depth = take(npix * 4);
    L.off_rgb = take(npix * 12);
    L.off_omask = take(npix);
    L.off_adepth = take(npix * 4);
    L.off_argb = take(npix * 12);
    L.off_a0 = take(npix * 16);
    L.off_a1 = take(npix * 16);
    L.off_dev = take(sizeof(DevState));
    L.off_stats = take(sizeof(DevStats));
    L.off_partials = take((size_t)L.max_blocks * TRACK_NV_MAX * sizeof(float));
    L.off_counter = take(sizeof(unsigned int));
    L.total = o;
    return L;
}

struct Request {
    int64_t tag;
    const float* depth;
    const float* rgb;
    std::vector<double> imu;
    int n_imu;
    double dt;
    double t_submit;
};

struct Stream {
    int id = 0;
    prism_config cfg{};
    KParams kp{};
    prism_state s1{};
    const float* init[4] = {nullptr, nullptr, nullptr, nullptr};
    StreamLayout L{};
    int slot = -1;                 // -1: waiting for admission (or released)
    bool closing = false;
    bool released = false;
    bool started = false;          // first request taken (later ones localise)
    int inflight = 0;
    std::deque<Request> pending;
    char* block = nullptr;
};

struct RingEntry {
    BatchDesc* desc = nullptr;     // pinned host
    double* imu = nullptr;         // pinned host
    ServeOut* out = nullptr;       // pinned host
    cudaEvent_t done = nullptr;
    bool busy = false;
};

struct Inflight {
    int ring;
    int64_t seq;
    int n;
    int ids[kServeMaxSlots];
    int64_t tags[kServeMaxSlots];
    double submit[kServeMaxSlots];
};

constexpr int kImuCap = 1 << 16;   // IMU rows per batch (all members)
constexpr int kRing = 5;

}  // namespace

struct prism_server {
    prism_serve_config cfg{};
    int sms = 152;
    cudaStream_t stream = nullptr;
    unsigned long long* check = nullptr;   // bounds-check build: the first violation of any stream
    BatchGrids grids{};
    SlotDesc* d_slots = nullptr;
    SlotDesc* h_slots = nullptr;   // pinned staging of slot-table entries
    BatchDesc* d_desc = nullptr;
    double* d_imu = nullptr;
    ServeOut* d_out = nullptr;
    RingEntry ring[kRing];
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_idle;
    std::map<int, Stream*> streams;
    std::deque<int> admit_q;
    int slot_owner[kServeMaxSlots];
    int next_id = 1;
    int64_t bytes_in_use = 0, bytes_peak = 0;
    std::deque<Inflight> inflight;
    std::deque<prism_serve_result> done;
    bool stop = false;
    bool failed = false;
    std::string err;
    int64_t batches = 0, frames = 0, max_batch = 0, launches = 0, graph_launches = 0;
    std::thread worker, completer;
};

namespace {

thread_local std::string g_serve_err;

prism_status sfail(prism_server* s, prism_status st, const std::string& m) {
    if (s) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = m;
    } else {
        g_serve_err = m;
    }
    return st;
}

// Marks the server failed (called with the mutex held).
void set_failed(prism_server* S, const std::string& m) {
    S->failed = true;
    S->err = m;
    S->cv_done.notify_all();
    S->cv_idle.notify_all();
    S->cv_work.notify_all();
}

bool has_work(prism_server* S) {
    for (auto& kv : S->streams) {
        Stream* st = kv.second;
        if (st->slot >= 0 && !st->pending.empty()) return true;
    }
    return false;
}

bool idle(prism_server* S) {
    if (!S->inflight.empty()) return false;
    for (auto& kv : S->streams)
        if (!kv.second->pending.empty()) return false;
    return true;
}

// ---------------------------------------------------------------- admission
// Enqueues the set-up of a stream in slot `slot` (batching thread, mutex not
// held); *kernels counts the kernels it launched.
cudaError_t setup_stream(prism_server* S, Stream* st, int slot, int* kernels) {
    cudaError_t e;
    void* p = nullptr;
    if ((e = cudaMallocAsync(&p, st->L.total, S->stream)) != cudaSuccess) return e;
    st->block = (char*)p;
    char* b = st->block;
    const StreamLayout& L = st->L;
    SlotDesc d{};
    d.P = st->kp;
    d.M.occ = b + L.off_map;
    d.M.r = b + L.off_map + L.plane;
    d.M.g = b + L.off_map + 2 * L.plane;
    d.M.b = b + L.off_map + 3 * L.plane;
    d.M.var_occ = b + L.off_map + 4 * L.plane;
    d.M.var_rgb = b + L.off_map + 5 * L.plane;
    d.M.tb = (float2*)(b + L.off_tb);
    d.M.bb = (float2*)(b + L.off_bb);
    d.dev = (DevState*)(b + L.off_dev);
    d.stats = (DevStats*)(b + L.off_stats);
    d.depth = (float*)(b + L.off_depth);
    d.rgb = (float*)(b + L.off_rgb);
    d.o_mask = (uint8_t*)(b + L.off_omask);
    d.a_depth = (float*)(b + L.off_adepth);
    d.a_rgb = (float*)(b + L.off_argb);
    d.a0 = (float4*)(b + L.off_a0);
    d.a1 = (float4*)(b + L.off_a1);
    d.partials = (float*)(b + L.off_partials);
    d.counter = (unsigned int*)(b + L.off_counter);
    d.pstride = L.max_blocks;
    d.grid_gn = track_launch_grid(st->kp, TRACK_GN, L.max_blocks);
    d.grid_lap = track_launch_grid(st->kp, TRACK_LAPLACE, L.max_blocks);
    d.px_spec = render_px_specialisation(st->kp);
    d.tiles_x = (st->kp.W + 15) / 16;
    const prism_config& c = st->cfg;
    if ((e = launch_map_fill(st->kp, d.M, (float)c.init_occ, (float)c.init_rgb, (float)c.prior_var, S->stream)) !=
        cudaSuccess)
        return e;
    if (st->init[0] || st->init[1] || st->init[2] || st->init[3]) {
        if ((e = launch_map_load(st->kp, d.M, st->init[0], st->init[1], st->init[2], st->init[3], S->stream)) !=
            cudaSuccess)
            return e;
        *kernels += 1;
    }
    if ((e = launch_tile_bounds(st->kp, d.M, S->stream)) != cudaSuccess) return e;
    *kernels += 2;
    *kernels += 1;
    // first state, as prism_set_state writes it (normalised pose, zero anchor)
    DevState ds;
    std::memset(&ds, 0, sizeof(ds));
    double pin[7], pn[7];
    std::memcpy(pin, st->s1.t, 3 * sizeof(double));
    std::memcpy(pin + 3, st->s1.q, 4 * sizeof(double));
    normalise_pose(pin, pn);
    std::memcpy(ds.t, pn, sizeof(ds.t));
    std::memcpy(ds.q, pn + 3, sizeof(ds.q));
    std::memcpy(ds.v, st->s1.v, sizeof(ds.v));
    std::memcpy(ds.w, st->s1.w, sizeof(ds.w));
    std::memcpy(ds.cov, st->s1.cov, sizeof(ds.cov));
    ds.n_localised = st->s1.n_localised;
    // pageable source: the copy is staged before the call returns
    if ((e = cudaMemcpyAsync(d.dev, &ds, sizeof(ds), cudaMemcpyHostToDevice, S->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d.stats, 0, sizeof(DevStats), S->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d.counter, 0, sizeof(unsigned int), S->stream)) != cudaSuccess) return e;
    PoseArg pa{};
    if ((e = launch_prep(d.dev, PREP_STATE, pa, S->stream)) != cudaSuccess) return e;
    *kernels += 1;
    S->h_slots[slot] = d;
    return cudaMemcpyAsync(S->d_slots + slot, S->h_slots + slot, sizeof(SlotDesc), cudaMemcpyHostToDevice,
                           S->stream);
}

// Admits waiting streams while a slot and the budget allow (mutex held on
// entry and exit; released around device calls).
bool admit_waiting(prism_server* S, std::unique_lock<std::mutex>& lk) {
    bool any = false;
    while (!S->admit_q.empty() && !S->failed) {
        Stream* st = S->streams[S->admit_q.front()];
        int slot = -1;
        for (int i = 0; i < S->cfg.max_slots; ++i)
            if (S->slot_owner[i] < 0) { slot = i; break; }
        if (slot < 0 || S->bytes_in_use + (int64_t)st->L.total > S->cfg.hbm_budget_bytes) break;
        S->admit_q.pop_front();
        S->slot_owner[slot] = st->id;
        S->bytes_in_use += (int64_t)st->L.total;
        S->bytes_peak = std::max(S->bytes_peak, S->bytes_in_use);
        lk.unlock();
        int kernels = 0;
        cudaError_t e = setup_stream(S, st, slot, &kernels);
        lk.lock();
        S->launches += kernels;
        if (e != cudaSuccess) {
            set_failed(S, std::string("stream admission: ") + cudaGetErrorString(e));
            return any;
        }
        st->slot = slot;
        any = true;
    }
    return any;
}

// Releases closed, drained streams (mutex held).
void release_closed(prism_server* S) {
    for (auto& kv : S->streams) {
        Stream* st = kv.second;
        if (st->closing && !st->released && st->slot >= 0 && st->pending.empty() && st->inflight == 0) {
            cudaFreeAsync(st->block, S->stream);   // ordered after the stream's last batch
            st->block = nullptr;
            S->slot_owner[st->slot] = -1;
            S->bytes_in_use -= (int64_t)st->L.total;
            st->slot = -1;
            st->released = true;
        }
    }
}

// ---------------------------------------------------------------- batching
// Forms and launches one batch (mutex held on entry and exit).
void run_batch(prism_server* S, std::unique_lock<std::mutex>& lk) {
    int r = -1;
    for (int i = 0; i < kRing; ++i)
        if (!S->ring[i].busy) { r = i; break; }
    if (r < 0) return;
    RingEntry& R = S->ring[r];
    BatchDesc& B = *R.desc;
    std::memset(&B, 0, sizeof(B));
    Inflight fl{};
    fl.ring = r;
    struct Up { float* dd; float* dr; const float* hd; const float* hr; size_t npix; };
    std::vector<Up> ups;
    int imu_rows = 0;
    // members in slot order: the oldest pending request of every resident stream
    for (int slot = 0; slot < S->cfg.max_slots && B.n < kServeMaxSlots; ++slot) {
        const int id = S->slot_owner[slot];
        if (id < 0) continue;
        Stream* st = S->streams[id];
        if (st->pending.empty()) continue;
        Request& q = st->pending.front();
        const int loc = st->started ? 1 : 0;
        const int n_imu = loc ? q.n_imu : 0;
        if (imu_rows + n_imu > kImuCap) break;
        const int i = B.n++;
        BatchMember& m = B.m[i];
        m.slot = slot;
        m.localise = loc;
        m.imu_off = imu_rows;
        m.n_imu = n_imu;
        m.dt = q.dt;
        if (n_imu) std::memcpy(R.imu + 7 * imu_rows, q.imu.data(), sizeof(double) * 7 * n_imu);
        imu_rows += n_imu;
        if (loc) B.loc[B.n_loc++] = i;
        const SlotDesc& d = S->h_slots[slot];
        const int npix = st->kp.W * st->kp.H;
        B.tiles_off[i + 1] = B.tiles_off[i] + d.tiles_x * ((st->kp.H + 7) / 8);
        B.pix_off[i + 1] = B.pix_off[i] + (npix + 255) / 256;
        B.fuse_off[i + 1] = B.fuse_off[i] + st->kp.nbx * st->kp.nby * st->kp.nbz;
        B.brick_off[i + 1] = B.brick_off[i] + st->kp.bb_len - st->kp.bb_off[st->kp.nlev];
        ups.push_back({d.depth, d.rgb, q.depth, q.rgb, (size_t)npix});
        fl.ids[i] = id;
        fl.tags[i] = q.tag;
        fl.submit[i] = q.t_submit;
        st->started = true;
        st->inflight += 1;
        st->pending.pop_front();
    }
    for (int k = 0; k < B.n_loc; ++k) {
        const SlotDesc& d = S->h_slots[B.m[B.loc[k]].slot];
        B.gn_off[k + 1] = B.gn_off[k] + d.grid_gn;
        B.lap_off[k + 1] = B.lap_off[k] + d.grid_lap;
    }
    if (B.n == 0) return;
    fl.n = B.n;
    fl.seq = S->batches++;
    S->max_batch = std::max<int64_t>(S->max_batch, B.n);
    R.busy = true;
    S->inflight.push_back(fl);
    const int n_gn = S->cfg.n_gn;
    const bool use_graph = S->gexec != nullptr;
    lk.unlock();
    NvtxRange range("prism serve batch");
    cudaError_t e = cudaSuccess;
    for (const Up& u : ups) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(u.dd, u.hd, u.npix * 4, cudaMemcpyDefault, S->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u.dr, u.hr, u.npix * 12, cudaMemcpyDefault, S->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_desc, R.desc, sizeof(BatchDesc), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess && imu_rows)
        e = cudaMemcpyAsync(S->d_imu, R.imu, sizeof(double) * 7 * imu_rows, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) {
        if (use_graph) e = cudaGraphLaunch(S->gexec, S->stream);
        else e = launch_batch_step(S->d_slots, S->d_desc, S->d_imu, S->d_out, n_gn, S->cfg.storage == PRISM_STORAGE_BF16,
                                   S->grids, S->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.out, S->d_out, sizeof(ServeOut) * B.n, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaEventRecord(R.done, S->stream);
    lk.lock();
    S->launches += 8 + n_gn;
    if (use_graph) S->graph_launches += 1;
    if (e != cudaSuccess) set_failed(S, std::string("batch launch: ") + cudaGetErrorString(e));
    S->cv_done.notify_all();   // wakes the completion thread
}

void worker_main(prism_server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop || S->failed) break;
        release_closed(S);
        admit_waiting(S, lk);
        if (S->failed) break;
        bool ring_free = false;
        for (int i = 0; i < kRing; ++i) ring_free = ring_free || !S->ring[i].busy;
        if ((int)S->inflight.size() < S->cfg.max_inflight && ring_free && has_work(S)) {
            run_batch(S, lk);
            continue;
        }
        S->cv_work.wait(lk);
    }
}

void completer_main(prism_server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (S->inflight.empty() && !S->stop && !S->failed) S->cv_done.wait(lk);
        if (S->inflight.empty() || S->failed) break;
        Inflight fl = S->inflight.front();
        cudaEvent_t ev = S->ring[fl.ring].done;
        lk.unlock();
        cudaError_t e = cudaEventSynchronize(ev);
        const double t = now_s();
        lk.lock();
        S->inflight.pop_front();
        if (e != cudaSuccess) {
            set_failed(S, std::string("batch execution: ") + cudaGetErrorString(e));
            break;
        }
        const ServeOut* out = S->ring[fl.ring].out;
        for (int i = 0; i < fl.n; ++i) {
            prism_serve_result res;
            std::memset(&res, 0, sizeof(res));
            res.stream_id = fl.ids[i];
            res.tag = fl.tags[i];
            res.batch = fl.seq;
            res.batch_size = fl.n;
            res.submit_s = fl.submit[i];
            res.done_s = t;
            res.latency_ms = 1e3 * (t - fl.submit[i]);
            res.status = out[i].flags ? PRISM_ENOTPD : PRISM_OK;
            std::memcpy(res.state.t, out[i].t, sizeof(res.state.t));
            std::memcpy(res.state.q, out[i].q, sizeof(res.state.q));
            std::memcpy(res.state.v, out[i].v, sizeof(res.state.v));
            std::memcpy(res.state.w, out[i].w, sizeof(res.state.w));
            std::memcpy(res.state.cov, out[i].cov, sizeof(res.state.cov));
            res.state.n_localised = out[i].n_localised;
            S->done.push_back(res);
            auto it = S->streams.find(fl.ids[i]);
            if (it != S->streams.end()) it->second->inflight -= 1;
        }
        S->frames += fl.n;
        S->ring[fl.ring].busy = false;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
        if (idle(S)) S->cv_idle.notify_all();
    }
}

bool valid_serve_config(const prism_serve_config* c, std::string& why) {
    if (!c) { why = "config is NULL"; return false; }
    if (c->hbm_budget_bytes <= 0) { why = "hbm_budget_bytes must be > 0"; return false; }
    if (c->max_slots < 1 || c->max_slots > PRISM_SERVE_MAX_SLOTS) { why = "max_slots out of range"; return false; }
    if (c->storage != PRISM_STORAGE_F32 && c->storage != PRISM_STORAGE_BF16) { why = "bad storage"; return false; }
    if (c->n_gn < 1 || c->n_gn > kServeMaxCounters - 2) { why = "n_gn must be in [1, 62]"; return false; }
    if (c->max_inflight < 1 || c->max_inflight > 4) { why = "max_inflight must be in [1, 4]"; return false; }
    return true;
}

void free_server(prism_server* S) {
    for (auto& kv : S->streams) {
        if (kv.second->block) cudaFreeAsync(kv.second->block, S->stream);
        delete kv.second;
    }
    S->streams.clear();
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->check) cudaFree(S->check);
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->graph) cudaGraphDestroy(S->graph);
    for (auto& R : S->ring) {
        if (R.desc) cudaFreeHost(R.desc);
        if (R.imu) cudaFreeHost(R.imu);
        if (R.out) cudaFreeHost(R.out);
        if (R.done) cudaEventDestroy(R.done);
    }
    if (S->h_slots) cudaFreeHost(S->h_slots);
    if (S->d_slots) cudaFree(S->d_slots);
    if (S->d_desc) cudaFree(S->d_desc);
    if (S->d_imu) cudaFree(S->d_imu);
    if (S->d_out) cudaFree(S->d_out);
    if (S->stream) cudaStreamDestroy(S->stream);
}

}  // namespace

extern "C" {

void prism_serve_config_default(prism_serve_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->hbm_budget_bytes = (int64_t)64 << 30;
    c->max_slots = 32;
    c->storage = PRISM_STORAGE_BF16;
    c->n_gn = 10;
    c->max_inflight = 2;
    c->use_graph = 1;
    c->device = 0;
}

int64_t prism_serve_stream_bytes(const prism_config* cfg, int32_t storage) {
    std::string why;
    if (!valid_config(cfg, why)) return -1;
    if (storage != PRISM_STORAGE_F32 && storage != PRISM_STORAGE_BF16) return -1;
    int dev = 0;
    int sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) sms = device_sms(dev);
    else cudaGetLastError();
    return (int64_t)layout_of(cfg, storage, sms).total;
}

prism_status prism_serve_create(const prism_serve_config* c, prism_server_handle* out) {
    std::string why;
    if (!out) return sfail(nullptr, PRISM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_serve_config(c, why)) return sfail(nullptr, PRISM_EINVAL, "invalid serve config: " + why);
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(nullptr, PRISM_EINVAL, "bad device ordinal");
    }
    prism_server* S = new (std::nothrow) prism_server();
    if (!S) return sfail(nullptr, PRISM_ENOMEM, "host allocation failed");
    S->cfg = *c;
    S->sms = device_sms(c->device);
    for (int i = 0; i < kServeMaxSlots; ++i) S->slot_owner[i] = -1;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    ok(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
    ok(cudaMalloc(&S->d_slots, sizeof(SlotDesc) * kServeMaxSlots));
    ok(cudaMallocHost(&S->h_slots, sizeof(SlotDesc) * kServeMaxSlots));
    ok(cudaMalloc(&S->d_desc, sizeof(BatchDesc)));
    ok(cudaMalloc(&S->d_imu, sizeof(double) * 7 * kImuCap));
    ok(cudaMalloc(&S->d_out, sizeof(ServeOut) * kServeMaxSlots));
#ifdef PRISM_CHECKED
    ok(cudaMalloc(&S->check, sizeof(unsigned long long)));
    if (e == cudaSuccess) ok(cudaMemsetAsync(S->check, 0, sizeof(unsigned long long), S->stream));
#endif
    for (auto& R : S->ring) {
        ok(cudaMallocHost(&R.desc, sizeof(BatchDesc)));
        ok(cudaMallocHost(&R.imu, sizeof(double) * 7 * kImuCap));
        ok(cudaMallocHost(&R.out, sizeof(ServeOut) * kServeMaxSlots));
        ok(cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming));
    }
    if (e == cudaSuccess) ok(cudaMemsetAsync(S->d_slots, 0, sizeof(SlotDesc) * kServeMaxSlots, S->stream));
    if (e == cudaSuccess) ok(batch_grids(c->storage == PRISM_STORAGE_BF16, &S->grids));
    if (e == cudaSuccess && c->use_graph) {
        cudaStream_t cap = nullptr;
        ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        if (e == cudaSuccess) ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            cudaError_t le = launch_batch_step(S->d_slots, S->d_desc, S->d_imu, S->d_out, c->n_gn,
                                               c->storage == PRISM_STORAGE_BF16, S->grids, cap);
            cudaError_t ce = cudaStreamEndCapture(cap, &S->graph);
            ok(le);
            ok(ce);
        }
        if (e == cudaSuccess) ok(cudaGraphInstantiate(&S->gexec, S->graph, 0));
        if (cap) cudaStreamDestroy(cap);
    }
    if (e == cudaSuccess) ok(cudaStreamSynchronize(S->stream));
    if (e != cudaSuccess) {
        const std::string m = std::string("server set-up: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_server(S);
        delete S;
        return sfail(nullptr, e == cudaErrorMemoryAllocation ? PRISM_ENOMEM : PRISM_ECUDA, m);
    }
    S->worker = std::thread(worker_main, S);
    S->completer = std::thread(completer_main, S);
    *out = S;
    return PRISM_OK;
}

prism_status prism_serve_destroy(prism_server_handle S) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->completer.joinable()) S->completer.join();
    cudaSetDevice(S->cfg.device);
    free_server(S);
    delete S;
    return PRISM_OK;
}

prism_status prism_serve_open(prism_server_handle S, const prism_config* cfg, const prism_state* s1,
                              const float* occ, const float* rgb, const float* var_occ, const float* var_rgb,
                              int32_t* stream_id) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    if (!stream_id) return sfail(S, PRISM_EINVAL, "stream_id is NULL");
    std::string why;
    if (!valid_config(cfg, why)) return sfail(S, PRISM_EINVAL, "invalid config: " + why);
    if (cfg->optimiser != PRISM_OPT_GAUSS_NEWTON)
        return sfail(S, PRISM_EINVAL, "the server localises with Gauss-Newton (optimiser 0)");
    if (s1) {
        double p[7];
        std::memcpy(p, s1->t, 3 * sizeof(double));
        std::memcpy(p + 3, s1->q, 4 * sizeof(double));
        if (!finite_pose(p)) return sfail(S, PRISM_EINVAL, "initial state pose is not finite");
    }
    Stream* st = new (std::nothrow) Stream();
    if (!st) return sfail(S, PRISM_ENOMEM, "host allocation failed");
    st->cfg = *cfg;
    st->cfg.storage = S->cfg.storage;
    st->cfg.n_gn = S->cfg.n_gn;
    fill_kparams(&st->cfg, st->kp);
    st->kp.check = S->check;
    if (s1) {
        st->s1 = *s1;
    } else {
        std::memset(&st->s1, 0, sizeof(st->s1));
        st->s1.q[0] = 1.0;
        for (int i = 0; i < 12; ++i) st->s1.cov[13 * i] = 1e-8;
    }
    st->init[0] = occ;
    st->init[1] = rgb;
    st->init[2] = var_occ;
    st->init[3] = var_rgb;
    st->L = layout_of(&st->cfg, S->cfg.storage, S->sms);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->failed) { delete st; return PRISM_ECUDA; }
    if ((int64_t)st->L.total > S->cfg.hbm_budget_bytes) {
        delete st;
        S->err = "stream footprint exceeds the whole budget";
        return PRISM_ENOMEM;
    }
    st->id = S->next_id++;
    S->streams[st->id] = st;
    S->admit_q.push_back(st->id);
    *stream_id = st->id;
    S->cv_work.notify_all();
    return PRISM_OK;
}

prism_status prism_serve_submit(prism_server_handle S, int32_t stream_id, const double* imu, int32_t n, double dt,
                                const float* depth, const float* rgb, int64_t tag) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    if (!depth || !rgb) return sfail(S, PRISM_EINVAL, "depth or rgb is NULL");
    if (n < 0 || (n > 0 && !imu)) return sfail(S, PRISM_EINVAL, "bad IMU window");
    if (n > kImuCap) return sfail(S, PRISM_EINVAL, "IMU window too long");
    if (!(dt > 0) || !std::isfinite(dt)) return sfail(S, PRISM_EINVAL, "dt must be finite and > 0");
    for (int i = 0; i < 7 * n; ++i)
        if (!std::isfinite(imu[i])) return sfail(S, PRISM_EINVAL, "non-finite IMU value");
    Request q;
    q.tag = tag;
    q.depth = depth;
    q.rgb = rgb;
    q.n_imu = n;
    q.dt = dt;
    if (n > 0) q.imu.assign(imu, imu + 7 * (size_t)n);
    q.t_submit = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->failed) return PRISM_ECUDA;
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end()) { S->err = "unknown stream"; return PRISM_EINVAL; }
    if (it->second->closing) { S->err = "stream is closed"; return PRISM_ESTATE; }
    it->second->pending.push_back(std::move(q));
    S->cv_work.notify_all();
    return PRISM_OK;
}

prism_status prism_serve_close(prism_server_handle S, int32_t stream_id) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end()) { S->err = "unknown stream"; return PRISM_EINVAL; }
    Stream* st = it->second;
    st->closing = true;
    if (st->slot < 0 && !st->released) {   // never admitted: leave the queue, drop its requests
        S->admit_q.erase(std::remove(S->admit_q.begin(), S->admit_q.end(), st->id), S->admit_q.end());
        st->pending.clear();
        st->released = true;
    }
    S->cv_work.notify_all();
    if (idle(S)) S->cv_idle.notify_all();
    return PRISM_OK;
}

prism_status prism_serve_poll(prism_server_handle S, prism_serve_result* out, int32_t max, int32_t timeout_ms,
                              int32_t* n) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    if (!out || !n || max < 0) return sfail(S, PRISM_EINVAL, "bad poll arguments");
    *n = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && timeout_ms > 0 && !S->failed)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !S->done.empty() || S->failed; });
    int k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    *n = k;
    if (k == 0 && S->failed) return PRISM_ECUDA;
    return PRISM_OK;
}

prism_status prism_serve_drain(prism_server_handle S, int32_t timeout_ms) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_idle.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return idle(S) || S->failed; });
    if (S->failed) return PRISM_ECUDA;
    if (!ok) { S->err = "drain timed out"; return PRISM_ESTATE; }
    return PRISM_OK;
}

prism_status prism_serve_check_status(prism_server_handle S, uint64_t* word) {
    if (!S || !word) return sfail(S, PRISM_EINVAL, "server or word is NULL");
    *word = 0;
    if (!S->check) return PRISM_OK;
    unsigned long long v = 0;
    cudaError_t e = cudaStreamSynchronize(S->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, S->check, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(S, PRISM_ECUDA, std::string("check status: ") + cudaGetErrorString(e));
    }
    *word = v;
    return PRISM_OK;
}

prism_status prism_serve_get_stats(prism_server_handle S, prism_serve_stats* out) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    if (!out) return sfail(S, PRISM_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->batches = S->batches;
    out->frames = S->frames;
    out->max_batch = S->max_batch;
    out->bytes_in_use = S->bytes_in_use;
    out->bytes_peak = S->bytes_peak;
    out->budget = S->cfg.hbm_budget_bytes;
    for (auto& kv : S->streams) {
        if (kv.second->slot >= 0) out->streams_resident += 1;
        if (!kv.second->released) out->streams_open += 1;
    }
    out->streams_queued = (int32_t)S->admit_q.size();
    out->kernel_launches = S->launches;
    out->graph_launches = S->graph_launches;
    return S->failed ? PRISM_ECUDA : PRISM_OK;
}

prism_status prism_serve_map_store(prism_server_handle S, int32_t stream_id, float* occ, float* rgb, float* var_occ,
                                   float* var_rgb) {
    if (!S) return sfail(nullptr, PRISM_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second->slot < 0) {
        S->err = "stream is not resident";
        return PRISM_ESTATE;
    }
    const SlotDesc d = S->h_slots[it->second->slot];
    // enqueued under the mutex so that no release can free the map first
    cudaError_t e = launch_map_store(d.P, d.M, occ, rgb, var_occ, var_rgb, S->stream);
    if (e == cudaSuccess) S->launches += 1;
    lk.unlock();
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) return sfail(S, PRISM_ECUDA, std::string("map store: ") + cudaGetErrorString(e));
    return PRISM_OK;
}

const char* prism_serve_last_error(prism_server_handle S) {
    if (!S) return g_serve_err.c_str();
    std::lock_guard<std::mutex> lk(S->mu);
    thread_local std::string copy;
    copy = S->err;
    return copy.c_str();
}

}  // extern "C"
