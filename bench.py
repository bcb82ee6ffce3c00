#!/usr/bin/env python3
"""Throughput of the PRISM filter hot path (arXiv 2212.02988) on GB300.

One step is one full filter step through the C ABI (prism_step): predict
from the frame's IMU window, localise (10 Gauss-Newton passes and the
Laplace pass), fuse the frame into the map, render the next anchor — on
one 640x480 RGB-D frame against a 256^3 map (the workload's defaults).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is frames/s of the whole job with the frames
already on the device; `e2e` is the same metric through the host-frame
form of the call (prism_step_host), each frame handed over in pinned host
memory and uploaded by the library, the state read back every step.  Under torchrun each rank runs an independent filter replica on
its own GPU (the filter does not shard); the max elapsed time over ranks is
used.  `--impl reference` times the FP64 CPU oracle on the host instead.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filter frames/s & p50/p99 step latency; render Mrays/s and % of HBM peak"
UNIT = "frames/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="room256_640x480")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=6)
    ap.add_argument("--cpu-single-steps", type=int, default=2)
    ap.add_argument("--reference-budget-s", type=float, default=150.0)
    ap.add_argument("--serve", action="store_true",
                    help="run only the multi-stream serving workload (32 streams) and print its JSON line")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="length of the serving run (default 120 with --serve, 12 inside the default run)")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving run of the default bench")
    ap.add_argument("--no-bf16", action="store_true", help="skip the bf16-map sub-run (configuration 3)")
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    return ap.parse_args(argv)


# ------------------------------------------------------------------ ranks
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def combine_over_ranks(elapsed_s: float, units: float, group=None):
    """(max elapsed over ranks, sum of units over ranks); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return elapsed_s, units
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- roofline
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# the sources each profiled kernel is built from (a committed ncu summary
# counts only while their hash matches)
KERNEL_SOURCES = {"k_render": ("render.cu", "render_dev.cuh", "prism_dev.cuh"),
                  "k_fuse_list": ("fuse.cu", "fuse_dev.cuh", "prism_dev.cuh"),
                  "k_track_gn": ("track.cu", "track_dev.cuh", "prism_dev.cuh", "linalg64.cuh")}


def source_hash(kernel: str = "k_render"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2212_02988_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def render_source_hash():
    return source_hash("k_render")


def profiled_traffic(workload: str, kernel: str = "k_render"):
    """DRAM bytes per launch (or, where the summary gives it, per pass) of
    `kernel` from its committed ncu summary, if it was taken on the current
    sources; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("source_sha256", "dram_bytes_per_launch", "dram_bytes_per_pass")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != source_hash(kernel):
        return None
    try:
        return int(float(vals.get("dram_bytes_per_pass", vals.get("dram_bytes_per_launch"))))
    except (TypeError, ValueError):
        return None


def timed_filter(cfg, s1, maps, w, D, C, imus, K, W, T, local_rank):
    """A filter on the device-resident frames: W warm-up steps (with the
    render's detail counters on), K timed steps bracketed by a barrier and a
    device synchronisation, clocks sampled meanwhile, then T steps with the
    library's phase timers on (their events break the launch overlap
    between phases, so they stay off in the timed loop).  Returns the
    filter (still open) and the measurements."""
    import torch
    from paper_2212_02988_gb300 import Filter
    F = Filter(cfg, s1, device=local_rank)
    F.map_load(*maps)
    F.step(None, w.dt, D[0], C[0])
    F.set_detail_counters(True)
    st_w0 = F.stats()
    for i in range(1, 1 + W):
        F.step(imus[i], w.dt, D[i], C[i])
    st_w1 = F.stats()
    F.set_detail_counters(False)
    st0 = F.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()   # as timeit does: no cyclic collection pauses inside the timed loops
    sampler.start()
    e_start.record()
    for j in range(K):
        i = 1 + W + j
        ev[j][0].record()
        F.step(imus[i], w.dt, D[i], C[i])
        ev[j][1].record()
    e_end.record()
    torch.cuda.synchronize()
    gc.enable()
    barrier()
    clocks = sampler.stop()
    st1 = F.stats()
    F.set_timing(True)
    F.timing_reset()
    for j in range(T):
        i = 1 + W + K + j
        F.step(imus[i], w.dt, D[i], C[i])
    torch.cuda.synchronize()
    tm = F.timing()
    F.set_timing(False)
    return F, {"total_ms": e_start.elapsed_time(e_end), "step_ms": [a.elapsed_time(b) for a, b in ev],
               "tm": tm, "clocks": clocks, "st0": st0, "st1": st1, "st_w0": st_w0, "st_w1": st_w1}


def render_bytes(run, K, storage):
    """Render byte counts per launch: G (logical gathered voxel bytes of the
    evaluated samples) and U (per-ray unique bytes, from the fraction of
    distinct corners counted in the warm-up steps)."""
    st0, st1, w0, w1 = run["st0"], run["st1"], run["st_w0"], run["st_w1"]
    d = {k: st1[k] - st0[k] for k in st1}
    warm = {k: w1[k] - w0[k] for k in w1}
    b = 2 if storage == "bf16" else 4
    samp, hits = d["render_samples"] / max(K, 1), d["render_hits"] / max(K, 1)
    u_ratio = warm["render_unique_corners"] / max(warm["render_samples"] * 8, 1)
    return {"rays": d["render_rays"] / max(K, 1), "samples": samp, "hits": hits, "bytes_per_corner": b,
            "G": samp * 8 * b + hits * 2 * 8 * 3 * b, "U": samp * 8 * b * u_ratio + hits * 8 * 3 * b}


def gn_pass_ms(tm, n_gn):
    """The Gauss-Newton pass's live duration: the localisation phase less its
    Laplace pass, over the passes (the first also evaluates the depth
    validity)."""
    return (tm["localise_ms"] / max(tm["localise_n"], 1) - tm["laplace_ms"] / max(tm["laplace_n"], 1)) / n_gn


# the localisation pass's algorithmic bytes per observed pixel (observation
# 16 B: depth and colour; anchor gathers 56 B: the nearest pixel's normal and
# depth, the bilinear colour taps)
GN_BYTES_PER_PIXEL = 72


# ------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import synth
    from paper_2212_02988_gb300 import Filter, config, make_state
    from synth.gpu_frames import raycast_frames

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.PRESETS[args.workload]
    K, W = args.steps, max(args.warmup, 0)
    T = min(K, 60)   # steps after the timed ones with the library's phase timers on
    n_frames = 1 + W + K + T
    seq = synth.Sequence(w, n_frames=n_frames, seed=w.seed + 100 * rank)
    occ, rgb, vo, vr = seq.settled_map()
    maps = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (occ, rgb, vo, vr)]
    D, C = [], []
    for c0 in range(0, n_frames, 64):
        d, c = raycast_frames(seq, range(c0, min(n_frames, c0 + 64)), dev)
        D.append(d)
        C.append(c)
    D, C = torch.cat(D), torch.cat(C)
    imus = [None] + [seq.imu_window(i) for i in range(1, n_frames)]
    storage = "bf16" if w.storage == "bf16" else "f32"
    cfg = config(w.n, w.extent, w.width, w.height, storage=storage)
    s1 = make_state(seq.pose7(0), seq.velocity(0))

    # ---- device-resident run ----
    F, run = timed_filter(cfg, s1, maps, w, D, C, imus, K, W, T, local_rank)
    total_ms, step_ms, tm, clocks = run["total_ms"], run["step_ms"], run["tm"], run["clocks"]
    st0, st1, st_w0, st_w1 = run["st0"], run["st1"], run["st_w0"], run["st_w1"]
    elapsed, frames = combine_over_ranks(total_ms / 1000.0, float(K))
    # render adjoint (config with the differentiation path): timed separately,
    # at the final state's pose, with resident upstream gradients
    adj = None
    n_adj = min(K, 50)
    from paper_2212_02988_gb300 import state_arrays
    pose_last = state_arrays(F.get_state())["pose"]
    # Samples of the full march (every d_k = k eps, no brick skipping) against
    # the samples the kernel evaluates, at the final pose and map: the render
    # skips the samples whose bricks cannot hold a hit, so the method's march
    # gathers `full_ratio` times the bytes the kernel reads.
    m_last = F.map_store()
    F0 = Filter(config(w.n, w.extent, w.width, w.height, storage=storage, skip_empty=0), s1, device=local_rank)
    F0.map_load(m_last["occ"], m_last["rgb"], m_last["var_occ"], m_last["var_rgb"])
    counts = []
    for Fx in (F, F0):
        Fx.set_detail_counters(True)
        a = Fx.stats()
        Fx.render(pose_last)
        torch.cuda.synchronize()
        counts.append(Fx.stats()["render_samples"] - a["render_samples"])
        Fx.set_detail_counters(False)
    F0.close()
    del m_last
    full_ratio = counts[1] / max(counts[0], 1)
    if n_adj > 0:
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        gD = torch.randn((w.height, w.width), generator=gen, device=dev)
        gC = torch.randn((w.height, w.width, 3), generator=gen, device=dev)
        go = torch.zeros(maps[0].shape, device=dev)
        gr = torch.zeros(maps[1].shape, device=dev)
        F.render_backward(pose_last, gD, gC, go, gr)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(n_adj):   # device-side gradients only: no host read-back per call
            F.render_backward_async(pose_last, gD, gC, go, gr)
        a1.record()
        torch.cuda.synchronize()
        adj_ms = a0.elapsed_time(a1) / n_adj
        adj = {"ms_per_call": adj_ms, "calls": n_adj, "mrays_per_s": w.width * w.height / (adj_ms * 1e-3) / 1e6,
               "note": "prism_render_backward (pose + per-voxel gradients, FP32 atomics), not part of the step"}

    # Predictive rollouts (App. I) from the final belief: 32 candidate control
    # sequences of 10 frames (the recorded IMU windows with a constant offset
    # on the specific force and the angular rate per candidate), the states
    # read back and every predicted frame rendered, in one call; not part of
    # the step.
    roll = None
    n_roll = min(K, 5)
    if n_roll > 0:
        n_seq, k_roll = 32, 10
        rs = np.random.default_rng(11)
        base = [imus[1 + W + j % K] for j in range(k_roll)]
        wins = []
        for _ in range(n_seq):
            da, dg = rs.normal(0, 0.5, 3), rs.normal(0, 0.2, 3)
            cand = []
            for x in base:
                y = x.copy()
                y[:, 1:4] += da
                y[:, 4:7] += dg
                cand.append(y)
            wins.append(cand)
        bufs = F.rollout(wins, w.dt)   # allocates the image buffers (untimed)
        bufs = {"depth": bufs["depth"], "rgb": bufs["rgb"]}
        F.rollout(wins, w.dt, out=bufs)
        torch.cuda.synchronize()
        a = F.stats()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_r = time.perf_counter()
        r0.record()
        for _ in range(n_roll):
            F.rollout(wins, w.dt, out=bufs)   # states read back: each call synchronises
        r1.record()
        torch.cuda.synchronize()
        roll_wall = (time.perf_counter() - t_r) / n_roll
        roll_dev = r0.elapsed_time(r1) / n_roll
        bst = F.stats()
        fr = n_seq * k_roll
        roll_samples = (bst["render_samples"] - a["render_samples"]) / n_roll
        roll_hits = (bst["render_hits"] - a["render_hits"]) / n_roll
        s0, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(n_roll):
            F.rollout(wins, w.dt, images=False)
        s1e.record()
        torch.cuda.synchronize()
        roll = {"sequences": n_seq, "frames_per_sequence": k_roll, "calls": n_roll,
                "ms_per_call": roll_wall * 1e3, "device_ms_per_call": roll_dev,
                "states_only_ms_per_call": s0.elapsed_time(s1e) / n_roll,
                "predicted_frames_per_s": fr / roll_wall,
                "render_mrays_per_s": fr * w.width * w.height / roll_wall / 1e6,
                "samples_per_frame": roll_samples / fr, "hits_per_frame": roll_hits / fr,
                "note": "prism_rollout: states (one block per sequence) + all 320 images in one render "
                        "launch, wall time per call with the states read back; not part of the step"}
    F.close()

    # Closed-form against gradient-descent mapping (Sec. 4.4); not part of the step.
    mapping = mapping_comparison(dev) if K > 0 else None

    # The paper's pose optimiser (App. F.2: Adam, momentum off, 1000 steps of
    # 200 pixels) on the same frames, for its localisation time beside the
    # Gauss-Newton passes it is the alternative to; not part of the step.
    adam = None
    n_adam = min(K, 8)
    if n_adam > 0:
        Fa = Filter(config(w.n, w.extent, w.width, w.height, storage=storage, optimiser=1), s1, device=local_rank)
        Fa.map_load(*maps)
        Fa.step(None, w.dt, D[0], C[0])
        Fa.step(imus[1], w.dt, D[1], C[1])
        Fa.set_timing(True)
        Fa.timing_reset()
        for i in range(2, 2 + n_adam):
            Fa.step(imus[i], w.dt, D[i], C[i])
        torch.cuda.synchronize()
        ta = Fa.timing()
        ca = Fa.cfg
        adam = {"ms_per_localise": ta["localise_ms"] / max(ta["localise_n"], 1), "frames": n_adam,
                "steps": ca.adam_steps, "pixels_per_step": ca.adam_pixels,
                "note": "Adam with momentum off (App. F.2) and the Laplace pass, one block; not part of the step"}
        Fa.close()

    d_st = {k: st1[k] - st0[k] for k in st1}
    rb = render_bytes(run, K, storage)
    rays_per, samp_per, G, U, b = rb["rays"], rb["samples"], rb["G"], rb["U"], rb["bytes_per_corner"]
    render_ms = tm["render_ms"] / max(tm["render_n"], 1)
    peak, peak_kind = measured_peaks()
    achieved_G = G / (render_ms * 1e-3) / 1e9
    achieved_U = U / (render_ms * 1e-3) / 1e9
    # the map update: the map-plane bytes its updates read and write
    fuse_ms = tm["fuse_ms"] / max(tm["fuse_n"], 1)
    fb = 2 if storage == "bf16" else 4
    fuse_upd, fuse_col = d_st["fuse_updates"] / max(K, 1), d_st["fuse_colour_updates"] / max(K, 1)
    fuse_bytes = fuse_upd * 2 * 2 * fb + fuse_col * 4 * 2 * fb
    # the dominant kernel by device time: the Gauss-Newton pass
    npx = w.width * w.height
    gn_ms = gn_pass_ms(tm, cfg.n_gn)
    gn_bytes = GN_BYTES_PER_PIXEL * npx
    loc_ms = tm["localise_ms"] / max(tm["localise_n"], 1)

    # bf16 map storage (configuration 3: the same 256^3 map and 640x480 frames)
    bf16 = None
    if not args.no_bf16 and storage == "f32" and K > 0:
        wb = synth.PRESETS[w.name + "_bf16"] if (w.name + "_bf16") in synth.PRESETS else None
        if wb is not None:
            Kb, Tb = min(K, 200), min(T, 40)
            nb = 1 + W + Kb + Tb
            sb = synth.Sequence(wb, n_frames=nb, seed=wb.seed + 100 * rank)
            mb = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in sb.settled_map()]
            Db, Cb = [], []
            for c0 in range(0, nb, 64):
                d, c = raycast_frames(sb, range(c0, min(nb, c0 + 64)), dev)
                Db.append(d)
                Cb.append(c)
            Db, Cb = torch.cat(Db), torch.cat(Cb)
            ib = [None] + [sb.imu_window(i) for i in range(1, nb)]
            cfgb = config(wb.n, wb.extent, wb.width, wb.height, storage="bf16")
            Fb, rbn = timed_filter(cfgb, make_state(sb.pose7(0), sb.velocity(0)), mb, wb, Db, Cb, ib, Kb, W, Tb,
                                   local_rank)
            Fb.close()
            tb = rbn["tm"]
            rbb = render_bytes(rbn, Kb, "bf16")
            rms = tb["render_ms"] / max(tb["render_n"], 1)
            gnb = gn_pass_ms(tb, cfgb.n_gn)
            bf16 = {"workload": wb.name, "steps": Kb, "warmup": W,
                    "frames_per_s": Kb / (rbn["total_ms"] * 1e-3), "ms_per_step": rbn["total_ms"] / Kb,
                    "p50_step_ms": statistics.median(rbn["step_ms"]),
                    "p99_step_ms": float(np.percentile(rbn["step_ms"], 99)),
                    "phase_ms_per_step": {k[:-3]: tb[k] / max(tb[k[:-3] + "_n"], 1) for k in
                                          ("predict_ms", "localise_ms", "fuse_ms", "render_ms", "anchor_ms")},
                    "gauss_newton_pass_ms": gnb,
                    "render_mrays_per_s": rbb["rays"] / (rms * 1e-3) / 1e6,
                    "render_samples_per_launch": rbb["samples"],
                    "render_frac_unique": rbb["U"] / (rms * 1e-3) / 1e9 / peak,
                    "render_frac_gathered": rbb["G"] / (rms * 1e-3) / 1e9 / peak,
                    "clocks": rbn["clocks"],
                    "note": "map means and variances stored in bf16 (2 B a value), render and fuse math FP32, "
                            "6x6 solve and state covariance FP64; its own seeded scene"}
            del Db, Cb, mb

    # ---- end to end through the same public call ----
    e2e = calib = None
    if not args.no_e2e:
        # frames in pinned host memory, handed to prism_step_host, which
        # uploads each one on its prediction stream behind the previous
        # posterior (overlapping the previous step's map update and render)
        Dh = D.cpu().pin_memory()
        Ch = C.cpu().pin_memory()
        F2 = Filter(cfg, s1, device=local_rank)
        F2.map_load(*maps)
        F2.step_host(None, w.dt, Dh[0], Ch[0])
        for i in range(1, 1 + W):
            F2.step_host(imus[i], w.dt, Dh[i], Ch[i])
        torch.cuda.synchronize()
        barrier()
        lat, e2e_states = [], []
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for j in range(K):
            i = 1 + W + j
            ts = time.perf_counter()
            e2e_states.append(F2.step_host(imus[i], w.dt, Dh[i], Ch[i], want_state=True))   # state read back
            lat.append((time.perf_counter() - ts) * 1e3)
        torch.cuda.synchronize()   # the last step's map update and render are part of the run
        e2e_s = time.perf_counter() - t0
        gc.enable()
        barrier()
        e2e_elapsed, e2e_frames = combine_over_ranks(e2e_s, float(K))
        F2.close()
        imu_bytes = sum(imus[1 + W + j].nbytes for j in range(K)) / K
        from paper_2212_02988_gb300._lib import State
        import ctypes
        e2e = {"value": e2e_frames / e2e_elapsed, "unit": UNIT,
               "h2d_bytes_per_step": int(Dh[0].numel() * 4 + Ch[0].numel() * 4 + imu_bytes),
               "path": "prism_step_host: pinned host frames and IMU window in, state out, every step",
               "d2h_bytes_per_step": ctypes.sizeof(State),
               "p50_step_ms": statistics.median(lat), "p99_step_ms": float(np.percentile(lat, 99))}
        # State-uncertainty calibration (App. G) of the states read back in
        # that run, against the trajectory's true poses
        from paper_2212_02988_gb300 import calibration, state_arrays
        sa = [state_arrays(x) for x in e2e_states]
        cr = calibration.calibrate(np.array([a["pose"] for a in sa]), np.array([a["cov"] for a in sa]),
                                   np.array([seq.pose7(1 + W + j) for j in range(K)]))
        p95 = calibration.chi2_cdf(cr["nssr"] * cr["scale"], 6) <= 0.95
        calib = {"frames": K, "rms_translation_m": cr["rms_translation"],
                 "rms_rotation_deg": cr["rms_rotation_deg"], "ml_scale": cr["scale"],
                 "frac_within_chi2_95_unscaled": float(np.mean(p95)),
                 "curve_observed_at": {f"{q:.2f}": float(o) for q, o in zip(cr["levels"], cr["observed"])
                                       if round(q * 20) % 4 == 2},
                 "note": "pose residuals against the true poses whitened by the filter's pose covariance "
                         "(App. G); ml_scale > 1: the covariances are smaller than the errors, < 1: pessimistic"}

    res = {
        "metric": METRIC, "value": frames / elapsed, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 6x6 solve and state covariance)" if storage == "f32" else "bf16 map, f32 math",
        "data": "synthetic (seeded analytic scene; RGB-D frames ray-cast on the GPU, IMU from the trajectory)",
        "config": {"workload": w.name, "map": f"{w.n}^3 @ {w.voxel * 100:.2f} cm, {storage}",
                   "frames": f"{w.width}x{w.height} RGB-D at {w.rate:g} Hz, IMU {w.imu_rate:g} Hz",
                   "gauss_newton_iterations": cfg.n_gn,
                   "l2": "no flush; working set larger than L2 (map planes 6 x %.0f MB)" % (
                       (w.n + 2) ** 3 * b / 1e6),
                   "parallelism": f"replicas x{world}"},
        "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
        "render_mrays_per_s": rays_per / (render_ms * 1e-3) / 1e6,
        "render_pct_hbm_peak": 100.0 * achieved_G / peak,
        "render_full_march": {"samples_per_launch": samp_per * full_ratio,
                              "pct_hbm_peak": 100.0 * achieved_G * full_ratio / peak,
                              "note": "the march's logical gathered bytes (every sample, as without brick "
                                      "skipping) over the render's time; render_pct_hbm_peak counts only the "
                                      "samples the kernel evaluates"},
        "phase_ms_per_step": {k[:-3]: tm[k] / max(tm[k[:-3] + "_n"], 1) for k in
                              ("predict_ms", "localise_ms", "fuse_ms", "render_ms", "anchor_ms")},
        "roofline": {"kernel": "Gauss-Newton pass (k_track_coop: passes 2-10 in one cooperative launch; "
                               "k_track<GN>: pass 1)", "bound": "hbm",
                     "achieved": gn_bytes / (gn_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": gn_bytes / (gn_ms * 1e-3) / 1e9 / peak, "peak_source": peak_kind,
                     "traffic": profiled_traffic(args.workload, "k_track_gn"),
                     "algorithmic_bytes": "%d B per observed pixel (observation 16 B + anchor gathers 56 B) x %d "
                                          "pixels, per pass" % (GN_BYTES_PER_PIXEL, npx),
                     "bytes_per_pass": gn_bytes, "ms_per_pass": gn_ms, "passes_per_step": cfg.n_gn,
                     "note": "the dominant kernel by device time (10 passes a step); latency-bound: the pixel "
                             "loop over all SMs, a grid barrier, then the FP64 finish (solve, retraction) that "
                             "every block repeats; ms_per_pass = (localisation - Laplace pass) / passes, from "
                             "the library's CUDA events on its stream; traffic is per pass"},
        "roofline_render": {"kernel": "k_render", "bound": "instruction issue (ncu: issue-active, L1-resident "
                                                           "map; DRAM carries a few MB a launch)",
                            "achieved_unique": achieved_U, "achieved_gathered": achieved_G, "peak": peak,
                            "unit": "GB/s", "frac_unique": achieved_U / peak, "frac_gathered": achieved_G / peak,
                            "peak_source": peak_kind, "traffic": profiled_traffic(args.workload, "k_render"),
                            "algorithmic_bytes": "U = distinct occupancy corners per ray x %d B + hits x 8 x 3 x "
                                                 "%d B colour corners; G = evaluated samples x 8 x %d B + hits x "
                                                 "2 x 8 x 3 x %d B, per launch" % (b, b, b, b),
                            "unique_bytes_per_launch": U, "gathered_bytes_per_launch": G,
                            "samples_per_launch": samp_per, "ms_per_launch": render_ms},
        "roofline_fuse": {"kernel": "k_fuse_cull + k_fuse_list + k_brick_bounds (the map-update phase)",
                          "bound": "latency (dependent pixel, map and store round trips per tile; the listed "
                                   "tiles' occupancy read for their bounds)",
                          "achieved": fuse_bytes / (fuse_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": fuse_bytes / (fuse_ms * 1e-3) / 1e9 / peak, "peak_source": peak_kind,
                          "traffic": profiled_traffic(args.workload, "k_fuse_list"),
                          "algorithmic_bytes": "occupancy mean and variance read and written (%d B) per updated "
                                               "voxel + four colour planes read and written (%d B) per colour "
                                               "update, per step" % (4 * fb, 8 * fb),
                          "updates_per_step": fuse_upd, "colour_updates_per_step": fuse_col,
                          "bytes_per_step": fuse_bytes, "ms_per_step": fuse_ms},
        "localisation": {"ms_per_step": loc_ms, "gauss_newton_passes": cfg.n_gn, "gauss_newton_pass_ms": gn_ms,
                         "laplace_pass_ms": tm["laplace_ms"] / max(tm["laplace_n"], 1)},
        "bf16_map": bf16,
        "e2e": e2e,
        "render_adjoint": adj,
        "pose_optimiser_adam": adam,
        "rollout": roll,
        "mapping_comparison": mapping,
        "calibration": calib,
        "gpu_launches": int(d_st["kernel_launches"]),
        "clocks": clocks,
    }
    return res


# ------------------------------------------------- mapping: closed form vs descent
def mapping_comparison(dev, n_start: int = 8, n_frames: int = 8, budget_its: int = 240):
    """Closed-form map updates against gradient-descent mapping (Sec. 4.4,
    Fig. sdfvsvi) on the 128^3 / 320x240 room: both start from the map that
    closed-form updates of frames 0..n_start-1 leave (at the true poses) and
    take in frames n_start..n_start+n_frames-1; the error is the mean
    absolute difference between the map's render at those poses and the
    noise-free depth.  Device time (CUDA events around the calls)."""
    import numpy as np
    import torch

    import synth
    from paper_2212_02988_gb300 import Filter, config, make_state
    from synth.gpu_frames import raycast_frames

    w = synth.ROOM128
    seq = synth.Sequence(w, n_frames=n_start + n_frames + 1, seed=w.seed + 7)
    idx = list(range(n_start + n_frames))
    D, Cc = raycast_frames(seq, idx, dev)
    Dc, _ = raycast_frames(seq, idx, dev, noise=False)
    cfg = config(w.n, w.extent, w.width, w.height)
    F = Filter(cfg, make_state(seq.pose7(0)), device=dev.index)
    for i in range(n_start):
        F.set_state(make_state(seq.pose7(i)))
        F.update_map(D[i], Cc[i])
    start = F.map_store()
    test = list(range(n_start, n_start + n_frames))
    poses = np.stack([seq.pose7(i) for i in test])
    tD, tC = D[n_start:].contiguous(), Cc[n_start:].contiguous()

    def depth_error():
        errs = []
        for j, i in enumerate(test):
            r = F.render(poses[j])
            m = (r["mask"] > 0) & (Dc[i] > 0)
            errs.append(torch.abs(r["depth"][m] - Dc[i][m]).mean().item())
        return float(np.mean(errs))

    def reset():
        F.map_load(start["occ"], start["rgb"], start["var_occ"], start["var_rgb"])
        torch.cuda.synchronize()

    e0 = depth_error()
    # closed form: one map update a frame (the fuse, App. D)
    cf_ms = 0.0
    for j, i in enumerate(test):
        F.set_state(make_state(poses[j]))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        F.update_map(tD[j], tC[j])
        b.record()
        torch.cuda.synchronize()
        cf_ms += a.elapsed_time(b)
    e_cf = depth_error()
    # descent: plain steps over all the frames; the step size is the best of
    # a short sweep (20 steps each), then a longer run
    sd, sc = 0.02, 0.1
    best = None
    for lr in (5e-9, 1e-8, 2e-8, 5e-8, 1e-7):
        reset()
        for _ in range(20):
            loss = F.map_descent(poses, tD, tC, sd, sc, lr, 5 * lr, want_loss=False)
        loss = F.map_descent(poses, tD, tC, sd, sc, 0.0, 0.0)
        if np.isfinite(loss) and (best is None or loss < best[1]):
            best = (lr, loss)
    lr = best[0]
    reset()
    curve, ms, matched = [(0.0, e0)], 0.0, None
    marks = {1, 2, 4, 8, 16, 32, 64, 128, 240}
    for it in range(1, budget_its + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        F.map_descent(poses, tD, tC, sd, sc, lr, 5 * lr, want_loss=False)
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        if it in marks:
            e = depth_error()
            curve.append((ms, e))
            if matched is None and e <= e_cf:
                matched = ms
    F.close()
    return {"workload": w.name, "start_frames": n_start, "frames": n_frames,
            "start_depth_error_m": e0,
            "closed_form": {"ms": cf_ms, "depth_error_m": e_cf},
            "descent": {"lr_occ": lr, "lr_rgb": 5 * lr, "sd": sd, "sc": sc,
                        "curve_ms_error_m": curve, "ms_to_match_closed_form": matched,
                        "ms_per_step": ms / budget_its},
            "note": "gradient-descent mapping through the render adjoint (prism_map_descent) against the "
                    "closed-form update (prism_update_map) on the same frames and start map; depth error of "
                    "the map's renders against noise-free depth at the frames' poses"}


# ---------------------------------------------------------------- serving
def prepare_serving(duration_s: float, frames_per_cycle: int, dev, seed: int = 4000):
    """The stream mix and, per stream, its pre-rendered frame cycle in pinned
    host memory, IMU windows, first state and request arrival times."""
    import numpy as np
    import synth
    from paper_2212_02988_gb300 import config, make_state
    from synth.gpu_frames import raycast_frames
    from synth.serving import request_times, serving_plan
    plans = serving_plan(32, duration_s, seed, frames_per_cycle)
    rng = np.random.default_rng(seed + 1)
    streams = []
    for p in plans:
        w = p.workload
        seq = synth.Sequence(w)
        P = w.n_frames
        d, c = raycast_frames(seq, range(P), dev, seed=p.index)
        streams.append({"plan": p, "w": w, "D": d.cpu().pin_memory(), "C": c.cpu().pin_memory(),
                        "imus": [None] + [seq.imu_window(i) for i in range(1, P + 1)],
                        "cfg": config(w.n, w.extent, w.width, w.height),
                        "s1": make_state(seq.pose7(0), seq.velocity(0)),
                        "times": request_times(p, rng, duration_s)})
    return streams


def _frame_of(st, k):
    P = st["w"].n_frames
    imu = None if k == 0 else st["imus"][((k - 1) % P) + 1]
    return imu, st["D"][k % P], st["C"][k % P]


def _events(streams):
    ev = []
    for i, st in enumerate(streams):
        ts = st["times"]
        if len(ts) == 0:
            continue
        ev.append((ts[0], 0, i, -1))                       # open
        ev += [(t, 1, i, k) for k, t in enumerate(ts)]       # requests
        ev.append((ts[-1], 2, i, -1))                        # close after its last request
    return sorted(ev)


def _lat_stats(lat, frames, span):
    import numpy as np
    lat = np.asarray(lat)
    return {"frames": int(frames), "frames_per_s": frames / span if span > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None}


def serve_batched(streams, budget_bytes, device):
    """The arrival schedule through the multi-stream server (bf16 maps)."""
    from paper_2212_02988_gb300.serve import Server
    srv = Server(budget_bytes, max_slots=64, storage="bf16", device=device)
    ev = _events(streams)
    ids, lat, results = {}, [], []
    t0 = time.perf_counter()
    for t, kind, i, k in ev:
        while True:
            now = time.perf_counter() - t0
            if now >= t:
                break
            results += srv.poll(256, timeout_ms=0)
            time.sleep(min(2e-4, t - now))
        st = streams[i]
        if kind == 0:
            ids[i] = srv.open(st["cfg"], st["s1"])
        elif kind == 1:
            imu, d, c = _frame_of(st, k)
            srv.submit(ids[i], imu, st["w"].dt, d, c, tag=(i, k))
        else:
            srv.close(ids[i])
    srv.drain(600000)
    results += srv.poll(1 << 16, timeout_ms=0)
    stats = srv.stats()
    srv.destroy()
    lat = [r["latency_ms"] for r in results]
    span = max(r["done_s"] for r in results) - min(r["submit_s"] for r in results)
    out = _lat_stats(lat, len(results), span)
    out.update({"batches": stats["batches"], "mean_batch": len(results) / max(stats["batches"], 1),
                "max_batch": stats["max_batch"], "bytes_peak": stats["bytes_peak"], "budget": stats["budget"],
                "kernel_launches": stats["kernel_launches"], "graph_launches": stats["graph_launches"],
                "not_pd_steps": sum(1 for r in results if r["status"] != 0)})
    return out


def serve_plain(streams, device):
    """The same schedule served one request at a time, in arrival order, by
    one single-stream f32 filter per stream (host copy in, state out)."""
    import torch
    from paper_2212_02988_gb300 import Filter
    ev = _events(streams)
    F, bufs, lat = {}, {}, []
    t0 = time.perf_counter()
    t_first = t_last = None
    for t, kind, i, k in ev:
        now = time.perf_counter() - t0
        if now < t:
            time.sleep(t - now)
        st = streams[i]
        if kind == 0:
            F[i] = Filter(st["cfg"], st["s1"], device=device)
            bufs[i] = (torch.empty_like(st["D"][0], device="cuda"), torch.empty_like(st["C"][0], device="cuda"))
        elif kind == 1:
            imu, d, c = _frame_of(st, k)
            db, cb = bufs[i]
            db.copy_(d, non_blocking=True)
            cb.copy_(c, non_blocking=True)
            F[i].step(imu, st["w"].dt, db, cb, want_state=True)
            done = time.perf_counter() - t0
            lat.append(1e3 * (done - t))
            t_first = t if t_first is None else t_first
            t_last = done
        else:
            F.pop(i).close()
            bufs.pop(i)
    for f in F.values():
        f.close()
    return _lat_stats(lat, len(lat), (t_last or 0) - (t_first or 0))


def serve_saturation(streams, seconds, budget_bytes, device):
    """Closed loop over the first 32 streams (no churn): frames/s when every
    stream always has two requests waiting (server) or when the streams are
    stepped round-robin as fast as possible (plain f32 filters)."""
    import torch
    from paper_2212_02988_gb300 import Filter
    from paper_2212_02988_gb300.serve import Server
    pool = streams[:32]
    srv = Server(budget_bytes, max_slots=64, storage="bf16", device=device)
    ids = [srv.open(st["cfg"], st["s1"]) for st in pool]
    nxt = [0] * len(pool)
    sid_to = {sid: j for j, sid in enumerate(ids)}

    def sub(j):
        imu, d, c = _frame_of(pool[j], nxt[j])
        srv.submit(ids[j], imu, pool[j]["w"].dt, d, c)
        nxt[j] += 1

    for j in range(len(pool)):
        sub(j)
        sub(j)
    for _ in range(3):                      # warm-up: let every stream finish its first steps
        for r in srv.poll(512, timeout_ms=2000):
            sub(sid_to[r["stream"]])
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for r in srv.poll(512, timeout_ms=50):
            done += 1
            sub(sid_to[r["stream"]])
    el = time.perf_counter() - t0
    st = srv.stats()
    srv.destroy()
    batched = {"frames_per_s": done / el, "mean_batch": None if not st["batches"] else st["frames"] / st["batches"]}
    filters = [Filter(st_["cfg"], st_["s1"], device=device) for st_ in pool]
    bufs = [(torch.empty_like(st_["D"][0], device="cuda"), torch.empty_like(st_["C"][0], device="cuda"))
            for st_ in pool]
    k = [0] * len(pool)

    def step(j):
        imu, d, c = _frame_of(pool[j], k[j])
        bufs[j][0].copy_(d, non_blocking=True)
        bufs[j][1].copy_(c, non_blocking=True)
        filters[j].step(imu, pool[j]["w"].dt, bufs[j][0], bufs[j][1], want_state=True)
        k[j] += 1

    for j in range(len(pool)):
        step(j)
        step(j)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        step(n % len(pool))
        n += 1
    el = time.perf_counter() - t0
    for f in filters:
        f.close()
    return {"batched_bf16": batched, "plain_f32": {"frames_per_s": n / el}, "streams": len(pool),
            "seconds": seconds}


def run_serving(args, local_rank, seconds, frames_per_cycle):
    import torch
    dev = torch.device("cuda", local_rank)
    t_prep = time.perf_counter()
    streams = prepare_serving(seconds, frames_per_cycle, dev)
    prep_s = time.perf_counter() - t_prep
    budget = int(args.serve_budget_gb * (1 << 30))
    sizes = {}
    for st in streams:
        key = f"{st['w'].n}^3/{st['w'].width}x{st['w'].height}"
        sizes[key] = sizes.get(key, 0) + 1
    batched = serve_batched(streams, budget, local_rank)
    plain = serve_plain(streams, local_rank)
    sat = serve_saturation(streams, min(8.0, max(3.0, seconds / 4)), budget, local_rank)
    return {"workload": "32 concurrent streams, maps {64,128,256}^3, frames {160x120,320x240,640x480}, "
                        "10-30 Hz Poisson arrivals, streams arriving and retiring",
            "seconds": seconds, "streams_total": len(streams), "requests": int(sum(len(s["times"]) for s in streams)),
            "stream_mix": sizes, "frames_per_cycle": frames_per_cycle, "prepare_s": prep_s,
            "batched_bf16": batched, "plain_f32": plain, "saturation": sat}


def cpu_baseline(args):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    full filter steps of the same configuration on the host, with every
    host core (the oracle's threaded loops), and the same steps on one
    thread."""
    import synth
    from oracle import oracle as O
    w = synth.PRESETS[args.workload]
    n = max(1, args.cpu_sample_steps)
    n1 = max(1, min(n, args.cpu_single_steps))
    seq = synth.Sequence(w, n_frames=n + 2)
    p = O.params(w)
    frames = [seq.frame(i) for i in range(n + 1)]
    cores = O.threads()

    def run(steps, threads):
        O.set_threads(threads)
        try:
            F = O.Filter(p, seq.settled_map(), O.make_state(seq.pose7(0), seq.velocity(0)))
            F.step(frames[0]["depth"], frames[0]["rgb"])
            t0 = time.perf_counter()
            for i in range(1, steps + 1):
                F.step(frames[i]["depth"], frames[i]["rgb"], seq.imu_window(i), w.dt)
            return steps / (time.perf_counter() - t0)
        finally:
            O.set_threads(0)

    v = run(n, cores)
    v1 = run(n1, 1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} full filter steps (frames 1-{n}) of {w.name}, FP64 C oracle on {cores} threads",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} full filter steps (frames 1-{n1}), one thread"}}


def run_reference(args, rank):
    """Reference arm: the oracle timed on the host cores (all of them, the
    oracle's threaded loops), on our config and metric."""
    import synth
    from oracle import oracle as O
    w = synth.PRESETS[args.workload]
    cores = O.threads()
    K, W = args.steps, max(args.warmup, 0)
    seq = synth.Sequence(w, n_frames=min(1 + W + K, w.n_frames))
    p = O.params(w)
    F = O.Filter(p, seq.settled_map(), O.make_state(seq.pose7(0), seq.velocity(0)))
    f0 = seq.frame(0)
    F.step(f0["depth"], f0["rgb"])
    # warm-up: one step (the oracle has no caches to warm beyond the first)
    t_w = time.perf_counter()
    for i in range(1, 1 + min(W, 1)):
        f = seq.frame(i)
        F.step(f["depth"], f["rgb"], seq.imu_window(i), w.dt)
    per_step = time.perf_counter() - t_w if W else 5.0
    n_run = max(1, min(K, int(args.reference_budget_s / max(per_step, 1e-3))))
    frames = [seq.frame(i) for i in range(2, 2 + n_run)]
    t0 = time.perf_counter()
    for j, f in enumerate(frames):
        F.step(f["depth"], f["rgb"], seq.imu_window(2 + j), w.dt)
    el = time.perf_counter() - t0
    v = n_run / el
    sample = (f"{n_run} of {K} requested full filter steps of {w.name} (frames 2-{1 + n_run}), "
              f"FP64 C oracle on {cores} threads, time-bounded at {args.reference_budget_s:.0f} s")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": n_run,
            "warmup": min(W, 1), "ms_per_step": 1e3 * el / n_run, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name}, "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                                              "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank)))
        return 0
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.serve:
        if rank == 0:
            secs = args.serve_seconds if args.serve_seconds is not None else 120.0
            torch.cuda.set_device(local_rank)
            srv = run_serving(args, local_rank, secs, 32)
            b = srv["batched_bf16"]
            line = {"metric": "serving: p50/p99 step latency and aggregate frames/s, 32 concurrent streams",
                    "value": b["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": b["frames"],
                    "warmup": 0, "ms_per_step": b["p50_ms"], "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "bf16 map, f32 math", "data": "synthetic",
                    "config": {"workload": "serving_32_streams"}, "serving": srv}
            print(json.dumps(line))
        return 0
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args)
        else:
            res["cpu_baseline"] = None
        if world == 1 and not args.no_serve:
            secs = args.serve_seconds if args.serve_seconds is not None else 12.0
            res["serving"] = run_serving(args, local_rank, secs, 16)
        print(json.dumps(res))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
