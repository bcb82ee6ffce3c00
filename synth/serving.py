"""Seeded stream mix of the serving workload: many concurrent camera/IMU
streams on one GPU, each with its own seeded scene, arriving and retiring
over the run.

Per stream: a map of 64^3 (4 m cube, 6.25 cm), 128^3 or 256^3 (6.4 m cube,
5 / 2.5 cm) voxels and frames of 160x120, 320x240 or 640x480, each drawn
uniformly; a frame rate uniform in [10, 30] Hz; requests arrive as a
Poisson process of that rate (the frames themselves are taken every 1/rate
s of sensor time); a lifetime uniform in [0.25, 0.75] of the run.  The
initial population opens within the first second; every retirement is
followed, after an exponential delay of mean 0.5 s, by a new stream, so the
number of concurrent streams stays near the initial one.

A stream's trajectory is periodic over `frames_per_cycle` frames (the
motion repeats exactly), so a bounded set of pre-rendered frames and IMU
windows serves any number of steps: step k uses frame k mod P and, for
k >= 1, the IMU window ending at frame ((k - 1) mod P) + 1 (window P ends
where frame 0's content is seen again)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .configs import Workload

MAPS = ((64, 4.0), (128, 6.4), (256, 6.4))
FRAMES = ((160, 120), (320, 240), (640, 480))


@dataclass(frozen=True)
class StreamPlan:
    index: int
    workload: Workload
    arrival_s: float
    lifetime_s: float


def stream_workload(k: int, rng: np.random.Generator, frames_per_cycle: int) -> Workload:
    n, ext = MAPS[int(rng.integers(len(MAPS)))]
    W, H = FRAMES[int(rng.integers(len(FRAMES)))]
    rate = float(rng.uniform(10.0, 30.0))
    n_prims = int(rng.integers(12, 41))
    return Workload(f"stream{k}_{n}^3_{W}x{H}", n, ext, W, H, frames_per_cycle, rate, 200.0, 1.5, 120.0,
                    False, n_prims, True, storage="bf16", seed=5000 + k, periodic=True)


def serving_plan(n_concurrent: int = 32, duration_s: float = 120.0, seed: int = 4000,
                 frames_per_cycle: int = 32) -> list[StreamPlan]:
    rng = np.random.default_rng(seed)
    plans = []

    def new(t0: float) -> StreamPlan:
        k = len(plans)
        w = stream_workload(k, rng, frames_per_cycle)
        p = StreamPlan(k, w, t0, float(rng.uniform(0.25, 0.75)) * duration_s)
        plans.append(p)
        return p

    for _ in range(n_concurrent):
        new(float(rng.uniform(0.0, 1.0)))
    i = 0
    while i < len(plans):
        end = plans[i].arrival_s + plans[i].lifetime_s
        if end < duration_s:
            new(end + float(rng.exponential(0.5)))
        i += 1
    return sorted(plans, key=lambda p: p.arrival_s)


def request_times(plan: StreamPlan, rng: np.random.Generator, duration_s: float) -> np.ndarray:
    """Arrival times of the stream's requests (Poisson process at its frame
    rate), inside its lifetime and the run."""
    end = min(plan.arrival_s + plan.lifetime_s, duration_s)
    t, out = plan.arrival_s, []
    while t < end:
        out.append(t)
        t += float(rng.exponential(1.0 / plan.workload.rate))
    return np.array(out)
