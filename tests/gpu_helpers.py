"""Shared set-up for the GPU parity tests: a CUDA filter and the oracle's
parameters for the same workload, and host/device conversions."""
import numpy as np
import torch

import synth


def dev():
    return torch.device("cuda", 0)


def t(a, dtype=None):
    a = np.ascontiguousarray(a)
    x = torch.from_numpy(a)
    if dtype is not None:
        x = x.to(dtype)
    return x.to(dev())


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest-even) and back, on the host."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def make_pair(w, O, storage="f32", map_arrays=None, s1_pose=None, vel=None, **over):
    """(CUDA Filter, oracle params) for workload w, with the map loaded."""
    from paper_2212_02988_gb300 import Filter, config, make_state
    cfg = config(w.n, w.extent, w.width, w.height, storage=storage, **over)
    s = None
    if s1_pose is not None:
        s = make_state(s1_pose, vel)
    F = Filter(cfg, s, device=0)
    if map_arrays is not None:
        F.map_load(*(t(np.asarray(a, dtype=np.float32)) for a in map_arrays))
    p = O.params(w, **{k: v for k, v in over.items() if k in ("n_gn", "max_depth")})
    return F, p


def quat_angle_deg(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return np.degrees(2 * np.arccos(min(1.0, d)))
