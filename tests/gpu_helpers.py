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
    p = O.params(w, **{k: v for k, v in over.items()
                       if k in ("n_gn", "max_depth", "optimiser") or k.startswith("adam_")})
    return F, p


def quat_angle_deg(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return np.degrees(2 * np.arccos(min(1.0, d)))


def world_frame_scale(H, anchor_pose7):
    """Error scale of a world-frame 6x6 sum H = T H' T^T, T = diag(Ra, Ra),
    whose camera-frame terms H' the kernels add in FP32 (App. E.3): each H'_kl
    is off by at most a multiple of eps32 * sqrt(H'_kk H'_ll) (Cauchy-Schwarz
    over the pixels), so H_ij is off by at most that multiple of
    sigma_i sigma_j with sigma_i = sum_k |T_ik| sqrt(H'_kk) (>= sqrt(H_ii)).
    Returns the matrix sigma sigma^T."""
    from scipy.spatial.transform import Rotation
    w, x, y, z = anchor_pose7[3:]
    Ra = Rotation.from_quat([x, y, z, w]).as_matrix()
    T = np.zeros((6, 6))
    T[:3, :3] = Ra
    T[3:, 3:] = Ra
    Hc = T.T @ H @ T
    sigma = np.abs(T) @ np.sqrt(np.clip(np.diag(Hc), 0.0, None))
    return np.outer(sigma, sigma)


# Render bar: hit indices bit-exact, depth and colour within 1e-5 relative.
RTOL = 1e-5


def check_render(out, ref, atol_rgb=1e-6):
    """GPU render outputs (tensors; mask optional) against an oracle render."""
    hk = out["hitk"].cpu().numpy().reshape(ref["hitk"].shape)
    assert np.array_equal(hk, ref["hitk"]), f"{np.sum(hk != ref['hitk'])} hit indices differ"
    if out.get("mask") is not None:
        mask = out["mask"].cpu().numpy().reshape(ref["mask"].shape)
        assert np.array_equal(mask, ref["mask"])
    d = out["depth"].cpu().numpy().reshape(ref["depth"].shape)
    m = ref["mask"] > 0
    assert np.all(d[~m] == 0)
    err = np.abs(d[m] - ref["depth"][m])
    assert np.all(err <= RTOL * ref["depth"][m]), err.max()
    c = out["rgb"].cpu().numpy().reshape(ref["rgb"].shape)
    np.testing.assert_allclose(c[m], ref["rgb"][m], rtol=RTOL, atol=atol_rgb)
