"""GPU parity of gradient-descent mapping (prism_map_descent; Sec. 4.4, Fig.
sdfvsvi) with the FP64 oracle, through the C ABI.

Bars.  Both sides render the same FP32 map, so every hit decision is the
same; the loss within 1e-3 relative; the change of every map mean within
1e-4 of the largest change plus 5e-3 of its own size (the gradient's FP32
residuals, render values and adjoint atomics against FP64: the render
adjoint's own bar, widened by the depth residuals' relative FP32 error)
plus two FP32 units of the mean."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import bf16_round, make_pair, t

pytestmark = pytest.mark.gpu

SD, SC = 0.02, 0.1


def problem(s, w, frames=(5, 10, 15), shift=0.03):
    """The settled map with every surface moved by `shift` (occupancy is the
    negated truncated distance, so a constant offset moves the surfaces
    along their normals), and noisy frames at true poses."""
    occ, rgb, vo, vr = s.settled_map()
    occ = (occ - np.float32(shift)).astype(np.float32)
    rgb = np.clip(rgb + np.float32(0.05), 0, 1).astype(np.float32)
    fr = [s.frame(i) for i in frames]
    poses = np.stack([s.pose7(i) for i in frames])
    return (occ, rgb, vo, vr), poses, np.stack([f["depth"] for f in fr]), np.stack([f["rgb"] for f in fr])


def check_change(got_new, start, ref_new, name):
    d_got = got_new.astype(np.float64) - start.astype(np.float64)
    d_ref = ref_new - start.astype(np.float64)
    ulp = np.spacing(np.abs(start).astype(np.float32)).astype(np.float64)
    bar = 1e-4 * np.abs(d_ref).max() + 5e-3 * np.abs(d_ref) + 2 * ulp
    err = np.abs(d_got - d_ref)
    assert np.all(err <= bar), (name, float((err / bar).max()), int(np.sum(err > bar)))


def test_descent_step_matches_oracle(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    m, poses, D, Cc = problem(s, w)
    F, p = make_pair(w, O, map_arrays=m)
    lr_occ, lr_rgb = 2e-6, 1e-5
    loss = F.map_descent(poses, t(D), t(Cc), SD, SC, lr_occ, lr_rgb)
    got = {k: v.cpu().numpy() for k, v in F.map_store().items()}
    occ_r, rgb_r, loss_r = O.map_descent(p, m[0], m[1], list(poses), list(D), list(Cc), SD, SC, lr_occ, lr_rgb)
    assert abs(loss - loss_r) <= 1e-3 * loss_r
    check_change(got["occ"], m[0], occ_r, "occ")
    check_change(got["rgb"], m[1], rgb_r, "rgb")
    assert np.abs(occ_r - m[0]).max() > 1e-4   # the step moved the map
    # variances untouched
    assert np.array_equal(got["var_occ"], m[2]) and np.array_equal(got["var_rgb"], m[3])
    F.close()


def test_zero_step_keeps_the_map_and_reports_the_loss(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    m, poses, D, Cc = problem(s, w, frames=(3, 20))
    for storage in ("f32", "bf16"):
        F, p = make_pair(w, O, storage=storage, map_arrays=m)
        before = F.map_store()
        loss = F.map_descent(poses, t(D), t(Cc), SD, SC, 0.0, 0.0)
        after = F.map_store()
        for k in ("occ", "rgb"):
            assert torch.equal(before[k], after[k])
        occ, rgb = (bf16_round(m[0]), bf16_round(m[1])) if storage == "bf16" else (m[0], m[1])
        ref = O.map_loss_grad(p, occ, rgb, list(poses), list(D), list(Cc), SD, SC)[0]
        assert abs(loss - ref) <= 1e-3 * ref
        F.close()


def test_descent_reduces_the_loss(oracle_mod):
    w = synth.ROOM64
    s = synth.Sequence(w)
    m, poses, D, Cc = problem(s, w, frames=(4, 8, 12, 16))
    F, _ = make_pair(w, oracle_mod, map_arrays=m)
    dD, dC = t(D), t(Cc)
    losses = [F.map_descent(poses, dD, dC, SD, SC, 2e-6, 1e-5) for _ in range(12)]
    assert losses[-1] < 0.7 * losses[0]
    assert all(np.isfinite(losses))
    F.close()


def test_descent_rejects_bad_arguments(oracle_mod):
    from paper_2212_02988_gb300 import _lib
    w = synth.ROOM64
    s = synth.Sequence(w)
    _, poses, D, Cc = problem(s, w, frames=(3,))
    F, _ = make_pair(w, oracle_mod)
    L = F.L
    dD, dC = t(D), t(Cc)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    pv = lambda x: C.c_void_p(x.data_ptr())
    good = np.ascontiguousarray(poses, dtype=np.float64)
    assert L.prism_map_descent(F.h, 1, dp(good), pv(dD), pv(dC), SD, SC, 0.0, 0.0, None) == _lib.OK
    bad_pose = good.copy()
    bad_pose[0, 2] = np.nan
    zero_q = good.copy()
    zero_q[0, 3:] = 0
    cases = [(0, good, SD, SC, 0.0), (1, bad_pose, SD, SC, 0.0), (1, zero_q, SD, SC, 0.0),
             (1, good, 0.0, SC, 0.0), (1, good, SD, -1.0, 0.0), (1, good, SD, SC, -1e-3),
             (1, good, SD, SC, np.inf)]
    for n, ps, sd, sc, lr in cases:
        assert L.prism_map_descent(F.h, n, dp(ps), pv(dD), pv(dC), sd, sc, lr, 0.0, None) == _lib.EINVAL
    assert L.prism_map_descent(F.h, 1, dp(good), None, pv(dC), SD, SC, 0.0, 0.0, None) == _lib.EINVAL
    F.close()
