"""The oracle's threaded loops give bit-identical results for any thread
count: rays, pixels and voxels write only their own outputs, and the
normal-equation sums are formed per fixed chunk of pixels and added in chunk
order.  Compared here: 1 thread against 5 (uneven ranges) and 8."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def case():
    w = synth.ROOM64
    s = synth.Sequence(w)
    return w, s, s.settled_map()


def with_threads(O, n, fn):
    old = O.threads()
    O.set_threads(n)
    try:
        return fn()
    finally:
        O.set_threads(old)


@pytest.mark.parametrize("n", [5, 8])
def test_render_and_residuals_do_not_depend_on_threads(oracle_mod, case, n):
    O = oracle_mod
    w, s, (occ, rgb, vo, vr) = case
    p = O.params(w)
    pose = s.pose7(4)
    a = with_threads(O, 1, lambda: O.render(p, occ, rgb, pose))
    b = with_threads(O, n, lambda: O.render(p, occ, rgb, pose))
    assert a["n_samples"] == b["n_samples"] > 0
    for k in ("depth", "rgb", "mask", "hitk"):
        assert np.array_equal(a[k], b[k]), k
    A = s.pose7(3)
    ad, ac = (x.astype(np.float32) for x in s.clean_frame(3))
    f = s.frame(4)
    ra = with_threads(O, 1, lambda: O.residuals(p, A, ad, ac, f["pose"], f["depth"], f["rgb"]))
    rb = with_threads(O, n, lambda: O.residuals(p, A, ad, ac, f["pose"], f["depth"], f["rgb"]))
    for k in ("r", "J", "assoc", "kept"):
        assert np.array_equal(ra[k], rb[k]), k
    na = with_threads(O, 1, lambda: O.normal_equations(p, A, ad, ac, f["pose"], f["depth"], f["rgb"]))
    nb = with_threads(O, n, lambda: O.normal_equations(p, A, ad, ac, f["pose"], f["depth"], f["rgb"]))
    for k in ("H", "g", "Ht"):
        assert np.array_equal(na[k], nb[k]), k
    assert na["cost"] == nb["cost"] and na["count"] == nb["count"]


def test_filter_steps_do_not_depend_on_threads(oracle_mod, case):
    O = oracle_mod
    w, s, m = case

    def run():
        F = O.Filter(O.params(w), m, O.make_state(s.pose7(0), s.velocity(0)))
        out = []
        for i in range(4):
            f = s.frame(i)
            st = F.step(f["depth"], f["rgb"], s.imu_window(i) if i else None, w.dt)
            out.append(O.state_arrays(st))
        return out, F.m, F.n_upd

    a, ma, ua = with_threads(O, 1, run)
    b, mb, ub = with_threads(O, 7, run)
    assert ua == ub > 0
    for x, y in zip(a, b):
        for k in ("pose", "vel", "cov"):
            assert np.array_equal(x[k], y[k]), k
    for k in ("occ", "rgb", "var_occ", "var_rgb"):
        assert np.array_equal(ma[k], mb[k]), k
