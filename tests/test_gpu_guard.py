"""The divergence guard on the GPU: a step whose prior pose covariance is not
positive definite is rejected.  The state (pose, velocities, covariance,
localisation count) and the map stay bit for bit as they were, the call
reports PRISM_ENOTPD, and the filter takes later steps (rejecting them while
the state stays indefinite, accepting them once a valid state is set).  The
server rejects such a step of one stream the same way and carries on with
every stream.  The indefinite covariance is made on the host: no GPU fault
is involved."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import make_pair, t
from test_gpu_serve import run_filter, run_server, same_state, stream_spec

pytestmark = pytest.mark.gpu

ENOTPD = -4


def indefinite_cov():
    """A 12x12 error-state covariance with a negative translation variance:
    after one prediction (dt = 0.1 s, the paper's sigma_pose and sigma_vel)
    the prior's (0, 0) entry stays about -0.0075."""
    cov = np.diag([1e-4] * 3 + [1e-5] * 3 + [1e-3] * 6)
    cov[0, 0] = -1e-2
    return cov


def raw_state(F):
    """prism_get_state through the C ABI: (status, state arrays)."""
    from paper_2212_02988_gb300 import state_arrays
    from paper_2212_02988_gb300._lib import State
    s = State()
    st = F.L.prism_get_state(F.h, C.byref(s))
    return st, state_arrays(s)


def raw_step(F, imu, dt, d, c):
    from paper_2212_02988_gb300 import state_arrays
    from paper_2212_02988_gb300._lib import State
    s = State()
    imu = np.ascontiguousarray(imu, dtype=np.float64)
    st = F.L.prism_step(F.h, imu.ctypes.data_as(C.POINTER(C.c_double)), len(imu), dt,
                        C.c_void_p(d.data_ptr()), C.c_void_p(c.data_ptr()), C.byref(s))
    return st, state_arrays(s)


def maps_equal(a, b):
    return all(torch.equal(a[k], b[k]) for k in ("occ", "rgb", "var_occ", "var_rgb"))


def test_rejected_step_leaves_state_and_map(oracle_mod):
    from paper_2212_02988_gb300 import PrismError, make_state, state_arrays
    w = synth.ROOM64
    s = synth.Sequence(w)
    F, _ = make_pair(w, oracle_mod, map_arrays=s.settled_map(), s1_pose=s.pose7(0), vel=s.velocity(0))
    frames = [s.frame(i) for i in range(6)]
    dev = [(t(f["depth"]), t(f["rgb"])) for f in frames]
    F.step(None, w.dt, *dev[0])
    good = state_arrays(F.step(s.imu_window(1), w.dt, *dev[1], want_state=True))
    assert good["n_localised"] == 1
    # an indefinite covariance, set on the host
    F.set_state(make_state(good["pose"], good["vel"], indefinite_cov(), n_localised=good["n_localised"]))
    st0, before = raw_state(F)
    assert st0 == 0
    map0 = F.map_store()
    for i in (2, 3):
        st, out = raw_step(F, s.imu_window(i), w.dt, *dev[i])
        assert st == ENOTPD
        assert b"rejected" in F.L.prism_last_error(F.h)
        for k in ("pose", "vel", "cov"):
            assert np.array_equal(out[k], before[k]), k
        assert out["n_localised"] == before["n_localised"]
        st1, after = raw_state(F)
        assert st1 == ENOTPD                        # the flags of the latest step, until the next prediction
        for k in ("pose", "vel", "cov"):
            assert np.array_equal(after[k], before[k]), k
        assert maps_equal(F.map_store(), map0)      # the rejected frame was not fused
    with pytest.raises(PrismError) as e:
        F.step(s.imu_window(4), w.dt, *dev[4], want_state=True)
    assert e.value.status == ENOTPD
    # a valid state again: the next step is accepted, and fuses its frame
    F.set_state(make_state(good["pose"], good["vel"], np.diag([1e-6] * 3 + [1e-7] * 3 + [1e-4] * 6),
                           n_localised=good["n_localised"]))
    ok = state_arrays(F.step(s.imu_window(5), w.dt, *dev[5], want_state=True))
    assert ok["n_localised"] == good["n_localised"] + 1
    assert np.all(np.linalg.eigvalsh(ok["cov"]) > 0)
    assert not maps_equal(F.map_store(), map0)
    F.close()


def test_server_rejects_one_stream_and_serves_the_others():
    from paper_2212_02988_gb300 import make_state
    good = stream_spec(synth.ROOM64, 21, 4)
    bad = stream_spec(synth.ROOM64, 22, 4)
    s0 = bad["seq"]
    bad["s1"] = make_state(s0.pose7(0), s0.velocity(0), indefinite_cov())
    (res_good, res_bad), (map_good, map_bad), _ = run_server([good, bad], "f32")
    ref_good, ref_map_good = run_filter(good, "f32")
    for r, q in zip(res_good, ref_good):
        assert r["status"] == 0 and same_state(r, q)
    assert maps_equal(map_good, ref_map_good)
    # the indefinite stream: its first step (fuse and render, no localisation) is
    # accepted; every later step is rejected and leaves its state and map as they were
    ref_first, ref_map_first = run_filter({**bad, "frames": bad["frames"][:1]}, "f32")
    assert res_bad[0]["status"] == 0 and same_state(res_bad[0], ref_first[0])
    assert len(res_bad) == 4
    for r in res_bad[1:]:
        assert r["status"] == ENOTPD
        assert same_state(r, res_bad[0])
    assert maps_equal(map_bad, ref_map_first)
