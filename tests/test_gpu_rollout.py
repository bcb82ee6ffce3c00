"""GPU parity of the predictive rollouts (prism_rollout; App. I) with the FP64
oracle, through the C ABI.

Bars.  States: the chained FP64 transition (App. E.1/E.2) runs the same
operations on both sides up to the order of a few sums, so the prediction
step's bar holds per frame, widened for the chain: positions and
velocities 1e-11, quaternion components 1e-12, covariance 1e-9 relative.
Images: against the oracle's render at the device's own predicted pose
(both sides normalise it in IEEE FP64 in the same order and round its
matrices by the same recipe, so every traversal decision is the same): hit
indices bit-exact, depth and colour 1e-5 relative."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import bf16_round, check_render, make_pair, t

pytestmark = pytest.mark.gpu


def candidates(s, start, n_seq, k, seed=0):
    """Candidate control sequences: the sequence's own IMU windows after
    frame `start` (candidate 0), the same with a constant offset on the
    specific force and the angular rate (candidates 1 ..), and, last, no
    controls at all (constant velocity)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_seq):
        if c == n_seq - 1 and n_seq > 1:
            out.append([None] * k)
            continue
        da, dg = (np.zeros(3), np.zeros(3)) if c == 0 else (rng.normal(0, 0.5, 3), rng.normal(0, 0.2, 3))
        seq = []
        for i in range(k):
            imu = s.imu_window(start + 1 + i).copy()
            imu[:, 1:4] += da
            imu[:, 4:7] += dg
            seq.append(imu)
        out.append(seq)
    return out


def start_state(s, i):
    cov = np.diag([4e-4, 4e-4, 4e-4, 1e-4, 1e-4, 1e-4, 2e-3, 2e-3, 2e-3, 3e-3, 3e-3, 3e-3])
    vel = s.velocity(i) + np.array([0.05, -0.02, 0.01, 0.1, -0.2, 0.05])
    return s.pose7(i), vel, cov


def check_states(got, ref):
    from paper_2212_02988_gb300 import state_arrays
    g = state_arrays(got)
    np.testing.assert_allclose(g["pose"][:3], ref["pose"][:3], rtol=0, atol=1e-11)
    # quaternions component by component (an arccos of their dot product
    # cannot resolve angles below ~1e-6 degrees); 1e-12 is ~1e-10 degrees
    q = g["pose"][3:] * np.sign(np.dot(g["pose"][3:], ref["pose"][3:]))
    np.testing.assert_allclose(q, ref["pose"][3:], rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["vel"], ref["vel"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(g["cov"], ref["cov"], rtol=1e-9, atol=1e-16)
    assert g["n_localised"] == ref["n_localised"]
    return g


def frame_out(out, si, i):
    return {key: out[key][si, i] for key in ("depth", "rgb", "hitk") if key in out}


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_rollout_states_and_images_match_oracle(oracle_mod, storage):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state
    m = s.settled_map()
    occ, rgb = (bf16_round(m[0]), bf16_round(m[1])) if storage == "bf16" else (m[0], m[1])
    F, p = make_pair(w, O, storage=storage, map_arrays=m)
    pose, vel, cov = start_state(s, 6)
    F.set_state(make_state(pose, vel, cov, n_localised=3))
    n_seq, k = 4, 5
    wins = candidates(s, 6, n_seq, k)
    out = F.rollout(wins, w.dt, hitk=True)
    from paper_2212_02988_gb300 import state_arrays
    for si in range(n_seq):
        ref, _ = O.rollout(p, O.make_state(pose, vel, cov, 3), wins[si], [w.dt] * k)
        for i in range(k):
            g = check_states(out["states"][si][i], ref[i])
            check_render(frame_out(out, si, i), O.render(p, occ, rgb, g["pose"]))
    F.close()


def test_rollout_ragged_frames_and_intervals(oracle_mod):
    """An 83x61 frame (ragged against the 16x8 render tiles), one sequence
    with frame intervals of its own, windows of 1 and 0 samples."""
    O = oracle_mod
    w = synth.tiny(n=24, width=83, height=61)
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state
    m = s.settled_map()
    F, p = make_pair(w, O, map_arrays=m)
    pose, vel, cov = start_state(s, 2)
    F.set_state(make_state(pose, vel, cov))
    k = 4
    seq = [s.imu_window(3)[:1], None, s.imu_window(4), s.imu_window(5)[:3]]
    dts = np.array([[0.05, 0.1, 0.02, 0.2]])
    out = F.rollout([seq], dts, hitk=True)
    ref, _ = O.rollout(p, O.make_state(pose, vel, cov), seq, list(dts[0]))
    for i in range(k):
        g = check_states(out["states"][0][i], ref[i])
        check_render(frame_out(out, 0, i), O.render(p, m[0], m[1], g["pose"]))
    F.close()


def test_rollout_leaves_the_filter_untouched(oracle_mod):
    """A filter that rolls out between its prediction and its localisation
    ends bit-for-bit where a twin that never rolled out does."""
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state, state_arrays
    m = s.settled_map()
    twins = [make_pair(w, O, map_arrays=m)[0] for _ in range(2)]
    f6, f7 = s.frame(6), s.frame(7)
    for F in twins:
        F.set_state(make_state(s.pose7(6), s.velocity(6)))
        F.render()   # anchor at the state mean
        F.predict(s.imu_window(7), w.dt)
    before = state_arrays(twins[0].get_state())
    twins[0].rollout(candidates(s, 7, 3, 6), w.dt, hitk=True)
    after = state_arrays(twins[0].get_state())
    for key in ("pose", "vel", "cov"):
        assert np.array_equal(before[key], after[key])
    res = [state_arrays(F.localise(t(f7["depth"]), t(f7["rgb"]))) for F in twins]
    for key in ("pose", "vel", "cov"):
        assert np.array_equal(res[0][key], res[1][key])
    a0 = twins[0].render()
    a1 = twins[1].render()
    assert torch.equal(a0["hitk"], a1["hitk"]) and torch.equal(a0["depth"], a1["depth"])
    for F in twins:
        F.close()


def test_rollout_outputs_are_optional(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state, state_arrays
    F, p = make_pair(w, O, map_arrays=s.settled_map())
    pose, vel, cov = start_state(s, 4)
    F.set_state(make_state(pose, vel, cov))
    wins = candidates(s, 4, 2, 3)
    r_states = F.rollout(wins, w.dt, images=False)
    assert "depth" not in r_states and r_states["states"] is not None
    r_none = F.rollout(wins, w.dt, images=False, want_states=False)
    assert r_none["states"] is None
    r_img = F.rollout(wins, w.dt, want_states=False)
    r_all = F.rollout(wins, w.dt)
    torch.cuda.synchronize()
    assert torch.equal(r_img["depth"], r_all["depth"]) and torch.equal(r_img["rgb"], r_all["rgb"])
    for si in range(2):
        for i in range(3):
            a = state_arrays(r_states["states"][si][i])
            b = state_arrays(r_all["states"][si][i])
            for key in ("pose", "vel", "cov"):
                assert np.array_equal(a[key], b[key])
    F.close()


def test_rollout_rejects_bad_arguments(oracle_mod):
    from paper_2212_02988_gb300 import _lib
    O = oracle_mod
    w = synth.ROOM64
    F, _ = make_pair(w, O)
    L = F.L
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    imu = np.zeros((4, 7))
    imu[:, 0] = np.arange(4) * 0.01
    cnt, dts = np.array([2, 2], np.int32), np.array([0.1, 0.1])
    assert L.prism_rollout(F.h, 1, 2, dp(imu), ip(cnt), dp(dts), None, None, None, None) == _lib.OK
    bad = [
        (0, 2, dp(imu), ip(cnt), dp(dts)),
        (1, 0, dp(imu), ip(cnt), dp(dts)),
        (300, 300, dp(imu), ip(cnt), dp(dts)),
        (1, 2, None, ip(cnt), dp(dts)),
        (1, 2, dp(imu), None, dp(dts)),
        (1, 2, dp(imu), ip(np.array([2, -1], np.int32)), dp(dts)),
        (1, 2, dp(imu), ip(cnt), dp(np.array([0.1, 0.0]))),
        (1, 2, dp(imu), ip(cnt), dp(np.array([0.1, np.nan]))),
    ]
    for n_seq, k, a, c, d in bad:
        assert L.prism_rollout(F.h, n_seq, k, a, c, d, None, None, None, None) == _lib.EINVAL
    imu_nan = imu.copy()
    imu_nan[3, 2] = np.inf
    assert L.prism_rollout(F.h, 1, 2, dp(imu_nan), ip(cnt), dp(dts), None, None, None, None) == _lib.EINVAL
    F.close()


def test_rollout_full_size_sampled(oracle_mod):
    """The 256^3 map and 640x480 frames of the benchmark workload: 32
    candidate sequences of 10 frames in one call, as the benchmark times
    it; every state against the oracle, and 1500 sampled rays of three
    frames rendered by the oracle one by one."""
    O = oracle_mod
    w = synth.ROOM256
    s = synth.Sequence(w, n_frames=24)
    from paper_2212_02988_gb300 import make_state
    m = s.settled_map()
    F, p = make_pair(w, O, map_arrays=m)
    pose, vel, cov = start_state(s, 3)
    F.set_state(make_state(pose, vel, cov))
    n_seq, k = 32, 10
    wins = candidates(s, 3, n_seq, k, seed=3)
    out = F.rollout(wins, w.dt, hitk=True)
    rng = np.random.default_rng(1)
    for si in range(n_seq):
        ref, _ = O.rollout(p, O.make_state(pose, vel, cov), wins[si], [w.dt] * k)
        for i in range(k):
            g = check_states(out["states"][si][i], ref[i])
            if (si, i) in ((0, 0), (5, 9), (n_seq - 1, 4)):
                pix = rng.choice(w.width * w.height, 1500, replace=False).astype(np.int32)
                ref_img = O.render(p, m[0], m[1], g["pose"], pix=pix)
                idx = torch.from_numpy(pix).long().to(out["depth"].device)
                sub = {key: v.reshape(-1, *v.shape[2:])[idx] for key, v in frame_out(out, si, i).items()}
                check_render(sub, ref_img)
    F.close()
