"""GPU parity of the localisation path with the FP64 oracle, through the C ABI:
one evaluation of the normal equations (App. E.3), the prediction step
(App. E.1/E.2), and the full localise (Gauss-Newton + Laplace + recombination).

Bars: kept-pixel count exact (the decisions are bit-identical at a given
pose); sums within 2e-4 of their scale (FP32 per-pixel arithmetic against
FP64; for the world-frame matrices the scale of the camera-frame sums they
are rotated from, gpu_helpers.world_frame_scale); poses within 1 mm / 0.05
deg; covariances within 1e-3 relative."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from gpu_helpers import make_pair, quat_angle_deg, t, world_frame_scale

pytestmark = pytest.mark.gpu


def perturb(pose7, d):
    w, x, y, z = pose7[3:]
    R = Rotation.from_rotvec(d[3:]).as_matrix() @ Rotation.from_quat([x, y, z, w]).as_matrix()
    qx, qy, qz, qw = Rotation.from_matrix(R).as_quat()
    return np.concatenate([pose7[:3] + d[:3], [qw, qx, qy, qz]])


def frames(s, w, i_anchor, i_obs):
    A = s.pose7(i_anchor)
    a_d, a_rgb = (x.astype(np.float32) for x in s.clean_frame(i_anchor))
    f = s.frame(i_obs)
    return A, a_d, a_rgb, f


@pytest.mark.parametrize("name", ["room64_80x60", "room128_320x240", "room256_640x480"])
def test_normal_equations_match_oracle(oracle_mod, name):
    """At 640x480 the pass runs its full grid (152 blocks of 512 threads) and
    the last block adds the FP32 block partials in a fixed order.  Each sum
    is a chain of at most about 60 FP32 additions: 16 terms a thread (4
    pixels x 4 residuals), 5 butterfly levels, 16 warps, 16 partials a lane
    and 5 shuffle levels; its rounding is bounded by 60 * 2^-24 ~ 3.6e-6 of
    the sum of the terms' magnitudes -- for H_ij at most sqrt(H_ii H_jj)
    (Cauchy-Schwarz) -- well inside the 2e-4 bar that the FP32 evaluation of
    each pixel's residuals and Jacobians sets."""
    O = oracle_mod
    w = synth.PRESETS[name]
    s = synth.Sequence(w)
    F, p = make_pair(w, O)
    A, a_d, a_rgb, f = frames(s, w, 4, 5)
    F.anchor_load(A, t(a_d), t(a_rgb))
    for pose in (f["pose"], perturb(f["pose"], np.array([0.004, -0.003, 0.002, 0.003, 0.002, -0.004]))):
        got = F.normal_equations(pose, t(f["depth"]), t(f["rgb"]))
        ref = O.normal_equations(p, A, a_d, a_rgb, pose, f["depth"], f["rgb"])
        assert got["count"] == ref["count"] > 0.5 * w.width * w.height
        assert got["cost"] == pytest.approx(ref["cost"], rel=1e-5)
        for k in ("H", "Ht"):
            scale = world_frame_scale(ref[k], A)
            assert np.all(np.abs(got[k] - ref[k]) <= 2e-4 * scale), (k, np.abs(got[k] - ref[k]) / scale)
        gscale = np.sqrt(np.diag(ref["H"]) * ref["cost"])
        assert np.all(np.abs(got["g"] - ref["g"]) <= 2e-4 * gscale)
    F.close()


def test_predict_matches_oracle(oracle_mod):
    """Localising an empty observation returns the prior unchanged (the pose
    is unobserved), which exposes the device's prediction step."""
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state, state_arrays
    cov = np.diag([4e-4, 4e-4, 4e-4, 1e-4, 1e-4, 1e-4, 2e-3, 2e-3, 2e-3, 3e-3, 3e-3, 3e-3])
    vel = s.velocity(6) + np.array([0.05, -0.02, 0.01, 0.1, -0.2, 0.05])
    F, p = make_pair(w, O)
    F.set_state(make_state(s.pose7(6), vel, cov))
    A, a_d, a_rgb, f = frames(s, w, 6, 7)
    F.anchor_load(A, t(a_d), t(a_rgb))
    imu = s.imu_window(7)
    F.predict(imu, w.dt)
    empty = np.zeros_like(f["depth"])
    got = state_arrays(F.localise(t(empty), t(f["rgb"])))
    pr = O.prior_arrays(O.predict(p, O.make_state(s.pose7(6), vel, cov), imu, w.dt))
    np.testing.assert_allclose(got["pose"][:3], pr["pose"][:3], rtol=0, atol=1e-12)
    assert quat_angle_deg(got["pose"][3:], pr["pose"][3:]) < 1e-9
    np.testing.assert_allclose(got["vel"], pr["vel"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["cov"], pr["cov"], rtol=1e-10, atol=1e-16)
    F.close()


@pytest.mark.parametrize("name,pairs", [("room64_80x60", [(3, 4), (10, 11)]), ("room128_320x240", [(5, 6)])])
def test_localise_matches_oracle(oracle_mod, name, pairs):
    O = oracle_mod
    w = synth.PRESETS[name]
    s = synth.Sequence(w)
    from paper_2212_02988_gb300 import make_state, state_arrays
    F, p = make_pair(w, O)
    for ia, io in pairs:
        A, a_d, a_rgb, f = frames(s, w, ia, io)
        prev_cov = np.diag([1e-6] * 3 + [1e-7] * 3 + [1e-4] * 6)
        st0 = make_state(A, s.velocity(ia), prev_cov, n_localised=1)
        F.set_state(st0)
        F.anchor_load(A, t(a_d), t(a_rgb))
        imu = s.imu_window(io)
        F.predict(imu, w.dt)
        got = state_arrays(F.localise(t(f["depth"]), t(f["rgb"])))
        ost = O.make_state(A, s.velocity(ia), prev_cov, n_localised=1)
        ref, diag = O.localise(p, O.predict(p, ost, imu, w.dt), ost, a_d, a_rgb, f["depth"], f["rgb"])
        ref = O.state_arrays(ref)
        assert np.linalg.norm(got["pose"][:3] - ref["pose"][:3]) < 1e-3
        assert quat_angle_deg(got["pose"][3:], ref["pose"][3:]) < 0.05
        assert np.linalg.norm(got["vel"] - ref["vel"]) < 1e-2
        np.testing.assert_allclose(got["cov"], ref["cov"], rtol=2e-2,
                                   atol=2e-2 * np.sqrt(np.outer(np.diag(ref["cov"]), np.diag(ref["cov"]))).max())
        assert got["n_localised"] == 2
    F.close()


def test_localise_requires_prior_and_anchor(oracle_mod):
    from paper_2212_02988_gb300 import PrismError
    w = synth.ROOM64
    F, _ = make_pair(w, oracle_mod)
    d = t(np.ones((w.height, w.width), np.float32))
    c = t(np.zeros((w.height, w.width, 3), np.float32))
    with pytest.raises(PrismError) as e:
        F.localise(d, c)
    assert e.value.status == -5
    with pytest.raises(ValueError):
        F.update_map(d[:, :-1].contiguous(), c)
    F.close()
