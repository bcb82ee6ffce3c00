"""Pins of the oracle's predictive rollout (App. I, "Prediction and Control";
Fig. 1): the prior of each frame, with no observation, becomes the next
frame's state, and each frame renders the map mean at its predicted pose.

The pins are closed forms of the transition of App. E.1 (with the velocity
integration of reading R12, v' = v + u dt, t' = t + v' dt) that hold exactly
when the angular velocity is zero or the controls are constant:
  * constant velocity and constant turn rate move the mean linearly;
  * a constant specific force integrates to t_k = t_0 + k dt v_0 +
    dt^2 u k (k + 1) / 2;
  * with w = 0 each axis is an integrated random walk, so the covariance
    after k frames has a closed form in sigma_vel, sigma_pose and k;
  * a camera driving at a fronto-parallel wall of a linear occupancy field
    sees z-depth = wall - camera z in every frame."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth


def R_of(q):
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def random_walk_cov(k, dt, c0, sv, sp):
    """Per-axis covariance of (pose, velocity) after k frames of
    v_j = v_{j-1} + e_v,j, p_j = p_{j-1} + dt v_j + e_p,j, starting from
    var(p_0) = var(v_0) = c0, cov(p_0, v_0) = 0 (e_v ~ N(0, sv^2),
    e_p ~ N(0, sp^2))."""
    var_p = c0 * (1.0 + (k * dt) ** 2) + dt * dt * sv * sv * k * (k + 1) * (2 * k + 1) / 6.0 + k * sp * sp
    cov_pv = c0 * k * dt + dt * sv * sv * k * (k + 1) / 2.0
    var_v = c0 + k * sv * sv
    return var_p, cov_pv, var_v


def test_constant_velocity_mean_and_closed_form_covariance(O):
    w = synth.ROOM64
    p = O.params(w)
    k, dt, c0 = 12, w.dt, 1e-8
    pose = np.array([0.1, -0.2, 0.3, 0.9, 0.1, -0.3, 0.2])
    pose[3:] /= np.linalg.norm(pose[3:])
    v = np.array([0.3, -0.1, 0.05])
    st = O.make_state(pose, np.concatenate([v, np.zeros(3)]), np.eye(12) * c0)
    states, images = O.rollout(p, st, [None] * k, [dt] * k)
    assert images == []
    for j, s in enumerate(states, start=1):
        np.testing.assert_allclose(s["pose"][:3], pose[:3] + j * dt * v, rtol=0, atol=1e-13)
        q = s["pose"][3:] * np.sign(s["pose"][3] * pose[3])
        np.testing.assert_allclose(q, pose[3:], rtol=0, atol=1e-15)
        np.testing.assert_allclose(s["vel"], np.concatenate([v, np.zeros(3)]), rtol=0, atol=0)
        C = s["cov"]
        expect = np.zeros((12, 12))
        for blk, (sv, sp) in enumerate(((p.sigma_vel[0], p.sigma_pose[0]), (p.sigma_vel[1], p.sigma_pose[1]))):
            vp, cpv, vv = random_walk_cov(j, dt, c0, sv, sp)
            for a in range(3):
                i_p, i_v = 3 * blk + a, 6 + 3 * blk + a
                expect[i_p, i_p], expect[i_v, i_v] = vp, vv
                expect[i_p, i_v] = expect[i_v, i_p] = cpv
        np.testing.assert_allclose(C, expect, rtol=1e-12, atol=1e-18)
        assert s["n_localised"] == 0


def test_constant_turn_rate_rotates_linearly(O):
    w = synth.ROOM64
    p = O.params(w)
    k, dt = 15, w.dt
    pose = np.array([0.0, 0.5, -0.2, 0.8, -0.2, 0.1, 0.3])
    pose[3:] /= np.linalg.norm(pose[3:])
    v, om = np.array([0.2, 0.1, 0.0]), np.array([0.1, -0.3, 0.6])
    st = O.make_state(pose, np.concatenate([v, om]))
    states, _ = O.rollout(p, st, [None] * k, [dt] * k)
    R0 = R_of(pose[3:])
    for j, s in enumerate(states, start=1):
        np.testing.assert_allclose(s["pose"][:3], pose[:3] + j * dt * v, rtol=0, atol=1e-13)
        Rk = Rotation.from_rotvec(j * dt * om).as_matrix() @ R0
        np.testing.assert_allclose(R_of(s["pose"][3:]), Rk, rtol=0, atol=1e-13)
        np.testing.assert_allclose(s["vel"], np.concatenate([v, om]), rtol=0, atol=0)


def test_constant_specific_force_integrates_in_closed_form(O):
    """Camera axes on the world axes, no rotation: the control is the
    specific force plus gravity, u = a + (0, 0, -9.81)."""
    w = synth.ROOM64
    p = O.params(w)
    k, dt, n = 10, w.dt, 20
    t0, v0 = np.array([0.2, -0.1, 0.4]), np.array([0.1, 0.0, -0.05])
    acc = np.array([0.4, -0.2, 9.81 + 0.1])
    u = acc + np.array([0.0, 0.0, -O.GRAVITY])
    windows = []
    for j in range(k):
        ts = j * dt + dt * (np.arange(n) + 1) / n
        windows.append(np.concatenate([ts[:, None], np.tile(acc, (n, 1)), np.zeros((n, 3))], axis=1))
    st = O.make_state(np.concatenate([t0, [1.0, 0.0, 0.0, 0.0]]), np.concatenate([v0, np.zeros(3)]))
    states, _ = O.rollout(p, st, windows, [dt] * k)
    for j, s in enumerate(states, start=1):
        np.testing.assert_allclose(s["vel"][:3], v0 + j * dt * u, rtol=0, atol=1e-13)
        np.testing.assert_allclose(s["pose"][:3], t0 + j * dt * v0 + dt * dt * u * j * (j + 1) / 2,
                                   rtol=0, atol=1e-13)
        np.testing.assert_allclose(s["pose"][3:], [1.0, 0.0, 0.0, 0.0], rtol=0, atol=1e-15)
        assert np.all(s["vel"][3:] == 0)


def test_driving_at_a_wall_renders_the_closing_distance(O):
    """Linear occupancy f(x) = z - z_wall (trilinear interpolation is exact on
    it), camera looking along world +z and moving at 0.2 m/s: every pixel's
    z-depth is z_wall - t_z at every predicted frame."""
    w = synth.tiny(n=32, width=40, height=30)
    p = O.params(w)
    n = w.n
    c = w.origin + (np.arange(n) + 0.5) * w.voxel
    z_wall = 1.1
    occ = np.broadcast_to((c - z_wall)[:, None, None], (n, n, n)).astype(np.float64).copy()
    rgb = np.full((n, n, n, 3), 0.25)
    k, dt = 6, 0.1
    t0, vz = np.array([0.05, -0.1, -0.6]), 0.2
    st = O.make_state(np.concatenate([t0, [1.0, 0.0, 0.0, 0.0]]), np.array([0, 0, vz, 0, 0, 0.0]))
    states, images = O.rollout(p, st, [None] * k, [dt] * k, occ, rgb)
    assert len(images) == k
    for j, (s, im) in enumerate(zip(states, images), start=1):
        tz = t0[2] + j * dt * vz
        assert abs(s["pose"][2] - tz) < 1e-13
        m = im["mask"] > 0
        assert m.mean() > 0.99
        np.testing.assert_allclose(im["depth"][m], z_wall - tz, rtol=2e-6)
        np.testing.assert_allclose(im["rgb"][m], 0.25, rtol=1e-6)
