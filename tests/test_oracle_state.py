"""Pins of the oracle's prediction step (App. E.1/E.2, Eq. statepropagation)
against Monte Carlo through the exact nonlinear transition, least-squares
regression on samples, and noise-free IMU on the true trajectory."""
from dataclasses import replace

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth


def R_of(q):
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


@pytest.fixture(scope="module")
def setup(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    p = O.params(w)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(12, 12)) * 0.2
    cov = np.diag([4e-4, 4e-4, 4e-4, 1e-4, 1e-4, 1e-4, 2e-3, 2e-3, 2e-3, 3e-3, 3e-3, 3e-3])
    L = np.linalg.cholesky(cov)
    cov = L @ (np.eye(12) + 0.3 * (A + A.T) / 2 @ (A + A.T).T / 12) @ L.T
    st = O.make_state(s.pose7(3), s.velocity(3) + np.array([0.05, -0.02, 0.01, 0.1, -0.2, 0.05]), cov)
    pr = O.predict(p, st, s.imu_window(4), w.dt)
    return O, w, s, p, st, pr, cov


def test_propagation_matches_monte_carlo(setup):
    O, w, s, p, st, pr, cov = setup
    sa, pa = O.state_arrays(st), O.prior_arrays(pr)
    dt = w.dt
    u_dt = pa["vel"] - sa["vel"]                      # control times dt, as applied
    N = 400_000
    rng = np.random.default_rng(9)
    x = rng.multivariate_normal(np.zeros(12), cov, size=N)
    t0, R0 = sa["pose"][:3], R_of(sa["pose"][3:])
    v = sa["vel"][None] + x[:, 6:] + u_dt[None]
    v[:, :3] += rng.normal(0, p.sigma_vel[0], (N, 3))
    v[:, 3:] += rng.normal(0, p.sigma_vel[1], (N, 3))
    t1 = t0[None] + x[:, :3] + v[:, :3] * dt + rng.normal(0, p.sigma_pose[0], (N, 3))
    Rs = Rotation.from_rotvec(x[:, 3:3 + 3]) * Rotation.from_matrix(R0)
    R1 = Rotation.from_rotvec(rng.normal(0, p.sigma_pose[1], (N, 3))) * \
        Rotation.from_rotvec(v[:, 3:] * dt) * Rs
    Rbar = Rotation.from_matrix(R_of(pa["pose"][3:]))
    e = np.concatenate([t1 - pa["pose"][None, :3], (R1 * Rbar.inv()).as_rotvec(),
                        v - pa["vel"][None]], axis=1)
    C = pa["cov"]
    sd = np.sqrt(np.diag(C))
    assert np.all(np.abs(e.mean(axis=0)) < 5 * sd / np.sqrt(N) + 2e-3 * sd)
    Ce = np.cov(e.T)
    tol = 5 * np.sqrt((np.outer(np.diag(C), np.diag(C)) + C ** 2) / N) + 3e-3 * np.outer(sd, sd)
    assert np.all(np.abs(Ce - C) < tol), np.abs(Ce - C).max()


def test_velocity_conditional_matches_regression(setup):
    O, w, s, p, st, pr, cov = setup
    pa = O.prior_arrays(pr)
    N = 400_000
    z = np.random.default_rng(2).multivariate_normal(np.zeros(12), pa["cov"], size=N)
    P, V = z[:, :6], z[:, 6:]
    Dt, *_ = np.linalg.lstsq(P, V, rcond=None)
    resid = V - P @ Dt
    np.testing.assert_allclose(pa["D"], Dt.T, atol=6 * np.sqrt(np.abs(pa["cov_vel"]).max()) /
                               np.sqrt(N) / np.sqrt(np.diag(pa["cov_pp"])).min())
    Cv = np.cov(resid.T)
    sdv = np.sqrt(np.diag(pa["cov_vel"]))
    assert np.all(np.abs(Cv - pa["cov_vel"]) < 6 * np.outer(sdv, sdv) / np.sqrt(N) * np.sqrt(2) + 1e-12)
    np.testing.assert_allclose(pa["cov_pp"], pa["cov"][:6, :6], rtol=0, atol=0)
    np.testing.assert_allclose(pa["prec_pp"] @ pa["cov_pp"], np.eye(6), atol=1e-9)


def test_noise_free_imu_tracks_truth(oracle_mod):
    O = oracle_mod
    w = replace(synth.ROOM64, acc_sigma=0.0, gyro_sigma=0.0, acc_bias_walk=0.0, gyro_bias_walk=0.0)
    s = synth.Sequence(w)
    p = O.params(w)
    for i in (3, 11, 27):
        st = O.make_state(s.pose7(i), s.velocity(i))
        pa = O.prior_arrays(O.predict(p, st, s.imu_window(i + 1), w.dt))
        tv = s.velocity(i + 1)
        assert np.linalg.norm(pa["vel"][:3] - tv[:3]) < 0.05
        assert np.linalg.norm(pa["vel"][3:] - tv[3:]) < 0.05
        # the transition integrates the pose with the new velocity (App. E.1):
        # compare with that Euler step taken from the true state and velocity
        t_euler = s.pose7(i)[:3] + tv[:3] * w.dt
        R_euler = Rotation.from_rotvec(tv[3:] * w.dt).as_matrix() @ R_of(s.pose7(i)[3:])
        assert np.linalg.norm(pa["pose"][:3] - t_euler) < 0.05 * w.dt
        dR = R_of(pa["pose"][3:]) @ R_euler.T
        assert np.linalg.norm(Rotation.from_matrix(dR).as_rotvec()) < 0.05 * w.dt


def test_no_controls_at_rest_keeps_the_mean(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    p = O.params(w)
    pose = np.array([0.1, -0.2, 0.3, 0.9, 0.1, -0.3, 0.2])
    pose[3:] /= np.linalg.norm(pose[3:])
    st = O.make_state(pose, np.zeros(6))
    pa = O.prior_arrays(O.predict(p, st, np.zeros((0, 7)), 0.05))
    np.testing.assert_allclose(pa["pose"][:3], pose[:3], atol=0)
    q = pa["pose"][3:] * np.sign(pa["pose"][3] * pose[3])
    np.testing.assert_allclose(q, pose[3:], atol=1e-15)
    assert np.all(pa["vel"] == 0)
    # covariance grows by the transition noise only (zero prior covariance part aside)
    assert np.all(np.diag(pa["cov"]) > np.diag(O.state_arrays(st)["cov"]))
