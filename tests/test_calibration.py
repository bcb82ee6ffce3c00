"""Pins of the state-uncertainty calibration (App. G, "Uncertainty
Analysis"): the rotation logarithm and the chi-squared CDF against library
routines, and the calibration of residuals drawn from known covariances
(exactly calibrated, pessimistic and optimistic models)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import chi2

from paper_2212_02988_gb300 import calibration as cal


def quat_of(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def test_so3_log_matches_library_including_near_pi():
    rng = np.random.default_rng(0)
    vecs = [np.zeros(3)]
    for a in (1e-9, 1e-4, 0.3, 1.5, 2.9, np.pi - 1e-3, np.pi - 1e-7):
        n = rng.normal(size=3)
        vecs.append(a * n / np.linalg.norm(n))
    for v in vecs:
        R = Rotation.from_rotvec(v).as_matrix()
        np.testing.assert_allclose(cal.so3_log(R), v, rtol=0, atol=1e-9 if np.linalg.norm(v) < 3 else 1e-6)


def test_quat_to_R_matches_library():
    rng = np.random.default_rng(1)
    for _ in range(5):
        R = Rotation.random(random_state=rng).as_matrix()
        np.testing.assert_allclose(cal.quat_to_R(quat_of(R) * 2.5), R, atol=1e-14)


def test_chi2_cdf_matches_library():
    x = np.concatenate([[0.0], np.logspace(-4, 2, 50)])
    for dof in (2, 4, 6, 12):
        np.testing.assert_allclose(cal.chi2_cdf(x, dof), chi2.cdf(x, dof), rtol=1e-12, atol=1e-15)
    with pytest.raises(ValueError):
        cal.chi2_cdf(x, 5)


def test_pose_residual_recovers_a_left_perturbation():
    rng = np.random.default_rng(2)
    R = Rotation.random(random_state=rng).as_matrix()
    t = rng.normal(size=3)
    d = np.array([0.01, -0.02, 0.005, 0.003, -0.001, 0.002])
    est = np.concatenate([t, quat_of(R)])
    tru = np.concatenate([t + d[:3], quat_of(Rotation.from_rotvec(d[3:]).as_matrix() @ R)])
    np.testing.assert_allclose(cal.pose_residual(est, tru), d, atol=1e-12)


def draw(T, cov_scale, seed=3):
    """T estimates whose true poses lie N(0, cov_scale Sigma_t) away, with
    random SPD pose covariances Sigma_t (reported as the 12x12 state covariance)."""
    rng = np.random.default_rng(seed)
    est, tru, covs = [], [], []
    for _ in range(T):
        A = rng.normal(size=(6, 6)) * 0.01
        S = A @ A.T + np.diag([1e-4] * 3 + [4e-5] * 3)
        C = np.eye(12)
        C[:6, :6] = S
        d = np.linalg.cholesky(cov_scale * S) @ rng.normal(size=6)
        R = Rotation.random(random_state=rng).as_matrix()
        t = rng.normal(size=3)
        est.append(np.concatenate([t, quat_of(R)]))
        tru.append(np.concatenate([t + d[:3], quat_of(Rotation.from_rotvec(d[3:]).as_matrix() @ R)]))
        covs.append(C)
    return np.array(est), np.array(covs), np.array(tru)


def test_calibrated_model_whitens_to_standard_normal():
    T = 8000
    est, covs, tru = draw(T, 1.0)
    r = cal.calibrate(est, covs, tru, scale=1.0)
    z = r["whitened"]
    assert np.all(np.abs(z.mean(axis=0)) < 5 / np.sqrt(T))
    np.testing.assert_allclose(np.cov(z.T), np.eye(6), atol=5 * np.sqrt(2 / T))
    # the curve lies on the diagonal within a Kolmogorov-Smirnov band
    assert np.max(np.abs(r["observed"] - r["levels"])) < 1.63 / np.sqrt(T)
    # the maximum-likelihood scale of a calibrated model is 1
    assert abs(cal.calibrate(est, covs, tru)["scale"] - 1.0) < 5 * np.sqrt(2 / (6 * T))


@pytest.mark.parametrize("true_scale", [0.25, 4.0])
def test_mis_scaled_models_bend_the_curve(true_scale):
    """Errors 4x smaller in variance than the covariance claims: pessimistic,
    curve above the diagonal; 4x larger: optimistic, below.  The
    maximum-likelihood correction recovers the factor and straightens the
    curve."""
    T = 8000
    est, covs, tru = draw(T, true_scale, seed=4)
    raw = cal.calibrate(est, covs, tru, scale=1.0)
    inner = (raw["levels"] > 0.05) & (raw["levels"] < 0.95)
    gap = raw["observed"][inner] - raw["levels"][inner]
    assert np.all(gap > 0.05) if true_scale < 1 else np.all(gap < -0.05)
    fit = cal.calibrate(est, covs, tru)
    assert abs(fit["scale"] / true_scale - 1.0) < 5 * np.sqrt(2 / (6 * T))
    assert np.max(np.abs(fit["observed"] - fit["levels"])) < 1.63 / np.sqrt(T) + 2e-3
    np.testing.assert_allclose(fit["precision"], 1.0 / np.diagonal(covs[:, :6, :6], axis1=1, axis2=2))


def test_rejects_mismatched_inputs():
    est, covs, tru = draw(3, 1.0)
    with pytest.raises(ValueError):
        cal.calibrate(est, covs[:2], tru)
    with pytest.raises(ValueError):
        cal.calibrate(est, covs, tru, scale=0.0)
