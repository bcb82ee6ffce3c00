"""State-uncertainty calibration against ground truth (App. G, "Uncertainty
Analysis"; Fig. stateuncertainty).

Host-side analysis of a filter's state history, not part of the filter
step: the pose residuals against true poses in the filter's error-state
convention (t_true = t + e_t, R_true = Exp(e_theta) R, as the state
covariance is defined), one global scalar correction applied to every pose
covariance, the residuals whitened by the covariances' Cholesky factors, the
normalised squared sum of residuals (NSSR, summed over the six pose
dimensions) and its chi-squared calibration curve (the cumulative chi-squared
probability of each NSSR against the fraction of frames observed at or below
it), and the per-dimension precision along the trajectory.
"""
from __future__ import annotations

import math

import numpy as np


def quat_to_R(q) -> np.ndarray:
    """Rotation matrix of a quaternion (w, x, y, z), normalised first."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def so3_log(R) -> np.ndarray:
    """Rotation vector theta with Exp(theta) = R (|theta| <= pi)."""
    R = np.asarray(R, dtype=np.float64)
    v = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])   # sin(a) axis
    c = 0.5 * (np.trace(R) - 1.0)                                                  # cos(a)
    s = np.linalg.norm(v)
    a = math.atan2(s, c)
    if s < 1e-7 and c > 0:
        return v * (1.0 + a * a / 6.0)            # a / sin(a) to second order
    if c > -0.9:
        return v * (a / s)
    # near pi: the axis from the symmetric part, R + R^T = 2 (cos a I + (1 - cos a) n n^T)
    B = 0.5 * (R + R.T) - c * np.eye(3)
    k = int(np.argmax(np.diag(B)))
    n = B[:, k] / np.linalg.norm(B[:, k])
    if np.dot(n, v) < 0:
        n = -n
    return a * n


def pose_residual(est_pose7, true_pose7) -> np.ndarray:
    """e = (t_true - t_est, Log(R_true R_est^T)): the true pose in the
    filter's error-state coordinates around the estimate."""
    est, tru = np.asarray(est_pose7, dtype=np.float64), np.asarray(true_pose7, dtype=np.float64)
    return np.concatenate([tru[:3] - est[:3], so3_log(quat_to_R(tru[3:]) @ quat_to_R(est[3:]).T)])


def chi2_cdf(x, dof: int = 6):
    """Chi-squared CDF for an even number of degrees of freedom:
    P(dof / 2, x / 2) = 1 - exp(-y) sum_{j < dof / 2} y^j / j!, y = x / 2."""
    if dof <= 0 or dof % 2:
        raise ValueError("dof must be a positive even number")
    y = 0.5 * np.asarray(x, dtype=np.float64)
    term, acc = np.ones_like(y), np.zeros_like(y)
    for j in range(dof // 2):
        if j:
            term = term * y / j
        acc = acc + term
    return 1.0 - np.exp(-y) * acc


def calibrate(est_poses, covs, true_poses, scale: float | str = "ml", levels=None) -> dict:
    """Calibration of the pose covariances along one or more trajectories.

    est_poses, true_poses: (T, 7) poses (t, q); covs: (T, 12, 12) state or
    (T, 6, 6) pose covariances (the pose block is used).  scale: the global
    scalar correction c applied to every covariance, or "ml" for the
    maximum-likelihood c of residuals distributed N(0, c Sigma_t), which
    is the mean NSSR over 6.  levels: probabilities of the calibration
    curve (default 0, 0.05, ..., 1)."""
    est = np.asarray(est_poses, dtype=np.float64)
    tru = np.asarray(true_poses, dtype=np.float64)
    S = np.asarray(covs, dtype=np.float64)[:, :6, :6]
    T = len(est)
    if T == 0 or tru.shape != est.shape or S.shape != (T, 6, 6):
        raise ValueError("est_poses, true_poses (T, 7) and covs (T, 12|6, 12|6) must match, T >= 1")
    e = np.stack([pose_residual(est[i], tru[i]) for i in range(T)])
    L = np.linalg.cholesky(S)
    w = np.linalg.solve(L, e[:, :, None])[:, :, 0]   # L_t w_t = e_t
    m = np.sum(w * w, axis=1)
    c = float(np.mean(m) / 6.0) if scale == "ml" else float(scale)
    if not c > 0:
        raise ValueError("the scale must be positive")
    z = w / math.sqrt(c)
    nssr = m / c
    lv = np.linspace(0.0, 1.0, 21) if levels is None else np.asarray(levels, dtype=np.float64)
    p = chi2_cdf(nssr, 6)
    observed = np.array([np.mean(p <= q) for q in lv])
    return {"residuals": e, "scale": c, "whitened": z, "nssr": nssr, "levels": lv, "observed": observed,
            "precision": 1.0 / np.diagonal(S, axis1=1, axis2=2),
            "rms_translation": float(np.sqrt(np.mean(np.sum(e[:, :3] ** 2, axis=1)))),
            "rms_rotation_deg": float(np.degrees(np.sqrt(np.mean(np.sum(e[:, 3:] ** 2, axis=1)))))}
