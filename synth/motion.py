"""Seeded smooth camera trajectories and the IMU readings they produce.

A trajectory is a sum of sinusoids in position and in yaw/pitch/roll, scaled
so that its speed and angular rate stay below the workload's limits and its
position stays inside a central region of the room.  Because it is analytic,
velocity and acceleration are exact; angular velocity is obtained by a
central difference of the rotation with a 1e-5 s step.

IMU model (camera frame, co-located with the camera):
  accelerometer  f = R^T (a_w - g) + b_a + n_a,   g = (0, 0, -9.81)
  gyroscope      w = R^T w_w + b_g + n_g
with white noise n ~ N(0, sigma^2) per sample and random-walk biases
b_{k+1} = b_k + sigma_walk * sqrt(dt) * N(0, 1), starting at zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._rot import expm_so3_batch, logm_so3_batch, quat_from_matrix, rot_zyx_batch
from .configs import Workload

GRAVITY = np.array([0.0, 0.0, -9.81])
# camera -> body (body: x forward, y left, z up; camera: x right, y down, z forward)
R_BODY_CAM = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


@dataclass
class Trajectory:
    centre: np.ndarray
    p_amp: np.ndarray     # (3, J)
    p_freq: np.ndarray    # (3, J) Hz
    p_phase: np.ndarray   # (3, J)
    yaw0: float
    r_amp: np.ndarray     # (3, K) yaw, pitch, roll amplitudes (rad)
    r_freq: np.ndarray    # (3, K)
    r_phase: np.ndarray   # (3, K)
    j_amp: np.ndarray     # (3, L) rotation jitter (rad), applied on the left
    j_freq: np.ndarray
    j_phase: np.ndarray

    # ---- position ----------------------------------------------------------
    def position(self, t):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        arg = 2 * np.pi * self.p_freq[None] * t[:, None, None] + self.p_phase[None]
        return self.centre[None] + np.sum(self.p_amp[None] * np.sin(arg), axis=2)

    def velocity(self, t):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        w = 2 * np.pi * self.p_freq[None]
        arg = w * t[:, None, None] + self.p_phase[None]
        return np.sum(self.p_amp[None] * w * np.cos(arg), axis=2)

    def acceleration(self, t):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        w = 2 * np.pi * self.p_freq[None]
        arg = w * t[:, None, None] + self.p_phase[None]
        return -np.sum(self.p_amp[None] * w * w * np.sin(arg), axis=2)

    # ---- orientation -------------------------------------------------------
    def rotation(self, t):
        """Camera-to-world rotations at times t, (n, 3, 3)."""
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        ang = np.sum(self.r_amp[None] * np.sin(2 * np.pi * self.r_freq[None] * t[:, None, None]
                                               + self.r_phase[None]), axis=2)
        ang[:, 0] += self.yaw0
        jit = np.sum(self.j_amp[None] * np.sin(2 * np.pi * self.j_freq[None] * t[:, None, None]
                                               + self.j_phase[None]), axis=2)
        Rwb = rot_zyx_batch(ang[:, 0], ang[:, 1], ang[:, 2])
        return expm_so3_batch(jit) @ Rwb @ R_BODY_CAM[None]

    def rotation1(self, t: float):
        return self.rotation(np.array([t]))[0]

    def omega_world(self, t, h: float = 1e-5):
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        Rp, Rm = self.rotation(t + h), self.rotation(t - h)
        return logm_so3_batch(Rp @ np.transpose(Rm, (0, 2, 1))) / (2 * h)

    def pose(self, t: float):
        """(translation (3,), quaternion (w, x, y, z)) of the camera at time t."""
        return self.position(t)[0], quat_from_matrix(self.rotation1(t))


def make_trajectory(w: Workload, rng: np.random.Generator, duration: float,
                    wall_margin: float, period: float | None = None) -> Trajectory:
    """With `period`, every frequency drawn is moved to the nearest positive
    multiple of 1/period, so the whole motion repeats with that period (the
    random draws, and hence all other trajectories, are unchanged)."""
    def per(f):
        return f if period is None else np.maximum(1.0, np.round(f * period)) / period

    half = 0.5 * w.extent
    region = np.array([half - wall_margin - 1.0, half - wall_margin - 1.0,
                       0.3 if w.extent < 5 else 0.6])
    J = 3
    base_f = w.v_max / (2 * np.pi * region[:2].mean())
    p_freq = per(base_f * rng.uniform(0.6, 1.5, size=(3, J)))
    p_amp = rng.uniform(0.3, 1.0, size=(3, J))
    p_phase = rng.uniform(0, 2 * np.pi, size=(3, J))
    K = 2
    r_freq = per(rng.uniform(0.05, 0.4, size=(3, K)) * max(1.0, w.w_max_deg / 120.0))
    r_amp = np.stack([rng.uniform(0.5, 1.0, K), rng.uniform(0.05, 0.15, K),
                      rng.uniform(0.03, 0.08, K)])
    r_phase = rng.uniform(0, 2 * np.pi, size=(3, K))
    if w.jitter:
        j_freq = per(rng.uniform(7.0, 13.0, size=(3, 2)))
        j_amp = np.full((3, 2), 0.002)
        j_phase = rng.uniform(0, 2 * np.pi, size=(3, 2))
        pj_amp = np.full((3, 2), 0.002)
        pj_freq = per(rng.uniform(7.0, 13.0, size=(3, 2)))
        pj_phase = rng.uniform(0, 2 * np.pi, size=(3, 2))
    else:
        j_freq = np.zeros((3, 1))
        j_amp = np.zeros((3, 1))
        j_phase = np.zeros((3, 1))
    tr = Trajectory(np.zeros(3), p_amp, p_freq, p_phase, rng.uniform(-np.pi, np.pi),
                    r_amp, r_freq, r_phase, j_amp, j_freq, j_phase)
    ts = np.linspace(0.0, duration, max(400, int(duration * 50)))
    # scale position amplitudes: stay inside the region and below 0.9 v_max
    off = np.abs(tr.position(ts)).max(axis=0)
    s_ext = np.min(region / np.maximum(off, 1e-9))
    tr.p_amp = tr.p_amp * s_ext
    if w.jitter:
        tr.p_amp = np.concatenate([tr.p_amp, pj_amp], axis=1)
        tr.p_freq = np.concatenate([tr.p_freq, pj_freq], axis=1)
        tr.p_phase = np.concatenate([tr.p_phase, pj_phase], axis=1)
    vmax = np.linalg.norm(tr.velocity(ts), axis=1).max()
    if vmax > 0.9 * w.v_max:
        tr.p_amp = tr.p_amp * (0.9 * w.v_max / vmax)
    # scale rotation amplitudes to an angular-rate peak of 0.9 w_max
    wlim = np.deg2rad(w.w_max_deg) * 0.9
    ts_r = np.linspace(0.0, duration, max(200, int(duration * 20)))
    for _ in range(4):
        rate = np.linalg.norm(tr.omega_world(ts_r), axis=1).max()
        s = wlim / max(rate, 1e-9)
        tr.r_amp[0] *= s
        tr.r_amp[1:] = np.minimum(tr.r_amp[1:] * s, np.array([[0.3], [0.2]]))
    rate = np.linalg.norm(tr.omega_world(ts_r), axis=1).max()
    if rate > wlim:
        tr.r_amp *= wlim / rate
    return tr


@dataclass
class ImuWindow:
    t: np.ndarray      # (k,) sample times
    acc: np.ndarray    # (k, 3) specific force, camera frame
    gyro: np.ndarray   # (k, 3) angular rate, camera frame

    def packed(self) -> np.ndarray:
        """(k, 7) rows of (t, acc_x, acc_y, acc_z, gyro_x, gyro_y, gyro_z)."""
        return np.concatenate([self.t[:, None], self.acc, self.gyro], axis=1)


def make_imu(w: Workload, tr: Trajectory, rng: np.random.Generator, t_end: float):
    n = int(np.floor(t_end * w.imu_rate)) + 1
    t = np.arange(n) / w.imu_rate
    dt = 1.0 / w.imu_rate
    R = tr.rotation(t)
    a = tr.acceleration(t)
    om = tr.omega_world(t)
    ba = np.cumsum(rng.normal(0, w.acc_bias_walk * np.sqrt(dt), size=(n, 3)), axis=0)
    bg = np.cumsum(rng.normal(0, w.gyro_bias_walk * np.sqrt(dt), size=(n, 3)), axis=0)
    acc = np.einsum("nji,nj->ni", R, a - GRAVITY[None]) + ba + rng.normal(0, w.acc_sigma, (n, 3))
    gyro = np.einsum("nji,nj->ni", R, om) + bg + rng.normal(0, w.gyro_sigma, (n, 3))
    return t, acc, gyro
