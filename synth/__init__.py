"""Seeded synthetic inputs for the PRISM filter hot path.

This package is the only code shared by the CUDA path's tests/bench and the
oracle: it produces inputs (scenes, trajectories, IMU windows, noisy RGB-D
frames, settled voxel maps) and holds none of the filter's arithmetic.

    seq = synth.Sequence(synth.ROOM64)
    f = seq.frame(3)            # dict: depth (H,W) f32, rgb (H,W,3) f32, pose, time
    imu = seq.imu_window(3)     # (k, 7) f64 rows (t, acc3, gyro3) in (t_2, t_3]
    occ, rgb, var_occ, var_rgb = seq.settled_map()
"""
from __future__ import annotations

import functools

import numpy as np

from ._rot import matrix_from_quat, quat_from_matrix
from .configs import PRESETS, ROOM64, ROOM128, ROOM256, ROOM256_BF16, Workload, tiny
from .motion import GRAVITY, make_imu, make_trajectory
from .scene import make_scene, raycast, settled_map

__all__ = ["Sequence", "Workload", "PRESETS", "ROOM64", "ROOM128", "ROOM256",
           "ROOM256_BF16", "tiny", "matrix_from_quat", "quat_from_matrix", "GRAVITY"]


class Sequence:
    """All seeded inputs of one workload.  Frame i is taken at time i / rate.

    The trajectory, scene and IMU stream depend only on the workload and the
    seed; `n_frames` only bounds which frames the caller intends to use (a
    value above the workload's own frame count extends the trajectory, which
    then differs from the default one)."""

    def __init__(self, w: Workload, n_frames: int | None = None, seed: int | None = None):
        self.w = w
        self.seed = w.seed if seed is None else seed
        self.n_frames = w.n_frames if n_frames is None else n_frames
        rng = np.random.default_rng(self.seed)
        duration = (max(w.n_frames, self.n_frames) + 1) / w.rate
        margin = 3.0 * w.voxel
        period = w.n_frames / w.rate if w.periodic else None
        self.traj = make_trajectory(w, rng, duration, margin, period)
        keep = self.traj.position(np.linspace(0, duration, max(200, int(duration * 40))))
        self.scene = make_scene(w, np.random.default_rng(self.seed + 1), keep)
        self.imu_t, self.imu_acc, self.imu_gyro = make_imu(
            w, self.traj, np.random.default_rng(self.seed + 2), duration)
        self._noise_seed = self.seed + 3

    # --------------------------------------------------------------- frames
    def time(self, i: int) -> float:
        return i / self.w.rate

    def pose(self, i: int):
        """True camera pose at frame i: (t (3,), q (4,) w-first)."""
        return self.traj.pose(self.time(i))

    def pose7(self, i: int) -> np.ndarray:
        t, q = self.pose(i)
        return np.concatenate([t, q])

    def velocity(self, i: int) -> np.ndarray:
        """True (linear, angular) world-frame velocity at frame i, (6,)."""
        ti = self.time(i)
        return np.concatenate([self.traj.velocity(ti)[0], self.traj.omega_world(ti)[0]])

    def clean_frame(self, i: int):
        t, q = self.pose(i)
        return raycast(self.scene, self.w, matrix_from_quat(q), t)

    def frame(self, i: int, noise: bool = True):
        depth, rgb = self.clean_frame(i)
        if noise:
            rng = np.random.default_rng([self._noise_seed, i])
            valid = depth > 0
            depth = np.where(valid, depth + rng.normal(0, self.w.depth_sigma, depth.shape), 0.0)
            rgb = rgb + rng.normal(0, self.w.rgb_sigma, rgb.shape)
        return {"depth": np.ascontiguousarray(depth, dtype=np.float32),
                "rgb": np.ascontiguousarray(rgb, dtype=np.float32),
                "pose": self.pose7(i), "time": self.time(i)}

    def imu_window(self, i: int) -> np.ndarray:
        """IMU samples with time in (t_{i-1}, t_i], packed (k, 7)."""
        t0, t1 = self.time(i - 1), self.time(i)
        eps = 1e-9
        sel = (self.imu_t > t0 + eps) & (self.imu_t <= t1 + eps)
        return np.ascontiguousarray(np.concatenate(
            [self.imu_t[sel, None], self.imu_acc[sel], self.imu_gyro[sel]], axis=1))

    # ------------------------------------------------------------------ map
    @functools.lru_cache(maxsize=2)
    def settled_map(self):
        return settled_map(self.scene, self.w)

    def prior_map(self, prior_var: float = 1e4, init_occ: float = -0.001):
        n = self.w.n
        return (np.full((n, n, n), init_occ, np.float32), np.zeros((n, n, n, 3), np.float32),
                np.full((n, n, n), prior_var, np.float32), np.full((n, n, n), prior_var, np.float32))
