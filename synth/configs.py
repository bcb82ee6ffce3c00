"""Workload presets for the seeded synthetic inputs.

Each preset fixes the sizes, rates and value distributions of one workload:
the voxel grid (cells per axis and edge length of the mapped cube), the
RGB-D frame size and pinhole intrinsics, the trajectory and IMU rates and
speed limits, and the number of scene primitives.  The generator in this
package turns a preset plus a seed into arrays; nothing here computes any
part of the filter itself.

Conventions shared by every array the generator emits:
  * world frame: z up, gravity (0, 0, -9.81) m/s^2;
  * camera frame: +x right, +y down, +z forward; a pose (t, q) maps camera
    coordinates to world coordinates, X_w = R(q) X_c + t, q = (w, x, y, z);
  * pixels: (u, v) with u the column, pixel centres at integer coordinates,
    cx = (W - 1) / 2, cy = (H - 1) / 2, fx = fy = 70 * W / 80;
  * depth images hold z-depth in metres, 0 where there is no return;
  * voxel (i, j, k) covers [o + i*vs, o + (i+1)*vs) per axis with its value
    at the centre; grids are stored z-major, x fastest: a[k, j, i].
"""
from __future__ import annotations

from dataclasses import dataclass, replace


@dataclass(frozen=True)
class Workload:
    name: str
    n: int                # voxels per axis (cube grid)
    extent: float         # edge length of the mapped cube, metres
    width: int
    height: int
    n_frames: int
    rate: float           # frame rate, Hz
    imu_rate: float       # IMU rate, Hz
    v_max: float          # trajectory speed limit, m/s
    w_max_deg: float      # trajectory angular-rate limit, deg/s
    jitter: bool          # add handheld high-frequency jitter
    n_prims: int          # boxes and spheres inside the room
    textured: bool        # walls carry random 8x8 colour checker patches
    storage: str = "f32"  # map storage type on the device: "f32" or "bf16"
    seed: int = 1000
    depth_sigma: float = 0.01
    rgb_sigma: float = 0.02
    acc_sigma: float = 0.02
    gyro_sigma: float = 0.002
    acc_bias_walk: float = 1e-3    # m/s^2 per sqrt(s)
    gyro_bias_walk: float = 1e-4   # rad/s per sqrt(s)
    periodic: bool = False         # trajectory repeats every n_frames / rate seconds

    @property
    def voxel(self) -> float:
        return self.extent / self.n

    @property
    def origin(self) -> float:
        return -0.5 * self.extent

    @property
    def fx(self) -> float:
        return 70.0 * self.width / 80.0

    @property
    def cx(self) -> float:
        return 0.5 * (self.width - 1)

    @property
    def cy(self) -> float:
        return 0.5 * (self.height - 1)

    @property
    def dt(self) -> float:
        return 1.0 / self.rate


# 64^3 grid at 6.25 cm over a 4 m cube; 80x60 frames; 12 primitives.
ROOM64 = Workload("room64_80x60", 64, 4.0, 80, 60, 50, 10.0, 200.0, 1.0, 60.0,
                  False, 12, False, seed=1000)
# 128^3 grid at 5 cm over 6.4 m; 320x240 frames at 20 Hz; 40 primitives,
# textured walls, handheld jitter.
ROOM128 = Workload("room128_320x240", 128, 6.4, 320, 240, 600, 20.0, 200.0, 1.5,
                   120.0, True, 40, True, seed=1001)
# 256^3 grid at 2.5 cm over 6.4 m; 640x480 frames at 30 Hz; fast UAV-like
# motion with a 1 kHz IMU.
ROOM256 = Workload("room256_640x480", 256, 6.4, 640, 480, 900, 30.0, 1000.0, 5.0,
                   300.0, False, 40, True, seed=1002)
# The same workload with the map stored in bf16.
ROOM256_BF16 = replace(ROOM256, name="room256_640x480_bf16", storage="bf16", seed=1003)

PRESETS = {w.name: w for w in (ROOM64, ROOM128, ROOM256, ROOM256_BF16)}


def tiny(n: int = 16, width: int = 24, height: int = 18, n_prims: int = 4,
         seed: int = 7, textured: bool = True) -> Workload:
    """A small workload for brute-force and finite-difference checks."""
    return Workload(f"tiny{n}_{width}x{height}", n, 4.0, width, height, 6, 10.0,
                    200.0, 1.0, 60.0, False, n_prims, textured, seed=seed)
