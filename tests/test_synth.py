"""The seeded synthetic inputs keep the recipe the benchmark and the parity
tests rely on: the same seed gives the same arrays, the trajectory stays
inside its workload's speed limits and in free space, frames follow the
camera and depth conventions, IMU windows partition the sensor time, the
settled map is the truncated signed distance of the scene, and the serving
mix draws its streams from the stated sets."""
import numpy as np
import pytest

import synth
from synth import serving


@pytest.fixture(scope="module")
def seq():
    return synth.Sequence(synth.ROOM64)


def test_same_seed_same_inputs_other_seed_other_inputs(seq):
    w = synth.ROOM64
    again = synth.Sequence(w)
    for i in (0, 7, 31):
        a, b = seq.frame(i), again.frame(i)
        assert np.array_equal(a["depth"], b["depth"]) and np.array_equal(a["rgb"], b["rgb"])
        assert np.array_equal(seq.pose7(i), again.pose7(i))
        if i:
            assert np.array_equal(seq.imu_window(i), again.imu_window(i))
    for x, y in zip(seq.settled_map(), again.settled_map()):
        assert np.array_equal(x, y)
    other = synth.Sequence(w, seed=w.seed + 17)
    assert not np.array_equal(seq.pose7(5), other.pose7(5))
    assert not np.array_equal(seq.frame(5)["depth"], other.frame(5)["depth"])


def test_trajectory_respects_the_workload_limits(seq):
    w = synth.ROOM64
    lo, hi = w.origin, w.origin + w.extent
    for i in range(0, w.n_frames, 3):
        v = seq.velocity(i)
        assert np.linalg.norm(v[:3]) <= w.v_max * 1.001
        assert np.degrees(np.linalg.norm(v[3:])) <= w.w_max_deg * 1.001
        t = seq.pose7(i)[:3]
        assert np.all(t > lo) and np.all(t < hi)
        q = seq.pose7(i)[3:]
        assert abs(np.linalg.norm(q) - 1.0) < 1e-12


def test_frames_follow_the_camera_conventions(seq):
    w = synth.ROOM64
    for i in (0, 12, 40):
        c = seq.frame(i, noise=False)
        d, rgb = c["depth"], c["rgb"]
        assert d.shape == (w.height, w.width) and rgb.shape == (w.height, w.width, 3)
        assert d.dtype == np.float32 and rgb.dtype == np.float32
        valid = d > 0
        assert valid.mean() > 0.99            # a closed room: every ray meets a surface
        assert np.all(d[valid] < np.sqrt(3) * w.extent)
        assert np.all(rgb >= 0) and np.all(rgb <= 1)
    # the noisy frame differs from the clean one by the stated noise levels
    n, c = seq.frame(9), seq.frame(9, noise=False)
    m = c["depth"] > 0
    assert abs(np.std(n["depth"][m] - c["depth"][m]) - w.depth_sigma) < 0.1 * w.depth_sigma
    assert abs(np.std(n["rgb"] - c["rgb"]) - w.rgb_sigma) < 0.1 * w.rgb_sigma


def test_imu_windows_partition_sensor_time(seq):
    w = synth.ROOM64
    per = w.imu_rate / w.rate
    prev_end = seq.time(0)
    for i in range(1, 20):
        win = seq.imu_window(i)
        assert win.shape[1] == 7 and abs(len(win) - per) <= 1
        assert np.all(win[:, 0] > seq.time(i - 1)) and np.all(win[:, 0] <= seq.time(i) + 1e-9)
        assert np.all(np.diff(win[:, 0]) > 0) and win[0, 0] > prev_end - 1e-12
        prev_end = win[-1, 0]
        # specific force magnitude near gravity for this gentle motion (|a| << g)
        assert np.all(np.abs(np.linalg.norm(win[:, 1:4], axis=1) - np.linalg.norm(synth.GRAVITY)) < 3.0)


def test_settled_map_is_the_truncated_signed_distance(seq):
    w = synth.ROOM64
    occ, rgb, var_occ, var_rgb = seq.settled_map()
    trunc = 2.0 * w.voxel
    assert occ.shape == (w.n,) * 3 and rgb.shape == (w.n,) * 3 + (3,)
    assert np.all(occ >= -trunc - 1e-6) and np.all(occ <= trunc + 1e-6)
    # camera centres lie in free space (occupancy at -trunc, far from surfaces)
    for i in range(0, w.n_frames, 7):
        t = seq.pose7(i)[:3]
        ijk = np.floor((t - w.origin) / w.voxel).astype(int)
        assert occ[ijk[2], ijk[1], ijk[0]] < 0
    seen = var_occ < 1.0
    assert np.all(var_occ[seen] == np.float32(0.1)) and np.all(var_occ[~seen] == np.float32(1e4))
    assert np.all(occ[~seen] == np.float32(-0.001))
    # colour only within the band around surfaces: none in deep free space
    # (occupancy clamped at -trunc) or in unseen voxels, some in the band
    free = occ <= -trunc + 1e-6
    assert free.mean() > 0.3
    assert np.all(rgb[free] == 0) and np.all(rgb[~seen] == 0)
    band = seen & (np.abs(occ) < trunc - 1e-6)
    assert np.mean(rgb[band].sum(axis=-1) > 0) > 0.99


def test_serving_mix_draws_from_the_stated_sets():
    plans = serving.serving_plan(32, 120.0, seed=4000)
    first = [p for p in plans if p.arrival_s <= 1.0]
    assert len(first) >= 32
    for p in plans:
        w = p.workload
        assert (w.n, w.extent) in serving.MAPS and (w.width, w.height) in serving.FRAMES
        assert 10.0 <= w.rate <= 30.0 and w.storage == "bf16" and w.periodic
        assert 0.25 * 120.0 <= p.lifetime_s <= 0.75 * 120.0
    assert plans == serving.serving_plan(32, 120.0, seed=4000)
    rng = np.random.default_rng(1)
    rt = serving.request_times(plans[0], rng, 120.0)
    assert np.all(np.diff(rt) > 0) and rt[0] == plans[0].arrival_s
