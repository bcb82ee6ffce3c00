"""Brick skipping (prism_config.skip_empty): rays jump over 4^3 bricks (or
the largest skippable brick of the 8^3 .. 32^3 levels above them) whose
occupancy bound shows that no sample in them can be a hit.  The renders
(depth, colour, mask, hit index) and whole filter steps must be bit-identical
with and without it, on settled, fused, random and bf16 maps; it must only
evaluate fewer samples."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu


def renders(O, w, maps, poses, storage="f32", **over):
    out = {}
    for skip in (0, 1):
        F, _ = make_pair(w, O, storage=storage, map_arrays=maps, skip_empty=skip, **over)
        s0 = F.stats()["render_samples"]
        res = [F.render(p) for p in poses]
        out[skip] = (res, F.stats()["render_samples"] - s0)
        F.close()
    return out


def assert_same(a, b):
    for k in ("depth", "rgb", "mask", "hitk"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("name,frames,storage", [("room64_80x60", (0, 7, 23), "f32"),
                                                 ("room64_80x60", (3, 30), "bf16"),
                                                 ("room128_320x240", (0, 51), "f32"),
                                                 ("room256_640x480", (0,), "f32")])
def test_skipping_changes_no_render(oracle_mod, name, frames, storage):
    w = synth.PRESETS[name]
    s = synth.Sequence(w, n_frames=max(frames) + 2)
    out = renders(oracle_mod, w, s.settled_map(), [s.pose7(i) for i in frames], storage)
    for a, b in zip(out[0][0], out[1][0]):
        assert_same(a, b)
    assert out[1][1] < out[0][1]


def test_skipping_on_random_field_and_outside_cameras(oracle_mod):
    w = synth.tiny(n=24, width=83, height=61)
    rng = np.random.default_rng(9)
    n = w.n
    c = w.origin + (np.arange(n) + 0.5) * w.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    occ = -0.3 * np.ones((n, n, n))
    for _ in range(6):
        ctr = rng.uniform(-1.5, 1.5, 3)
        occ = np.maximum(occ, rng.uniform(0.2, 0.6) - np.sqrt((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 +
                                                              (Z - ctr[2]) ** 2))
    occ = occ + rng.normal(0, 0.02, occ.shape)
    occ[occ.shape[0] // 2] = -1e-7             # a slab just below tau (no margin to skip it)
    occ = occ.astype(np.float32)
    rgb = rng.uniform(0, 1, (n, n, n, 3)).astype(np.float32)
    var = np.ones((n, n, n), np.float32)
    poses = [np.array([-1.7, 0.3, 0.1, 0.9, 0.1, -0.2, 0.3]), np.array([0.2, -1.9, 1.2, 0.2, 0.6, 0.1, -0.7]),
             np.array([5.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]), np.array([0.0, 0.0, 0.0, 0.5, -0.5, 0.5, 0.5])]
    out = renders(oracle_mod, w, (occ, rgb, var, var), poses)
    for a, b in zip(out[0][0], out[1][0]):
        assert_same(a, b)


def random_field(shape, origin, voxel, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(*(origin + (np.arange(m) + 0.5) * voxel for m in (nz, ny, nx)), indexing="ij")
    occ = -0.3 * np.ones(shape)
    for _ in range(6):
        ctr = rng.uniform(-1.5, 1.5, 3)
        occ = np.maximum(occ, rng.uniform(0.2, 0.6) - np.sqrt((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 +
                                                              (Z - ctr[2]) ** 2))
    occ = (occ + rng.normal(0, 0.02, occ.shape)).astype(np.float32)
    rgb = rng.uniform(0, 1, shape + (3,)).astype(np.float32)
    return occ, rgb


def test_skipping_on_a_non_cubic_grid(oracle_mod):
    """48 x 40 x 24 voxels: 12 x 10 x 6 bricks of 4^3, then 6 x 5 x 3 of 8^3,
    where the pyramid stops (an odd count); different brick counts per axis."""
    w = synth.tiny(n=48, width=71, height=53)
    nx, ny, nz = 48, 40, 24
    org = -0.5 * w.extent
    occ, rgb = random_field((nz, ny, nx), org, w.voxel, seed=21)
    var = np.ones((nz, ny, nx), np.float32)
    poses = [np.array([-1.2, 0.3, 0.1, 0.9, 0.1, -0.2, 0.3]), np.array([0.2, -1.9, -0.8, 0.2, 0.6, 0.1, -0.7]),
             np.array([0.0, 0.0, -1.5, 0.5, -0.5, 0.5, 0.5])]
    out = renders(oracle_mod, w, (occ, rgb, var, var), poses, nx=nx, ny=ny, nz=nz)
    for a, b in zip(out[0][0], out[1][0]):
        assert_same(a, b)
    assert out[1][1] < out[0][1]


@pytest.mark.parametrize("name,storage,start", [("room128_320x240", "f32", "prior"),
                                                ("room128_320x240", "bf16", "prior"),
                                                ("room256_640x480", "f32", "settled"),
                                                ("tiny_83x61", "f32", "prior")])
def test_skipping_changes_no_filter_step(oracle_mod, name, storage, start):
    """From the prior map the fuse writes the tile bounds the render skips
    by; every state and the final map agree bit for bit.  With skipping, the
    brick-bound launch also plans the anchor render's tile order from the
    last anchor render's tile costs (from the second step on), which must
    change nothing either."""
    from paper_2212_02988_gb300 import state_arrays
    # tiny_83x61: a ragged image (6 x 8 tiles of 16x8, the last column and row partial)
    w = synth.tiny(n=32, width=83, height=61) if name == "tiny_83x61" else synth.PRESETS[name]
    s = synth.Sequence(w, n_frames=6)
    frames = [s.frame(i) for i in range(5)]
    runs = {}
    for skip in (0, 1):
        F, _ = make_pair(w, oracle_mod, storage=storage,
                         map_arrays=s.prior_map() if start == "prior" else s.settled_map(), s1_pose=s.pose7(0),
                         vel=s.velocity(0), skip_empty=skip)
        states = [state_arrays(F.step(s.imu_window(i) if i else None, w.dt, t(f["depth"]), t(f["rgb"]),
                                      want_state=True)) for i, f in enumerate(frames)]
        runs[skip] = (states, F.map_store(), F.render(s.pose7(5)), F.stats()["render_samples"])
        F.close()
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a["pose"], b["pose"]) and np.array_equal(a["cov"], b["cov"])
    for k in ("occ", "rgb", "var_occ", "var_rgb"):
        assert torch.equal(runs[0][1][k], runs[1][1][k])
    assert_same(runs[0][2], runs[1][2])
    assert runs[1][3] < runs[0][3]
