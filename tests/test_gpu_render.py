"""GPU parity of the render (App. B) with the FP64 oracle, through the C ABI.

Bar: hit sample indices (the traversal) bit-exact; depth and colour within
1e-5 relative of the oracle (FP32 arithmetic against FP64; the absolute
floor 1e-6 covers colours near zero)."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import RTOL, bf16_round, check_render, make_pair, t

pytestmark = pytest.mark.gpu



@pytest.mark.parametrize("name,frames", [("room64_80x60", (0, 7, 23)), ("room128_320x240", (0, 51))])
def test_render_settled_map(oracle_mod, name, frames):
    O = oracle_mod
    w = synth.PRESETS[name]
    s = synth.Sequence(w)
    m = s.settled_map()
    F, p = make_pair(w, O, map_arrays=m)
    for i in frames:
        out = F.render(s.pose7(i))
        ref = O.render(p, m[0], m[1], s.pose7(i))
        check_render(out, ref)
    F.close()


def test_render_ragged_image_and_random_field(oracle_mod):
    """83x61 image (ragged against the 16x8 tiles), a noisy random field with
    many near-tau values, a camera partly looking out of the grid."""
    O = oracle_mod
    w = synth.tiny(n=24, width=83, height=61)
    rng = np.random.default_rng(4)
    n = w.n
    c = w.origin + (np.arange(n) + 0.5) * w.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    occ = -0.3 * np.ones((n, n, n))
    for _ in range(8):
        ctr = rng.uniform(-1.5, 1.5, 3)
        occ = np.maximum(occ, rng.uniform(0.2, 0.6) - np.sqrt((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 + (Z - ctr[2]) ** 2))
    occ = (occ + rng.normal(0, 0.02, occ.shape)).astype(np.float32)
    rgb = rng.uniform(0, 1, (n, n, n, 3)).astype(np.float32)
    var = np.ones((n, n, n), np.float32)
    F, p = make_pair(w, O, map_arrays=(occ, rgb, var, var))
    poses = [np.array([-1.7, 0.3, 0.1, 0.9, 0.1, -0.2, 0.3]), np.array([0.2, -1.9, 1.2, 0.2, 0.6, 0.1, -0.7])]
    for pose in poses:
        check_render(F.render(pose), O.render(p, occ, rgb, pose))
    F.close()


def test_render_edge_cases(oracle_mod):
    O = oracle_mod
    w = synth.tiny(n=16, width=20, height=14)
    n = w.n
    empty = np.full((n, n, n), -0.001, np.float32)
    zero = np.zeros((n, n, n, 3), np.float32)
    var = np.full((n, n, n), 1e4, np.float32)
    F, p = make_pair(w, O, map_arrays=(empty, zero, var, var))
    pose = np.array([0.1, 0.2, -0.3, 1.0, 0.0, 0.0, 0.0])
    out = F.render(pose)
    assert int(out["mask"].sum()) == 0 and float(out["depth"].abs().sum()) == 0.0
    check_render(out, O.render(p, empty, zero, pose))
    # camera outside the grid: background everywhere (reading R5)
    out = F.render(np.array([5.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]))
    assert int((out["hitk"] != 0).sum()) == 0
    # camera inside matter: hit at the first sample is invalid (hitk = -1)
    full = np.ones((n, n, n), np.float32)
    F.map_load(*(t(a) for a in (full, zero, var, var)))
    out = F.render(pose)
    assert bool((out["hitk"] == -1).all()) and int(out["mask"].sum()) == 0
    F.close()
    # max_depth limits the march
    w64 = synth.ROOM64
    s = synth.Sequence(w64)
    m = s.settled_map()
    F, p = make_pair(w64, O, map_arrays=m, max_depth=1.2)
    check_render(F.render(s.pose7(3)), O.render(p, m[0], m[1], s.pose7(3)))
    F.close()


def test_render_bf16_storage(oracle_mod):
    """bf16 storage: both sides read the same bf16-rounded map values."""
    O = oracle_mod
    w = synth.ROOM128
    s = synth.Sequence(w)
    occ, rgb, vo, vr = (bf16_round(a) for a in s.settled_map())
    F, p = make_pair(w, O, storage="bf16", map_arrays=(occ, rgb, vo, vr))
    for i in (0, 40):
        check_render(F.render(s.pose7(i)), O.render(p, occ, rgb, s.pose7(i)))
    stored = F.map_store()
    assert np.array_equal(stored["occ"].cpu().numpy(), occ)
    F.close()


def test_render_full_size_sampled(oracle_mod):
    """The 256^3 map and 640x480 frame of the benchmark workload, in the
    launch configuration the benchmark times; the oracle checks 4000
    sampled rays one by one."""
    O = oracle_mod
    w = synth.ROOM256
    s = synth.Sequence(w, n_frames=8)
    m = s.settled_map()
    F, p = make_pair(w, O, map_arrays=m)
    rng = np.random.default_rng(0)
    for i in (0, 5):
        out = F.render(s.pose7(i))
        pix = rng.choice(w.width * w.height, 4000, replace=False).astype(np.int32)
        ref = O.render(p, m[0], m[1], s.pose7(i), pix=pix)
        sub = {k: (v.reshape(-1, *v.shape[2:])[torch.from_numpy(pix).long().to(v.device)]
                   if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
        check_render(sub, ref)
    F.close()
