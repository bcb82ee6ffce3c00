"""GPU parity of the map update (App. D, Eq. mapupdategauss) with the FP64
oracle, through the C ABI.  The set of updated voxels is bit-identical
(same FP32 decisions); variances and colours agree within 1e-5 relative
(FP32 update arithmetic against FP64).  Occupancy means are averages of
projective SDF values D - z whose FP32 camera depth z carries the rounding
of the voxel centre, the rounded pose matrices and three fused
multiply-adds: at most about 16 * 2^-24 * extent absolute (extent = edge of
the mapped cube), which is the absolute floor used for them."""
import numpy as np
import pytest

import synth
from gpu_helpers import bf16_round, make_pair, t

pytestmark = pytest.mark.gpu


def geom_atol(w):
    return 16 * 2.0 ** -24 * w.extent


def run_both(O, w, s, storage, start, frames_idx):
    F, p = make_pair(w, O, storage=storage, map_arrays=start)
    m = O.map64(*start)
    n_ref = 0
    for i in frames_idx:
        f = s.frame(i)
        from paper_2212_02988_gb300 import make_state
        F.set_state(make_state(f["pose"]))
        F.update_map(t(f["depth"]), t(f["rgb"]))
        n_ref += O.fuse(p, m, f["pose"], f["depth"], f["rgb"])
    got = {k: v.cpu().numpy() for k, v in F.map_store().items()}
    st = F.stats()
    F.close()
    return got, m, n_ref, st


@pytest.mark.parametrize("name", ["room64_80x60", "room128_320x240"])
def test_fuse_from_prior_matches_oracle(oracle_mod, name):
    O = oracle_mod
    w = synth.PRESETS[name]
    s = synth.Sequence(w)
    start = s.prior_map()
    got, ref, n_ref, st = run_both(O, w, s, "f32", start, [0, 1, 2])
    assert st["fuse_updates"] == n_ref
    changed_got = got["var_occ"] != start[2]
    changed_ref = ref["var_occ"] != start[2]
    assert np.array_equal(changed_got, changed_ref)
    np.testing.assert_allclose(got["var_occ"], ref["var_occ"], rtol=1e-5)
    np.testing.assert_allclose(got["var_rgb"], ref["var_rgb"], rtol=1e-5)
    np.testing.assert_allclose(got["occ"], ref["occ"], rtol=1e-5, atol=geom_atol(w))
    np.testing.assert_allclose(got["rgb"], ref["rgb"], rtol=1e-5, atol=1e-6)


def test_fuse_settled_map_matches_oracle(oracle_mod):
    O = oracle_mod
    w = synth.ROOM128
    s = synth.Sequence(w)
    start = s.settled_map()
    got, ref, n_ref, st = run_both(O, w, s, "f32", start, [10, 11])
    assert st["fuse_updates"] == n_ref
    np.testing.assert_allclose(got["occ"], ref["occ"], rtol=1e-5, atol=geom_atol(w))
    np.testing.assert_allclose(got["var_occ"], ref["var_occ"], rtol=1e-5)


def test_fuse_bf16_error_is_bounded(oracle_mod):
    """bf16 storage rounds every stored mean and variance (8-bit mantissa):
    per update the error is at most half an ulp of the stored value, i.e.
    2^-9 relative; after k updates the decision set is still the same (the
    decisions do not read the map) and the error stays below k * 2^-8."""
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    start = tuple(bf16_round(a) for a in s.prior_map())
    got, ref, n_ref, st = run_both(O, w, s, "bf16", start, [0, 1, 2, 3])
    assert st["fuse_updates"] == n_ref
    k = 4
    trunc = 2 * w.voxel
    assert np.all(np.abs(got["var_occ"] - ref["var_occ"]) <= k * 2 ** -8 * np.abs(ref["var_occ"]))
    assert np.all(np.abs(got["occ"] - ref["occ"]) <= k * 2 ** -8 * (np.abs(ref["occ"]) + trunc))
