"""The localisation's two launch forms (prism_set_cooperative): the
Gauss-Newton passes after the first in one cooperative launch (a grid
barrier between passes, the FP64 finish repeated in every block), or one
launch per pass.  Both sum the same pixels in the same order and run the
same FP64 finishes, so every state, the map and the work counters agree bit
for bit, accepted steps and rejected ones alike; the cooperative form
launches n_gn - 2 fewer kernels a localisation."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu

ENOTPD = -4


def run(oracle_mod, w, s, storage, n_gn, coop, frames, bad_from=None):
    """Filter steps over `frames` in one launch form; from step `bad_from` on
    the state is first given an indefinite covariance (set on the host), so
    that those steps are rejected.  Returns (statuses, states, map, stats)."""
    from paper_2212_02988_gb300 import make_state, state_arrays
    from paper_2212_02988_gb300._lib import State
    F, _ = make_pair(w, oracle_mod, storage=storage, map_arrays=s.prior_map(), s1_pose=s.pose7(0),
                     vel=s.velocity(0), n_gn=n_gn)
    F.set_cooperative(coop)
    statuses, states = [], []
    for i, (d, c) in enumerate(frames):
        if bad_from is not None and i == bad_from:
            cur = states[-1]
            cov = np.diag([1e-4] * 3 + [1e-5] * 3 + [1e-3] * 6)
            cov[0, 0] = -1e-2
            F.set_state(make_state(cur["pose"], cur["vel"], cov, n_localised=cur["n_localised"]))
        out = State()
        imu = np.ascontiguousarray(s.imu_window(i) if i else np.zeros((0, 7)), dtype=np.float64)
        st = F.L.prism_step(F.h, imu.ctypes.data_as(C.POINTER(C.c_double)), len(imu) if i else 0, w.dt,
                            C.c_void_p(d.data_ptr()), C.c_void_p(c.data_ptr()), C.byref(out))
        statuses.append(st)
        states.append(state_arrays(out))
    torch.cuda.synchronize()
    res = (statuses, states, F.map_store(), F.stats())
    F.close()
    return res


@pytest.mark.parametrize("name,storage,n_gn", [("room128_320x240", "f32", 10),
                                               ("room128_320x240", "bf16", 3),
                                               ("room256_640x480", "f32", 10),
                                               ("tiny_83x61", "f32", 2)])
def test_cooperative_launch_changes_no_bit(oracle_mod, name, storage, n_gn):
    # tiny_83x61: a ragged image whose pixels fill fewer blocks than the device holds
    w = synth.tiny(n=32, width=83, height=61) if name == "tiny_83x61" else synth.PRESETS[name]
    s = synth.Sequence(w, n_frames=6)
    frames = [(t(f["depth"]), t(f["rgb"])) for f in (s.frame(i) for i in range(5))]
    runs = {coop: run(oracle_mod, w, s, storage, n_gn, coop, frames) for coop in (False, True)}
    (st0, a0, m0, k0), (st1, a1, m1, k1) = runs[False], runs[True]
    assert st0 == st1 == [0] * 5
    for x, y in zip(a0, a1):
        for k in ("pose", "vel", "cov"):
            assert np.array_equal(x[k], y[k]), k
        assert x["n_localised"] == y["n_localised"]
    for k in ("occ", "rgb", "var_occ", "var_rgb"):
        assert torch.equal(m0[k], m1[k]), k
    for k in ("track_pixels", "fuse_updates", "fuse_colour_updates", "render_samples"):
        assert k0[k] == k1[k], k
    # four localisations: n_gn + 1 launches each against three
    assert k0["kernel_launches"] - k1["kernel_launches"] == 4 * (n_gn - 2)


def test_cooperative_launch_rejects_alike(oracle_mod):
    """Steps whose prior is indefinite: both forms raise the same flags and
    reject the same steps, leaving the same state and map."""
    w = synth.ROOM64
    s = synth.Sequence(w, n_frames=6)
    frames = [(t(f["depth"]), t(f["rgb"])) for f in (s.frame(i) for i in range(5))]
    runs = {coop: run(oracle_mod, w, s, "f32", 10, coop, frames, bad_from=3) for coop in (False, True)}
    (st0, a0, m0, _), (st1, a1, m1, _) = runs[False], runs[True]
    assert st0 == st1 and st1[:3] == [0] * 3 and st1[3:] == [ENOTPD] * 2
    for x, y in zip(a0, a1):
        for k in ("pose", "vel", "cov"):
            assert np.array_equal(x[k], y[k]), k
    for k in ("occ", "rgb", "var_occ", "var_rgb"):
        assert torch.equal(m0[k], m1[k]), k
