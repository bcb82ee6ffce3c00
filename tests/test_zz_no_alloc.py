"""The allocation-free normal-equation entry point (for callers that may not
allocate device memory at run time) against the handle-based one.

It is called twice in a row through the C ABI; each result must match what
prism_anchor_load + prism_normal_equations give for the same inputs, within
the tolerance of tests/test_gpu_track.py, and the second call must leave the
device's free memory unchanged (nothing allocated).  This file is collected
last, so a run that stops at the first failure has run every other test."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu


def _close(got, ref):
    assert got["count"] == ref["count"] > 0
    assert got["cost"] == pytest.approx(ref["cost"], rel=1e-5)
    for k in ("H", "Ht"):
        scale = np.sqrt(np.outer(np.diag(ref[k]), np.diag(ref[k])))
        assert np.all(np.abs(got[k] - ref[k]) <= 2e-4 * scale), k
    gscale = np.sqrt(np.diag(ref["H"]) * ref["cost"])
    assert np.all(np.abs(got["g"] - ref["g"]) <= 2e-4 * gscale)


@pytest.mark.parametrize("w", [synth.ROOM128, synth.ROOM256], ids=lambda w: w.name)
def test_noalloc_matches_handle_path(oracle_mod, w):
    """320x240, and 640x480: the stated maximum, which fills the scratch
    array's anchor and mask regions exactly."""
    from paper_2212_02988_gb300 import PrismError, config, normal_equations_noalloc
    s = synth.Sequence(w)
    F, _ = make_pair(w, oracle_mod)
    A = s.pose7(8)
    a_d, a_rgb = (x.astype(np.float32) for x in s.clean_frame(8))
    f = s.frame(9)
    poses = [f["pose"], s.pose7(10)]
    F.anchor_load(A, t(a_d), t(a_rgb))
    refs = [F.normal_equations(p, t(f["depth"]), t(f["rgb"])) for p in poses]
    F.close()
    cfg = config(w.n, w.extent, w.width, w.height)
    ad, ac, od, oc = t(a_d), t(a_rgb), t(f["depth"]), t(f["rgb"])
    torch.cuda.synchronize()
    got0 = normal_equations_noalloc(cfg, A, ad, ac, poses[0], od, oc)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    got1 = normal_equations_noalloc(cfg, A, ad, ac, poses[1], od, oc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    _close(got0, refs[0])
    _close(got1, refs[1])
    # one pixel column beyond the stated maximum is rejected before any GPU work
    big = config(w.n, w.extent, 641, 480)
    bd = torch.ones((480, 641), device=ad.device)
    bc = torch.zeros((480, 641, 3), device=ad.device)
    with pytest.raises(PrismError) as e:
        normal_equations_noalloc(big, A, bd, bc, poses[0], bd, bc)
    assert e.value.status == -1 and "at most" in str(e.value)
