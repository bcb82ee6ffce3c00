"""The bounds-check build (libprism_checked.so, prism_check_status in
include/prism.h): on small workloads through every kernel family -- filter
steps in both storages with the planned anchor-render order (80x60 and
320x240; the Gauss-Newton passes after the first in one cooperative
launch), renders of a ragged image from cameras inside and outside the
grid, the render adjoint, rollouts, a map-descent step, two streams through
the server -- it records no index violation, and its results are
bit-identical to the plain library's (the tests change no arithmetic)
except for the sums formed by atomic adds (the adjoint's gradients, the map
loss), whose order varies from run to run in either library.  Each build
runs in its own process (the binding loads one library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run(tmp_path, checked):
    lib = "libprism_checked.so" if checked else "libprism.so"
    if not os.path.exists(os.path.join(ROOT, "paper_2212_02988_gb300", lib)):
        raise RuntimeError(f"{lib} is missing: run the package build")
    path = os.path.join(tmp_path, f"{'checked' if checked else 'plain'}.npz")
    env = dict(os.environ)
    env.pop("PRISM_CHECKED", None)
    if checked:
        env["PRISM_CHECKED"] = "1"
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workloads.py"), path], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(path))


def test_checked_build_records_nothing_and_changes_nothing(tmp_path):
    c = run(tmp_path, True)
    p = run(tmp_path, False)
    assert int(c["checked_build"]) == 1 and int(p["checked_build"]) == 0
    assert c["words"].shape == (5,) and np.all(c["words"] == 0), [hex(int(x)) for x in c["words"]]
    assert np.all(p["words"] == 0)
    # the adjoint's gradients and the map loss are sums by atomic adds, whose
    # order varies from run to run: compared to their rounding
    atomic = {"bwd_pose": 1e-5, "bwd_occ": 1e-5, "descent_loss": 1e-9}
    for k in p:
        if k in ("checked_build", "words"):
            continue
        if k in atomic:
            scale = np.abs(p[k]).max() if p[k].size else 0.0
            assert np.allclose(c[k], p[k], rtol=atomic[k], atol=atomic[k] * scale), k
        else:
            assert np.array_equal(c[k], p[k], equal_nan=True), k
