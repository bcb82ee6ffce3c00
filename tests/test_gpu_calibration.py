"""State-uncertainty calibration (App. G) of the GPU filter's own output on a
synthetic trajectory with known true poses: the filter steps through the
C ABI, the states come back each frame, and the analysis whitens the pose
residuals by the filter's pose covariances."""
import numpy as np
import pytest

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu


def test_calibration_of_the_filter_on_a_synthetic_trajectory(oracle_mod):
    from paper_2212_02988_gb300 import calibration, state_arrays
    w = synth.ROOM128
    n = 80
    s = synth.Sequence(w, n_frames=n)
    F, _ = make_pair(w, oracle_mod, map_arrays=s.settled_map(), s1_pose=s.pose7(0), vel=s.velocity(0))
    est, covs = [], []
    for i in range(n):
        f = s.frame(i)
        st = state_arrays(F.step(s.imu_window(i) if i else None, w.dt, t(f["depth"]), t(f["rgb"]),
                                 want_state=True))
        est.append(st["pose"])
        covs.append(st["cov"])
    F.close()
    true = np.array([s.pose7(i) for i in range(n)])
    # frame 0 is the given state s_1 (no localisation): calibrate the localised frames
    r = calibration.calibrate(np.array(est[1:]), np.array(covs[1:]), true[1:])
    assert r["rms_translation"] < 0.01 and r["rms_rotation_deg"] < 0.5
    assert np.isfinite(r["scale"]) and r["scale"] > 0
    assert r["whitened"].shape == (n - 1, 6) and np.all(np.isfinite(r["whitened"]))
    np.testing.assert_allclose(np.mean(r["nssr"]), 6.0, rtol=1e-12)   # the ML correction's defining property
    assert r["observed"][0] == 0.0 and r["observed"][-1] == 1.0
    assert np.all(np.diff(r["observed"]) >= 0)
    assert np.all(r["precision"] > 0)
