"""State-uncertainty calibration (App. G) of the GPU filter's own output on a
synthetic trajectory with known true poses: the filter steps through the
C ABI, the states come back each frame, and the analysis whitens the pose
residuals by the filter's pose covariances.  The same analysis of the FP64
oracle's filter on the same frames gives the same correction and curve: the
over-confidence the correction measures belongs to the method as read (the
Laplace covariance of per-pixel independent residuals), not to the kernels."""
import numpy as np
import pytest

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu

N = 60   # frames of room128_320x240 from its settled map (free-running parity holds over them)


@pytest.fixture(scope="module")
def histories(oracle_mod):
    from paper_2212_02988_gb300 import state_arrays
    O = oracle_mod
    w = synth.ROOM128
    s = synth.Sequence(w, n_frames=max(N, w.n_frames))
    m = s.settled_map()
    F, p = make_pair(w, O, map_arrays=m, s1_pose=s.pose7(0), vel=s.velocity(0))
    OF = O.Filter(p, m, O.make_state(s.pose7(0), s.velocity(0)))
    gpu, ora = ([], []), ([], [])
    for i in range(N):
        f = s.frame(i)
        imu = s.imu_window(i) if i else None
        st = state_arrays(F.step(imu, w.dt, t(f["depth"]), t(f["rgb"]), want_state=True))
        so = O.state_arrays(OF.step(f["depth"], f["rgb"], imu, w.dt))
        for h, x in ((gpu, st), (ora, so)):
            h[0].append(x["pose"])
            h[1].append(x["cov"])
    F.close()
    true = np.array([s.pose7(i) for i in range(N)])
    # frame 0 is the given state s_1 (no localisation): the localised frames only
    return ({"est": np.array(gpu[0][1:]), "cov": np.array(gpu[1][1:])},
            {"est": np.array(ora[0][1:]), "cov": np.array(ora[1][1:])}, true[1:])


def test_calibration_of_the_filter_on_a_synthetic_trajectory(histories):
    from paper_2212_02988_gb300 import calibration
    g, _, true = histories
    r = calibration.calibrate(g["est"], g["cov"], true)
    n = len(true)
    assert r["rms_translation"] < 0.02 and r["rms_rotation_deg"] < 0.5
    assert np.isfinite(r["scale"]) and r["scale"] > 0
    assert r["whitened"].shape == (n, 6) and np.all(np.isfinite(r["whitened"]))
    np.testing.assert_allclose(np.mean(r["nssr"]), 6.0, rtol=1e-12)   # the ML correction's defining property
    assert r["observed"][0] == 0.0 and r["observed"][-1] == 1.0
    assert np.all(np.diff(r["observed"]) >= 0)
    assert np.all(r["precision"] > 0)


def test_oracle_states_calibrate_the_same(histories):
    """The oracle's states give the GPU filter's maximum-likelihood
    correction within 5 % and the same calibration curve within two frames
    per level.  (The poses agree within 1 mm and the covariances within 1e-3
    relative, tests/test_gpu_horizon.py; a frame's NSSR moves by at most a
    few per cent with that, and so does their mean.)"""
    from paper_2212_02988_gb300 import calibration
    g, o, true = histories
    rg = calibration.calibrate(g["est"], g["cov"], true)
    ro = calibration.calibrate(o["est"], o["cov"], true)
    print(f"\nml scale: GPU {rg['scale']:.1f}, oracle {ro['scale']:.1f}; "
          f"rms {1e3 * rg['rms_translation']:.2f} / {1e3 * ro['rms_translation']:.2f} mm")
    assert rg["scale"] == pytest.approx(ro["scale"], rel=0.05)
    n = len(true)
    assert np.all(np.abs(rg["observed"] - ro["observed"]) <= 2.0 / n + 1e-12)
    # with the oracle's own correction, the GPU's frames fall on the oracle's curve
    rx = calibration.calibrate(g["est"], g["cov"], true, scale=ro["scale"])
    assert np.all(np.abs(rx["observed"] - ro["observed"]) <= 2.0 / n + 1e-12)
