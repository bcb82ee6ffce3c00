"""Pins of the oracle's paper-literal pose optimiser (App. F.2, "Pose
optimisation": Adam with momentum off, 1000 steps of 200 uniformly drawn
pixels, step sizes 1e-3 / 3.6e-4): its pixel generator against SplitMix64's
published outputs, the Adam update against its closed form on the first
step, exact fixed points, and the generator's ground-truth pose."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from test_oracle_track import R_of, make_prior, perturb


def test_generator_reproduces_splitmix64(oracle_mod):
    """SplitMix64 (Steele, Lea and Flood 2014) started at state 0: the first
    three outputs published with its reference implementation."""
    O = oracle_mod
    assert [O.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                      0x06C45D188009454F]


def test_pixel_draws_are_uniform_and_in_range(oracle_mod):
    O = oracle_mod
    for n in (1, 7, 4800, 307200):
        draws = [O.sample_pixel(99, i, n) for i in range(2000)]
        assert min(draws) >= 0 and max(draws) < n
    counts = np.bincount([O.sample_pixel(3, i, 7) for i in range(70000)], minlength=7)
    chi2 = ((counts - 10000.0) ** 2 / 10000.0).sum()
    assert chi2 < 27.9                                # 6 degrees of freedom, 0.01 % tail


@pytest.fixture(scope="module")
def case():
    """Anchor at A, observation at B (exact ray casts of the analytic scene),
    prior mean 1.2 cm / 0.6 deg away from B."""
    w = synth.tiny(n=32, width=96, height=72, n_prims=6, seed=11, textured=True)
    s = synth.Sequence(w)
    A = s.pose7(2)
    B = perturb(A, np.array([0.02, -0.01, 0.015, 0.01, -0.015, 0.008]))
    a_d, a_rgb = (x.astype(np.float32) for x in synth.scene.raycast(s.scene, w, R_of(A), A[:3]))
    o_d, o_rgb = (x.astype(np.float32) for x in synth.scene.raycast(s.scene, w, R_of(B), B[:3]))
    start = perturb(B, np.array([0.008, 0.006, -0.007, 0.006, -0.004, 0.005]))
    cov_pp = np.diag([0.05 ** 2] * 3 + [0.02 ** 2] * 3)
    return w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp


def pose_of(start, xi):
    R = Rotation.from_rotvec(xi[3:]).as_matrix() @ R_of(start)
    return start[:3] + xi[:3], R


def test_adam_stays_put_without_pixels(oracle_mod, case):
    """No valid pixel: the gradient is the prior's L xi, 0 at xi = 0, and
    Adam's step lr g / (sqrt(v_hat) + eps) is exactly 0 at every step."""
    O = oracle_mod
    w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp = case
    p = O.params(w, adam_steps=50)
    xi, tr = O.adam(p, make_prior(O, start, cov_pp), A, a_d, a_rgb, np.zeros_like(o_d), o_rgb, 0, trace=True)
    assert not np.any(tr)


def test_adam_hovers_at_the_optimum(oracle_mod, case):
    """Observation = anchor and prior mean = the anchor's pose: the residuals
    are FP64 rounding (~1e-14) and their L1 subgradient is noise, which Adam
    normalises into steps of about its step size; the iterate stays within a
    few of them of xi = 0."""
    O = oracle_mod
    w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp = case
    p = O.params(w, adam_steps=300)
    xi, tr = O.adam(p, make_prior(O, A, cov_pp), A, a_d, a_rgb, a_d, a_rgb, 0, trace=True)
    assert np.abs(tr[:, :3]).max() < 5 * 1e-3          # 1.6 mm seen
    assert np.abs(tr[:, 3:]).max() < 5 * 3.6e-4        # 0.97 mrad seen


def test_first_step_moves_each_component_by_its_step_size(oracle_mod, case):
    """Step 1 has v = (1 - beta2) g^2 and v_hat = g^2, so xi_1 = -lr g / (|g| + eps):
    every component with |g| >> eps moves by exactly its step size."""
    O = oracle_mod
    w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp = case
    p = O.params(w, adam_steps=1)
    xi = O.adam(p, make_prior(O, start, cov_pp), A, a_d, a_rgb, o_d, o_rgb, 0)
    np.testing.assert_allclose(np.abs(xi), [1e-3] * 3 + [3.6e-4] * 3, rtol=1e-9)


def test_adam_lands_near_the_true_pose(oracle_mod, case):
    """From 1.2 cm / 0.6 deg away, 1000 steps end near B.  Adam's steps do not
    shrink (each moves a component by about its step size once v_hat tracks
    g^2), so the iterate hovers within a few step sizes of the optimum; the
    Gauss-Newton passes reach 0.8 mm on the same kind of case."""
    O = oracle_mod
    w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp = case
    p = O.params(w)
    xi, tr = O.adam(p, make_prior(O, start, cov_pp), A, a_d, a_rgb, o_d, o_rgb, 0, trace=True)
    t, R = pose_of(start, xi)
    assert np.linalg.norm(t - B[:3]) < 8e-3
    assert np.degrees(np.linalg.norm(Rotation.from_matrix(R @ R_of(B).T).as_rotvec())) < 0.5
    late = [np.linalg.norm(start[:3] + x[:3] - B[:3]) for x in tr[-200:]]
    assert np.mean(late) < 6e-3 < np.linalg.norm(start[:3] - B[:3]) / 2


def test_localise_with_adam_runs_the_same_optimiser(oracle_mod, case):
    """or_localise with optimiser 1 reaches the xi of or_adam with the frame's
    draws (numbered from n_localised x steps x pixels)."""
    O = oracle_mod
    w, A, B, a_d, a_rgb, o_d, o_rgb, start, cov_pp = case
    p = O.params(w, optimiser=1, adam_steps=30)
    pr = make_prior(O, start, cov_pp)
    prev = O.make_state(A, n_localised=3)
    out, diag = O.localise(p, pr, prev, a_d, a_rgb, o_d, o_rgb)
    xi = O.adam(p, pr, A, a_d, a_rgb, o_d, o_rgb, 3 * 30 * 200)
    assert np.array_equal(diag["xi"], xi)
    assert O.state_arrays(out)["n_localised"] == 4
