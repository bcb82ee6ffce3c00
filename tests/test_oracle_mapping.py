"""Pins of the oracle's gradient-descent mapping (the alternative to the
closed-form map update, Sec. 4.4, Fig. sdfvsvi): a rendering loss over
frames with known poses, its gradient carried to the map means by the render
adjoint (App. B), and plain descent steps.

  * observations rendered from the map itself: the data term and its
    gradient vanish, only the App. B prior remains;
  * the loss is quadratic in the colour means (the hit decisions depend on
    occupancy only), so central differences along a colour direction equal
    the gradient's projection up to rounding;
  * on a linear occupancy field (a wall) the depth is smooth in the
    occupancy values, so central differences along an occupancy direction
    match the gradient;
  * descent steps move the wall toward the observed one."""
import numpy as np
import pytest

import synth


def wall_map(w, z_wall, colour=0.4):
    n = w.n
    c = w.origin + (np.arange(n) + 0.5) * w.voxel
    occ = np.broadcast_to((c - z_wall)[:, None, None], (n, n, n)).astype(np.float64).copy()
    rgb = np.full((n, n, n, 3), colour)
    return occ, rgb


@pytest.fixture(scope="module")
def setup(oracle_mod):
    O = oracle_mod
    w = synth.tiny(n=32, width=40, height=30)
    p = O.params(w)
    poses = [np.array([0.05, -0.1, -0.6, 1.0, 0.0, 0.0, 0.0]),
             np.array([-0.2, 0.1, -0.5, 0.995, 0.05, -0.08, 0.0])]
    for q in poses:
        q[3:] /= np.linalg.norm(q[3:])
    return O, w, p, poses


def test_own_renders_leave_only_the_prior(setup):
    O, w, p, poses = setup
    occ, rgb = wall_map(w, 1.1)
    rgb += np.random.default_rng(0).uniform(-0.1, 0.1, rgb.shape)
    obs = [O.render(p, occ, rgb, q) for q in poses]
    loss, go, gr = O.map_loss_grad(p, occ, rgb, poses, [o["depth"] for o in obs], [o["rgb"] for o in obs],
                                   0.02, 0.1)
    v0 = p.prior_var
    np.testing.assert_allclose(go, (occ - p.init_occ) / v0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(gr, rgb / v0, rtol=0, atol=1e-15)
    prior = (np.sum((occ - p.init_occ) ** 2) + np.sum(rgb ** 2)) / (2 * v0)
    assert abs(loss - prior) <= 1e-12 * prior


def test_colour_gradient_is_exact(setup):
    O, w, p, poses = setup
    occ, rgb = wall_map(w, 1.1)
    rng = np.random.default_rng(1)
    obs_rgb = [rng.uniform(0, 1, (w.height, w.width, 3)) for _ in poses]
    obs_d = [O.render(p, occ, rgb, q)["depth"] + 0.01 for q in poses]
    loss, go, gr = O.map_loss_grad(p, occ, rgb, poses, obs_d, obs_rgb, 0.02, 0.1)
    d = rng.normal(size=rgb.shape)
    h = 1e-3
    lp = O.map_loss_grad(p, occ, rgb + h * d, poses, obs_d, obs_rgb, 0.02, 0.1)[0]
    lm = O.map_loss_grad(p, occ, rgb - h * d, poses, obs_d, obs_rgb, 0.02, 0.1)[0]
    fd = (lp - lm) / (2 * h)
    proj = float(np.sum(gr * d))
    assert abs(fd - proj) <= 1e-9 * abs(proj) + 1e-9 * loss
    assert np.count_nonzero(gr - rgb / p.prior_var) > 0


def test_occupancy_gradient_matches_central_differences(setup):
    O, w, p, poses = setup
    occ, rgb = wall_map(w, 1.1)
    obs = [O.render(p, *wall_map(w, 1.13), q) for q in poses]
    args = (poses, [o["depth"] for o in obs], [o["rgb"] for o in obs], 0.02, 0.1)
    loss, go, gr = O.map_loss_grad(p, occ, rgb, *args)
    d = np.random.default_rng(2).normal(size=occ.shape)
    h = 1e-6
    hits = [O.render(p, occ + s * h * d, rgb, q)["hitk"] for s in (1, -1) for q in poses]
    base = [O.render(p, occ, rgb, q)["hitk"] for q in poses]
    assert all(np.array_equal(a, b) for a, b in zip(hits, base + base))   # no hit sample moves
    lp = O.map_loss_grad(p, occ + h * d, rgb, *args)[0]
    lm = O.map_loss_grad(p, occ - h * d, rgb, *args)[0]
    fd = (lp - lm) / (2 * h)
    proj = float(np.sum(go * d))
    assert abs(proj) > 1.0
    assert abs(fd - proj) <= 1e-4 * abs(proj)


def test_descent_moves_the_wall_toward_the_observation(setup):
    O, w, p, poses = setup
    occ, rgb = wall_map(w, 1.1)
    obs = [O.render(p, *wall_map(w, 1.13), q) for q in poses]
    depths, rgbs = [o["depth"] for o in obs], [o["rgb"] for o in obs]
    losses = []
    for _ in range(15):
        occ, rgb, loss = O.map_descent(p, occ, rgb, poses, depths, rgbs, 0.02, 0.1, 1e-5, 1e-4)
        losses.append(loss)
    assert losses[-1] < 0.2 * losses[0]
    r = O.render(p, occ, rgb, poses[0])
    m = (r["mask"] > 0) & (obs[0]["mask"] > 0)
    gap0 = np.mean(np.abs(O.render(p, *wall_map(w, 1.1), poses[0])["depth"][m] - obs[0]["depth"][m]))
    assert np.mean(np.abs(r["depth"][m] - obs[0]["depth"][m])) < 0.5 * gap0
