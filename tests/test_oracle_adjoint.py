"""Pins of the oracle's render adjoint (App. B: the emission is
differentiable) against central finite differences of the oracle's forward
render, step 1e-4, on a smooth random scene."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth


def quat_wxyz(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def R_of(pose7):
    w, x, y, z = pose7[3:]
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def perturb(pose7, d):
    R = Rotation.from_rotvec(d[3:]).as_matrix() @ R_of(pose7)
    return np.concatenate([pose7[:3] + d[:3], quat_wxyz(R)])


@pytest.fixture(scope="module")
def scene(oracle_mod):
    O = oracle_mod
    n, extent = 24, 2.4
    w = synth.tiny(n=n, width=40, height=30)
    p = O.params(w)
    p.voxel = extent / n
    for a in range(3):
        p.origin[a] = -0.5 * extent
    p.eps = 0.4 * p.voxel
    p.fx = p.fy = 30.0
    p.cx, p.cy = 19.5, 14.5
    c = p.origin[0] + (np.arange(n) + 0.5) * p.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    rng = np.random.default_rng(12)
    occ = -0.4 * np.ones((n, n, n))
    for _ in range(5):
        ctr = rng.uniform(-0.6, 0.6, 3)
        occ = np.maximum(occ, rng.uniform(0.25, 0.45) - np.sqrt((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 +
                                                                 (Z - ctr[2]) ** 2))
    rgb = np.stack([0.5 + 0.3 * np.sin(3 * X + 1), 0.5 + 0.3 * np.cos(2 * Y - Z), 0.4 + 0.2 * np.sin(X * Y * 4)],
                   -1)
    R0 = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    pose = np.concatenate([[-1.05, 0.03, -0.02], quat_wxyz(Rotation.from_euler("zyx", [0.15, 0.05, -0.08]).as_matrix() @ R0)])
    gD = rng.normal(size=(p.height, p.width))
    gC = rng.normal(size=(p.height, p.width, 3))
    return O, p, occ, rgb, pose, gD, gC


def loss(O, p, occ, rgb, pose, gD, gC):
    r = O.render(p, occ, rgb, pose)
    return float(np.sum(gD * r["depth"]) + np.sum(gC * r["rgb"]))


def test_map_gradients_match_central_differences(scene):
    O, p, occ, rgb, pose, gD, gC = scene
    g = O.render_backward(p, occ, rgb, pose, gD, gC)
    assert np.abs(g["occ"]).max() > 0 and np.abs(g["rgb"]).max() > 0
    h = 1e-4
    rng = np.random.default_rng(3)
    nz = np.argwhere(np.abs(g["occ"]) > 1e-3 * np.abs(g["occ"]).max())
    pick = nz[rng.choice(len(nz), 25, replace=False)]
    bad = 0
    for idx in map(tuple, pick):
        op, om = occ.copy(), occ.copy()
        op[idx] += h
        om[idx] -= h
        fd = (loss(O, p, op, rgb, pose, gD, gC) - loss(O, p, om, rgb, pose, gD, gC)) / (2 * h)
        if abs(fd - g["occ"][idx]) > 1e-3 * abs(g["occ"][idx]) + 1e-6:
            bad += 1
    assert bad <= 1          # a hit index may flip inside +-h at a kink
    nzc = np.argwhere(np.abs(g["rgb"]) > 1e-3 * np.abs(g["rgb"]).max())
    for idx in map(tuple, nzc[rng.choice(len(nzc), 15, replace=False)]):
        rp, rm = rgb.copy(), rgb.copy()
        rp[idx] += h
        rm[idx] -= h
        fd = (loss(O, p, occ, rp, pose, gD, gC) - loss(O, p, occ, rm, pose, gD, gC)) / (2 * h)
        assert fd == pytest.approx(g["rgb"][idx], rel=1e-6, abs=1e-9)   # colour enters linearly


def test_pose_gradient_matches_central_differences(scene):
    """Per pose direction, over the rays whose hit keeps its sample index at
    +h, 0 and -h (a ray crossing a silhouette jumps to the background or to a
    surface behind, which no gradient represents, and a ray whose bracketing
    pair of samples changes has a kink in its depth).  Sample positions are FP32
    (the traversal recipe), which limits the quotient at h = 1e-4 to about
    1e-3 relative."""
    O, p, occ, rgb, pose, gD, gC = scene
    h = 1e-4
    r0 = O.render(p, occ, rgb, pose)
    m0, k0 = r0["mask"], r0["hitk"]
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        rp = O.render(p, occ, rgb, perturb(pose, e))
        rm = O.render(p, occ, rgb, perturb(pose, -e))
        stable = (rp["mask"] == m0) & (rm["mask"] == m0) & (rp["hitk"] == k0) & \
            (rm["hitk"] == k0)
        assert stable.mean() > 0.95
        gd, gc = gD * stable, gC * stable[..., None]
        fd = (np.sum(gd * (rp["depth"] - rm["depth"])) + np.sum(gc * (rp["rgb"] - rm["rgb"]))) / (2 * h)
        g = O.render_backward(p, occ, rgb, pose, gd, gc)["pose"][i]
        assert g == pytest.approx(fd, rel=1e-2, abs=1e-3), (i, g, fd)
