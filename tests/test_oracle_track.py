"""Pins of the oracle's localisation objective (App. E.3), its Jacobians,
the Laplace covariance (Sec. 4.1) and the Gauss-Newton solve, against
finite differences, the generator's ground-truth poses and closed forms."""
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
    """World-frame left perturbation: t' = t + d[:3], R' = Exp(d[3:]) R."""
    R = Rotation.from_rotvec(d[3:]).as_matrix() @ R_of(pose7)
    return np.concatenate([pose7[:3] + d[:3], quat_wxyz(R)])


@pytest.fixture(scope="module")
def tiny_pair():
    w = synth.tiny(n=32, width=48, height=36, n_prims=6, seed=11, textured=True)
    s = synth.Sequence(w)
    A = s.pose7(2)
    B = perturb(A, np.array([0.02, -0.01, 0.015, 0.01, -0.015, 0.008]))
    a_d, a_rgb = synth.scene.raycast(s.scene, w, R_of(A), A[:3])
    o_d, o_rgb = synth.scene.raycast(s.scene, w, R_of(B), B[:3])
    return w, s, A, B, a_d.astype(np.float32), a_rgb.astype(np.float32), \
        o_d.astype(np.float32), o_rgb.astype(np.float32)


def test_zero_residual_at_identical_pose(oracle_mod, tiny_pair):
    O = oracle_mod
    w, s, A, B, a_d, a_rgb, _, _ = tiny_pair
    p = O.params(w)
    out = O.residuals(p, A, a_d, a_rgb, A, a_d, a_rgb)
    kept = out["kept"] > 0
    assert kept.mean() > 0.6
    assert np.abs(out["r"][kept]).max() < 1e-9
    ne = O.normal_equations(p, A, a_d, a_rgb, A, a_d, a_rgb)
    assert ne["cost"] < 1e-6
    assert np.abs(ne["g"]).max() < 1e-6


def test_jacobians_match_central_differences(oracle_mod, tiny_pair):
    O = oracle_mod
    w, s, A, B, a_d, a_rgb, o_d, o_rgb = tiny_pair
    p = O.params(w)
    base = O.residuals(p, A, a_d, a_rgb, B, o_d, o_rgb)
    h = 1e-6
    checked = 0
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        rp = O.residuals(p, A, a_d, a_rgb, perturb(B, e), o_d, o_rgb)
        rm = O.residuals(p, A, a_d, a_rgb, perturb(B, -e), o_d, o_rgb)
        same = (base["kept"] > 0) & (rp["kept"] > 0) & (rm["kept"] > 0) & \
            np.all(rp["assoc"] == base["assoc"], axis=1) & np.all(rm["assoc"] == base["assoc"], axis=1)
        fd = (rp["r"] - rm["r"]) / (2 * h)
        J = base["J"][:, :, i]
        err = np.abs(fd[same] - J[same])
        scale = np.abs(J[same]) + 1.0
        assert np.all(err <= 2e-4 * scale), (i, err.max())
        checked += same.sum()
    assert checked > 1000


def planar_pair(O, W=40, H=30):
    """Anchor: a plane seen from the identity pose with colour linear in the
    anchor's pixel coordinates; observation: the same plane from pose B with
    colours sampled from that linear field.  Every residual is zero at B and
    smooth around it (bilinear interpolation of a linear field is exact)."""
    w = synth.tiny(width=W, height=H)
    p = O.params(w)
    A = np.array([0, 0, 0, 1.0, 0, 0, 0])
    nrm = np.array([0.1, -0.2, -1.0])
    nrm /= np.linalg.norm(nrm)
    c = -2.0
    u, v = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    ray = np.stack([(u - p.cx) / p.fx, (v - p.cy) / p.fy, np.ones_like(u)], -1)
    lin = lambda uu, vv: np.stack([0.3 + 0.004 * uu + 0.003 * vv, 0.5 - 0.002 * uu + 0.004 * vv,
                                   0.4 + 0.003 * uu - 0.002 * vv], -1)
    a_d = c / (ray @ nrm)
    a_rgb = lin(u, v)
    B = perturb(A, np.array([0.01, -0.02, 0.015, 0.01, 0.008, -0.006]))
    d = ray @ R_of(B).T
    sB = (c - nrm @ B[:3]) / (d @ nrm)
    X = B[:3] + sB[..., None] * d
    up, vp = p.fx * X[..., 0] / X[..., 2] + p.cx, p.fy * X[..., 1] / X[..., 2] + p.cy
    o_rgb = lin(up, vp)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return p, A, B, f(a_d), f(a_rgb), f(sB), f(o_rgb)


def test_laplace_hessian_is_twice_scaled_jtj(oracle_mod):
    """At zero residual, the Hessian of S = sum (r/b)^2 (the L1 terms treated
    as squares, Sec. 4.1 / App. E.3) is exactly 2 J^T J / b^2: compare a
    finite-difference Hessian of S with 2 * Ht."""
    O = oracle_mod
    p, A, B, a_d, a_rgb, o_d, o_rgb = planar_pair(O)
    base = O.residuals(p, A, a_d, a_rgb, B, o_d, o_rgb)
    kept = base["kept"] > 0
    assert kept.mean() > 0.5
    assert np.abs(base["r"][kept]).max() < 1e-5
    bvec = np.array([p.b_geo, p.b_rgb, p.b_rgb, p.b_rgb])
    h = 1e-4
    sel = kept.copy()
    evals = {}
    for i in range(6):
        for j in range(6):
            for si, sj in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                d = np.zeros(6)
                d[i] += si * h
                d[j] += sj * h
                r = O.residuals(p, A, a_d, a_rgb, perturb(B, d), o_d, o_rgb)
                sel &= np.all(r["assoc"] == base["assoc"], axis=1) & (r["kept"] > 0)
                evals[(i, j, si, sj)] = r["r"]
    assert sel.sum() > 0.8 * kept.sum()
    S = lambda r: np.sum(((r / bvec) ** 2)[sel])
    Hfd = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            Hfd[i, j] = sum(si * sj * S(evals[(i, j, si, sj)])
                            for si, sj in ((1, 1), (1, -1), (-1, 1), (-1, -1))) / (4 * h * h)
    Jk = base["J"][sel] / bvec[None, :, None]
    Ht_sel = np.einsum("nki,nkj->ij", Jk, Jk)
    np.testing.assert_allclose(Hfd, 2 * Ht_sel, rtol=1e-3, atol=1e-4 * np.abs(Ht_sel).max())
    # and the oracle's Ht is the same sum over all kept pixels
    Ht = O.normal_equations(p, A, a_d, a_rgb, B, o_d, o_rgb)["Ht"]
    Jall = base["J"][kept] / bvec[None, :, None]
    np.testing.assert_allclose(Ht, np.einsum("nki,nkj->ij", Jall, Jall), rtol=1e-12,
                               atol=1e-12 * np.abs(Ht).max())


def make_prior(O, pose7, cov_pp):
    pr = O.Prior()
    for a in range(3):
        pr.t[a] = pose7[a]
    for a in range(4):
        pr.q[a] = pose7[3 + a]
    prec = np.linalg.inv(cov_pp)
    cov = np.zeros((12, 12))
    cov[:6, :6] = cov_pp
    cov[6:, 6:] = np.eye(6) * 1e-4
    for i in range(36):
        pr.cov_pp[i] = cov_pp.flat[i]
        pr.prec_pp[i] = prec.flat[i]
        pr.D[i] = 0.0
        pr.cov_vel[i] = (np.eye(6) * 1e-4).flat[i]
    for i in range(144):
        pr.cov[i] = cov.flat[i]
    return pr


def test_gauss_newton_recovers_true_pose(oracle_mod):
    """Anchor and observation are exact ray casts of the analytic scene at
    poses A and B; starting 1 cm / 0.5 deg away, the MAP pose lands on B to
    within the bias of nearest-pixel association at this resolution (the
    bias shrinks with resolution: about 3.7 mm at 48x36, 0.8 mm here)."""
    O = oracle_mod
    w = synth.tiny(n=32, width=192, height=144, n_prims=6, seed=11, textured=True)
    s = synth.Sequence(w)
    A = s.pose7(2)
    B = perturb(A, np.array([0.02, -0.01, 0.015, 0.01, -0.015, 0.008]))
    a_d, a_rgb = (x.astype(np.float32) for x in synth.scene.raycast(s.scene, w, R_of(A), A[:3]))
    o_d, o_rgb = (x.astype(np.float32) for x in synth.scene.raycast(s.scene, w, R_of(B), B[:3]))
    p = O.params(w)
    start = perturb(B, np.array([0.008, 0.006, -0.007, 0.006, -0.004, 0.005]))
    cov_pp = np.diag([0.05 ** 2] * 3 + [0.02 ** 2] * 3)
    pr = make_prior(O, start, cov_pp)
    prev = O.make_state(A)
    out, diag = O.localise(p, pr, prev, a_d, a_rgb, o_d, o_rgb)
    est = O.state_arrays(out)["pose"]
    assert np.linalg.norm(est[:3] - B[:3]) < 1.5e-3
    ang = np.linalg.norm(Rotation.from_matrix(R_of(est) @ R_of(B).T).as_rotvec())
    assert np.degrees(ang) < 0.15
    # the prior pulled from 1 cm away; the data term moved it almost all the way
    assert np.linalg.norm(start[:3] - B[:3]) > 8 * np.linalg.norm(est[:3] - B[:3])


def test_prior_only_returns_prior(oracle_mod, tiny_pair):
    """No valid pixel: the optimum is the prior mean, the Laplace covariance
    is the prior covariance, and the recombined joint equals the propagated
    joint (the pose is unobserved)."""
    O = oracle_mod
    w, s, A, B, a_d, a_rgb, o_d, o_rgb = tiny_pair
    p = O.params(w)
    s0 = O.make_state(A, vel6=np.array([0.3, -0.1, 0.05, 0.1, 0.2, -0.3]),
                      cov=np.diag([1e-4] * 3 + [1e-5] * 3 + [1e-3] * 6))
    pr = O.predict(p, s0, s.imu_window(3), w.dt)
    empty = np.zeros_like(o_d)
    out, diag = O.localise(p, pr, s0, a_d, a_rgb, empty, o_rgb)
    pa, oa = O.prior_arrays(pr), O.state_arrays(out)
    assert diag["n_pixels"] == 0
    np.testing.assert_allclose(oa["pose"], pa["pose"], atol=1e-14)
    np.testing.assert_allclose(oa["vel"], pa["vel"], atol=1e-14)
    np.testing.assert_allclose(oa["cov"], pa["cov"], rtol=1e-9, atol=1e-15)
