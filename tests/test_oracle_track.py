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


PLANE_N = np.array([0.1, -0.2, -1.0]) / np.linalg.norm([0.1, -0.2, -1.0])


def sliding_pair(O, s_world, W=40, H=30):
    """The plane of planar_pair (n . x = -2, n = PLANE_N) seen from the
    identity anchor and from the anchor moved by s_world (no rotation): depth
    images by ray-plane intersection in FP64, colours from the same linear
    field."""
    w = synth.tiny(width=W, height=H)
    p = O.params(w)
    A = np.array([0, 0, 0, 1.0, 0, 0, 0])
    nrm = PLANE_N
    c = -2.0
    u, v = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    ray = np.stack([(u - p.cx) / p.fx, (v - p.cy) / p.fy, np.ones_like(u)], -1)
    lin = lambda uu, vv: np.stack([0.3 + 0.004 * uu + 0.003 * vv, 0.5 - 0.002 * uu + 0.004 * vv,
                                   0.4 + 0.003 * uu - 0.002 * vv], -1)
    a_d = c / (ray @ nrm)
    S = np.concatenate([s_world, [1.0, 0, 0, 0]])
    sS = (c - nrm @ s_world) / (ray @ nrm)
    X = s_world + sS[..., None] * ray
    up, vp = p.fx * X[..., 0] / X[..., 2] + p.cx, p.fy * X[..., 1] / X[..., 2] + p.cy
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return p, A, S, nrm, f(a_d), f(lin(u, v)), f(sS), f(lin(up, vp))


def test_point_to_plane_is_blind_to_sliding(oracle_mod):
    """A planar scene and a camera that slides 10 cm along the plane (App.
    E.3's point-to-plane term <p_hat - X, n_hat>): evaluated at the unmoved
    pose, every kept pixel's geometric residual stays at rounding level
    (both points lie on the plane, whichever anchor pixel X falls on) while
    the colour residuals see the slide; a 5 mm offset along the normal gives
    the same residual of 5 mm at every kept pixel, its sign following the
    offset's; and the translation Jacobian of the geometric residual is the
    unit normal (no in-plane component).  Catches a point-to-point
    distance, a normal taken from the wrong neighbours, and a residual or
    Jacobian off by a scale."""
    O = oracle_mod
    s_world = np.array([0.08, 0.06, 0.0])
    slide = s_world - (s_world @ PLANE_N) * PLANE_N   # along the plane
    p, A, S, nrm, a_d, a_rgb, o_d, o_rgb = sliding_pair(O, slide)
    assert abs(slide @ nrm) < 1e-15 and np.linalg.norm(slide) > 0.09
    # at the true pose every residual vanishes
    true = O.residuals(p, A, a_d, a_rgb, S, o_d, o_rgb)
    kept = true["kept"] > 0
    assert kept.mean() > 0.6
    assert np.abs(true["r"][kept]).max() < 1e-5
    # at the unmoved pose: the geometry cannot see the slide, the colour can
    slid = O.residuals(p, A, a_d, a_rgb, A, o_d, o_rgb)
    ks = slid["kept"] > 0
    assert ks.mean() > 0.5
    assert np.abs(slid["r"][ks, 0]).max() < 1e-5
    assert np.abs(slid["r"][ks, 1:]).max() > 5e-3
    # a pose off the plane by delta along the normal: r_geo = -delta <n, n_hat> everywhere
    for delta in (0.005, -0.005):
        off = O.residuals(p, A, a_d, a_rgb, np.concatenate([slide + delta * nrm, S[3:]]), o_d, o_rgb)
        ko = off["kept"] > 0
        assert ko.mean() > 0.5
        rg = off["r"][ko, 0]
        np.testing.assert_allclose(np.abs(rg), abs(delta), rtol=0, atol=2e-6)
        assert np.all(np.sign(rg) == np.sign(rg[0]))
        if delta > 0:
            sign_pos = np.sign(rg[0])
        else:
            assert np.sign(rg[0]) == -sign_pos
    # the translation Jacobian of r_geo is the (camera-facing) unit normal,
    # to the accuracy of a normal differenced from FP32 depths
    Jt = true["J"][kept, 0, :3]
    np.testing.assert_allclose(np.abs(Jt @ nrm), 1.0, rtol=0, atol=1e-5)
    inplane = np.cross(nrm, [1.0, 0.0, 0.0])
    inplane /= np.linalg.norm(inplane)
    for d in (inplane, np.cross(nrm, inplane)):
        assert np.abs(Jt @ d).max() < 1e-5


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


# ---------------------------------------------------------------------------
# Laplace assembly (Sec. 4.1, App. E.3), EMA (App. F.2) and recombination
# (Sec. 3.3.2), each rebuilt here from its definition: the Jacobians come from
# the oracle's residuals (pinned above by finite differences), the SO(3) left
# Jacobian from finite differences of SciPy's rotations, and everything else
# is numpy linear algebra written from the paper's formulas.

def left_jacobian_fd(phi, h=1e-6):
    """J_l(phi) defined by Exp(phi + d) = Exp(J_l d) Exp(phi) to first order,
    by central differences of SciPy's exponential and logarithm."""
    R0inv = Rotation.from_rotvec(phi).inv()
    J = np.zeros((3, 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        J[:, i] = ((Rotation.from_rotvec(phi + e) * R0inv).as_rotvec()
                   - (Rotation.from_rotvec(phi - e) * R0inv).as_rotvec()) / (2 * h)
    return J


def joint_prior(O, pose7, vel6, seed):
    """A prior in the form the prediction hands to the localisation (App. E.2):
    a random SPD 12x12 joint over (pose, velocity) split into the pose
    marginal and the velocity conditional v | p = vbar + D xi, with
    D = C_vp C_pp^-1 and Sigma_vel = C_vv - D C_pv."""
    rng = np.random.default_rng(seed)
    sd = np.array([0.01, 0.01, 0.01, 0.006, 0.006, 0.006, 0.2, 0.2, 0.2, 0.3, 0.3, 0.3])
    A = rng.normal(size=(12, 12))
    corr = A @ A.T + 12 * np.eye(12)
    corr /= np.sqrt(np.outer(np.diag(corr), np.diag(corr)))
    C = corr * np.outer(sd, sd)
    Cpp, Cvp, Cvv = C[:6, :6], C[6:, :6], C[6:, 6:]
    D = Cvp @ np.linalg.inv(Cpp)
    Svel = Cvv - D @ Cvp.T
    pr = O.Prior()
    for a in range(3):
        pr.t[a] = pose7[a]
        pr.v[a], pr.w[a] = vel6[a], vel6[3 + a]
    for a in range(4):
        pr.q[a] = pose7[3 + a]
    for i in range(144):
        pr.cov[i] = C.flat[i]
    L = np.linalg.inv(Cpp)
    for i in range(36):
        pr.cov_pp[i], pr.prec_pp[i] = Cpp.flat[i], L.flat[i]
        pr.D[i], pr.cov_vel[i] = D.flat[i], Svel.flat[i]
    return pr, {"L": L, "D": D, "Svel": Svel, "vbar": np.asarray(vel6, float)}


@pytest.fixture(scope="module")
def laplace_case(oracle_mod, tiny_pair):
    """One localisation of the tiny textured pair from a prior 6 mm / 0.5 deg
    off the observed pose, so the optimum xi* is far from 0."""
    O = oracle_mod
    w, s, A, B, a_d, a_rgb, o_d, o_rgb = tiny_pair
    p = O.params(w)
    mu = perturb(B, np.array([0.004, -0.003, 0.003, 0.005, -0.006, 0.004]))
    vel = np.array([0.4, -0.2, 0.1, 0.3, -0.1, 0.2])
    pr, parts = joint_prior(O, mu, vel, seed=5)
    return O, p, pr, parts, A, a_d, a_rgb, o_d, o_rgb


def laplace_by_hand(O, p, parts, A, a_d, a_rgb, o_d, o_rgb, pose, xi, factor=2.0, use_Minv=True):
    res = O.residuals(p, A, a_d, a_rgb, pose, o_d, o_rgb)
    kept = res["kept"] > 0
    b = np.array([p.b_geo, p.b_rgb, p.b_rgb, p.b_rgb])
    Js = res["J"][kept] / b[None, :, None]
    Ht = np.einsum("nki,nkj->ij", Js, Js)
    Mi = np.eye(6)
    if use_Minv:
        Mi[3:, 3:] = np.linalg.inv(left_jacobian_fd(xi[3:]))
    return np.linalg.inv(factor * Ht + Mi.T @ parts["L"] @ Mi), Mi, kept.sum()


def test_localise_returns_the_retraction_of_xi(laplace_case):
    """The returned pose is the prior mean moved by the reported optimum
    xi*: t = t_mu + xi_t, R = Exp(xi_theta) R_mu (reading R15's coordinates).
    Catches a retraction on the wrong side (R_mu Exp(xi_theta))."""
    O, p, pr, parts, A, a_d, a_rgb, o_d, o_rgb = laplace_case
    prev = O.make_state(A)
    out, diag = O.localise(p, pr, prev, a_d, a_rgb, o_d, o_rgb)
    est, mu, xi = O.state_arrays(out)["pose"], O.prior_arrays(pr)["pose"], diag["xi"]
    np.testing.assert_allclose(est[:3], mu[:3] + xi[:3], rtol=0, atol=1e-14)
    want = Rotation.from_rotvec(xi[3:]).as_matrix() @ R_of(mu)
    np.testing.assert_allclose(R_of(est), want, rtol=0, atol=1e-12)
    wrong = R_of(mu) @ Rotation.from_rotvec(xi[3:]).as_matrix()
    assert np.abs(wrong - want).max() > 1e-6
    assert np.linalg.norm(xi[3:]) > 3e-3 and diag["n_pixels"] > 500


def test_laplace_covariance_first_frame(laplace_case):
    """First localisation (no EMA): the pose covariance is
    (2 sum J^T J / b^2 + M^-T L M^-1)^-1 at the optimum, M = diag(I, J_l(xi*)).
    Catches: the factor 1 instead of 2 in front of the data term; the prior
    Hessian left in xi coordinates (no M^-1); the prior dropped."""
    O, p, pr, parts, A, a_d, a_rgb, o_d, o_rgb = laplace_case
    prev = O.make_state(A)
    out, diag = O.localise(p, pr, prev, a_d, a_rgb, o_d, o_rgb)
    pose = O.state_arrays(out)["pose"]
    got = O.state_arrays(out)["cov"][:6, :6]
    want, _, n = laplace_by_hand(O, p, parts, A, a_d, a_rgb, o_d, o_rgb, pose, diag["xi"])
    assert n == diag["n_pixels"]
    rel = lambda X: np.abs(X - want).max() / np.abs(want).max()
    tol = 1e-10
    assert rel(got) < tol
    Ht2 = np.linalg.inv(want) - np.linalg.inv(laplace_by_hand(
        O, p, parts, A, a_d, a_rgb, o_d, o_rgb, pose, diag["xi"], factor=0.0)[0])
    slips = {
        "factor 1": laplace_by_hand(O, p, parts, A, a_d, a_rgb, o_d, o_rgb, pose, diag["xi"], factor=1.0)[0],
        "no M^-1": laplace_by_hand(O, p, parts, A, a_d, a_rgb, o_d, o_rgb, pose, diag["xi"], use_Minv=False)[0],
        "no prior": np.linalg.inv(Ht2),
    }
    for name, X in slips.items():
        assert rel(X) > 100 * tol, name


def test_laplace_ema_on_later_frames(laplace_case):
    """A later localisation (n_localised > 0) returns 0.8 Sigma_prev +
    0.2 Sigma_Laplace (App. F.2, EMA coefficient 0.8).  The previous
    covariance is made 50x the Laplace one, so swapped weights (0.2 / 0.8),
    a missing EMA, or an EMA on the precision instead of the covariance all
    miss by far more than rounding."""
    O, p, pr, parts, A, a_d, a_rgb, o_d, o_rgb = laplace_case
    first, diag0 = O.localise(p, pr, O.make_state(A), a_d, a_rgb, o_d, o_rgb)
    lap = O.state_arrays(first)["cov"][:6, :6]
    prev_cov = np.eye(12) * 1e-4
    prev_cov[:6, :6] = 50 * lap + np.diag([1e-6] * 3 + [1e-7] * 3)
    prev = O.make_state(A, cov=prev_cov, n_localised=3)
    out, diag = O.localise(p, pr, prev, a_d, a_rgb, o_d, o_rgb)
    np.testing.assert_array_equal(diag["xi"], diag0["xi"])   # the EMA does not move the optimum
    got = O.state_arrays(out)["cov"][:6, :6]
    want = 0.8 * prev_cov[:6, :6] + 0.2 * lap
    rel = lambda X: np.abs(X - want).max() / np.abs(want).max()
    assert rel(got) < 1e-12
    assert O.state_arrays(out)["n_localised"] == 4
    for X in (0.2 * prev_cov[:6, :6] + 0.8 * lap, lap,
              np.linalg.inv(0.8 * np.linalg.inv(prev_cov[:6, :6]) + 0.2 * np.linalg.inv(lap))):
        assert rel(X) > 1e-3


def test_recombination_of_velocity(laplace_case):
    """Sec. 3.3.2: with v | p = vbar + D xi(p) and xi = xi* + M^-1 delta at
    the optimum, the velocity mean is vbar + D xi*, cov(v, p) = D M^-1 Sigma_p
    and cov(v) = D M^-1 Sigma_p M^-T D^T + Sigma_vel, Sigma_p the returned
    pose covariance.  Catches D used without M^-1, Sigma_vel dropped, and the
    cross block transposed."""
    O, p, pr, parts, A, a_d, a_rgb, o_d, o_rgb = laplace_case
    out, diag = O.localise(p, pr, O.make_state(A), a_d, a_rgb, o_d, o_rgb)
    sa = O.state_arrays(out)
    xi, S = diag["xi"], sa["cov"]
    Sp = S[:6, :6]
    Mi = np.eye(6)
    Mi[3:, 3:] = np.linalg.inv(left_jacobian_fd(xi[3:]))
    D, Svel = parts["D"], parts["Svel"]
    np.testing.assert_allclose(sa["vel"], parts["vbar"] + D @ xi, rtol=0, atol=1e-13)
    cross = D @ Mi @ Sp
    vv = cross @ Mi.T @ D.T + Svel
    rel = lambda X, Y: np.abs(X - Y).max() / np.abs(Y).max()
    tol = 1e-10
    assert rel(S[6:, :6], cross) < tol and rel(S[:6, 6:], cross.T) < tol
    assert rel(S[6:, 6:], vv) < tol
    assert rel(D @ Sp, cross) > 100 * tol                  # M^-1 matters at this xi*
    assert rel(D @ Sp @ D.T + Svel, vv) > 100 * tol
    assert rel(cross @ Mi.T @ D.T, vv) > 100 * tol         # Sigma_vel matters
    assert rel(cross.T, cross) > 100 * tol                 # the block is not symmetric
