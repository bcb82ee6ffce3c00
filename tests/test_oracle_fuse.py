"""Pins of the oracle's map update (App. D, Eq. mapupdategauss): the
recursive Gaussian product against the batch Curless-Levoy weighted average,
the frustum/truncation rule against an independent FP64 restatement, and
invariants (untouched voxels, non-increasing variance)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth


def R_of(q):
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


@pytest.fixture(scope="module")
def fused(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    p = O.params(w)
    pose = s.pose7(5)
    clean_d, clean_rgb = s.clean_frame(5)
    rng = np.random.default_rng(21)
    frames = []
    for k in range(4):
        d = (clean_d + rng.normal(0, w.depth_sigma, clean_d.shape)).astype(np.float32)
        c = (clean_rgb + rng.normal(0, w.rgb_sigma, clean_rgb.shape)).astype(np.float32)
        frames.append((d, c))
    m0 = O.map64(*s.prior_map())
    m = {k: v.copy() for k, v in m0.items()}
    counts = [O.fuse(p, m, pose, d, c) for d, c in frames]
    return O, w, s, p, pose, frames, m0, m, counts


def projective_sdf(p, pose, depth, mask):
    """FP64 restatement of the update rule: per voxel centre, camera-frame
    z, nearest pixel, sdf = D - z; returns sdf (nan where not updated) and
    the distance of each deciding quantity to its threshold."""
    n = p.nx
    c = p.origin[0] + (np.arange(n) + 0.5) * p.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    Pw = np.stack([X, Y, Z], -1).reshape(-1, 3)
    R = R_of(pose[3:])
    Xc = (Pw - pose[:3]) @ R
    z = Xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = p.fx * Xc[:, 0] / z + p.cx
        v = p.fy * Xc[:, 1] / z + p.cy
    iu, iv = np.floor(u + 0.5), np.floor(v + 0.5)
    ok = (z > 0) & (iu >= 0) & (iu <= p.width - 1) & (iv >= 0) & (iv <= p.height - 1)
    iu = np.where(ok, iu, 0).astype(int)
    iv = np.where(ok, iv, 0).astype(int)
    ok &= mask[iv, iu] > 0
    sdf = np.where(ok, depth[iv, iu].astype(np.float64) - z, np.nan)
    upd = ok & (sdf >= -p.trunc)
    margin = np.minimum.reduce([np.abs(u + 0.5 - np.round(u + 0.5)), np.abs(v + 0.5 - np.round(v + 0.5)),
                                np.abs(np.nan_to_num(sdf, nan=1.0) + p.trunc),
                                np.abs(np.abs(np.nan_to_num(sdf, nan=1.0)) - p.trunc)])
    return np.where(upd, sdf, np.nan), margin, ok


def test_recursive_product_equals_batch_weighted_average(fused):
    """n updates with sigma_update = 1 on the prior: the posterior mean is the
    Curless-Levoy weighted average (Lambda0 mu0 + sum f_i) / (Lambda0 + n) and
    the precision Lambda0 + n (App. D)."""
    O, w, s, p, pose, frames, m0, m, counts = fused
    L0 = 1.0 / p.prior_var
    num_o = L0 * m0["occ"].ravel().copy()
    den_o = np.full(num_o.shape, L0)
    num_c = L0 * m0["rgb"].reshape(-1, 3).copy()
    den_c = np.full(num_o.shape, L0)
    robust = np.ones(num_o.shape, bool)
    n_upd_ref = []
    for d, c in frames:
        mask = O.depth_mask(p, d)
        sdf, margin, ok = projective_sdf(p, pose, d, mask)
        robust &= margin > 1e-5
        upd = ~np.isnan(sdf)
        n_upd_ref.append(upd.sum())
        f = -np.clip(sdf, -p.trunc, p.trunc)
        num_o[upd] += f[upd]
        den_o[upd] += 1.0
        col = upd & (np.abs(sdf) <= p.trunc)
        # colour of the nearest pixel
        n = p.nx
        cc = p.origin[0] + (np.arange(n) + 0.5) * p.voxel
        Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
        Xc = (np.stack([X, Y, Z], -1).reshape(-1, 3) - pose[:3]) @ R_of(pose[3:])
        with np.errstate(divide="ignore", invalid="ignore"):
            iu = np.floor(p.fx * Xc[:, 0] / Xc[:, 2] + p.cx + 0.5)
            iv = np.floor(p.fy * Xc[:, 1] / Xc[:, 2] + p.cy + 0.5)
        iu = np.where(col, iu, 0).astype(int)
        iv = np.where(col, iv, 0).astype(int)
        num_c[col] += c[iv[col], iu[col]]
        den_c[col] += 1.0
    occ = m["occ"].ravel()
    np.testing.assert_allclose(occ[robust], (num_o / den_o)[robust], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(m["var_occ"].ravel()[robust], (1.0 / den_o)[robust], rtol=1e-12)
    rgb = m["rgb"].reshape(-1, 3)
    np.testing.assert_allclose(rgb[robust], (num_c / den_c[:, None])[robust], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(m["var_rgb"].ravel()[robust], (1.0 / den_c)[robust], rtol=1e-12)
    assert robust.mean() > 0.99
    for got, ref in zip(counts, n_upd_ref):
        assert abs(got - ref) <= 0.001 * ref + 2
    assert min(counts) > 1000


def test_untouched_voxels_and_variance(fused):
    O, w, s, p, pose, frames, m0, m, counts = fused
    changed = m["var_occ"] != m0["var_occ"]
    same = ~changed
    assert np.array_equal(m["occ"][same], m0["occ"][same])
    assert np.all(m["var_occ"] <= m0["var_occ"])
    assert np.all(m["var_rgb"] <= m0["var_rgb"])
    # voxels behind the camera are never updated
    n = p.nx
    c = p.origin[0] + (np.arange(n) + 0.5) * p.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    z = ((np.stack([X, Y, Z], -1) - pose[:3]) @ R_of(pose[3:]))[..., 2]
    assert not np.any(changed & (z < 0))
