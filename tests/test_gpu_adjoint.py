"""GPU parity of the render adjoint (App. B, differentiable emission) with
the FP64 oracle's adjoint and with central finite differences (step 1e-4) of
the GPU forward, and through the torch.autograd.Function.

Bars: per-voxel gradients within 1e-4 of the largest gradient magnitude
plus 1e-3 relative (FP32 values and atomics against FP64); the pose
gradient within 1e-3 relative of its norm against the oracle, 2 % against
the differences (FP32 forward outputs)."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import synth
from gpu_helpers import make_pair, t

pytestmark = pytest.mark.gpu


def quat_wxyz(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def R_of(pose7):
    w, x, y, z = pose7[3:]
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def perturb(pose7, d):
    R = Rotation.from_rotvec(d[3:]).as_matrix() @ R_of(pose7)
    return np.concatenate([pose7[:3] + d[:3], quat_wxyz(R)])


def check_grads(got, ref, name):
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-4 * scale + 1e-3 * np.abs(ref)), (name, err.max() / scale)


def adjoint_pair(O, w, m, pose, rng):
    F, p = make_pair(w, O, map_arrays=m)
    gD = rng.normal(size=(w.height, w.width)).astype(np.float32)
    gC = rng.normal(size=(w.height, w.width, 3)).astype(np.float32)
    n = w.n
    go = torch.zeros((n, n, n), device="cuda")
    gr = torch.zeros((n, n, n, 3), device="cuda")
    g6, g7 = F.render_backward(pose, t(gD), t(gC), go, gr)
    ref = O.render_backward(p, m[0], m[1], pose, gD, gC)
    return F, p, gD, gC, go.cpu().numpy(), gr.cpu().numpy(), g6, ref


@pytest.mark.parametrize("name,frame", [("room64_80x60", 7), ("room128_320x240", 20)])
def test_adjoint_matches_oracle(oracle_mod, name, frame):
    O = oracle_mod
    w = synth.PRESETS[name]
    s = synth.Sequence(w)
    m = s.settled_map()
    F, p, gD, gC, go, gr, g6, ref = adjoint_pair(O, w, m, s.pose7(frame), np.random.default_rng(frame))
    check_grads(go, ref["occ"], "occ")
    check_grads(gr, ref["rgb"], "rgb")
    assert np.linalg.norm(g6 - ref["pose"]) <= 1e-3 * np.linalg.norm(ref["pose"])
    F.close()


def test_adjoint_full_size(oracle_mod):
    """The 256^3 / 640x480 workload: pose gradient and the voxel gradients."""
    O = oracle_mod
    w = synth.ROOM256
    s = synth.Sequence(w, n_frames=4)
    m = s.settled_map()
    F, p, gD, gC, go, gr, g6, ref = adjoint_pair(O, w, m, s.pose7(2), np.random.default_rng(1))
    assert np.linalg.norm(g6 - ref["pose"]) <= 1e-3 * np.linalg.norm(ref["pose"])
    check_grads(go, ref["occ"], "occ")
    check_grads(gr, ref["rgb"], "rgb")
    F.close()


def test_adjoint_matches_finite_differences(oracle_mod):
    O = oracle_mod
    w = synth.ROOM64
    s = synth.Sequence(w)
    occ, rgb, vo, vr = s.settled_map()
    F, _ = make_pair(w, O, map_arrays=(occ, rgb, vo, vr))
    pose = s.pose7(11)
    rng = np.random.default_rng(2)
    gD = rng.normal(size=(w.height, w.width)).astype(np.float32)
    gC = rng.normal(size=(w.height, w.width, 3)).astype(np.float32)
    n = w.n
    go = torch.zeros((n, n, n), device="cuda")
    g6, _ = F.render_backward(pose, t(gD), t(gC), go, None)
    go = go.cpu().numpy()
    h = 1e-4

    def loss(pz, mask=None):
        o = F.render(pz)
        d, c = o["depth"].cpu().double().numpy(), o["rgb"].cpu().double().numpy()
        wd, wc = (gD, gC) if mask is None else (gD * mask, gC * mask[..., None])
        return float(np.sum(wd * d) + np.sum(wc * c)), o

    # voxel values
    nz = np.argwhere(np.abs(go) > 1e-2 * np.abs(go).max())
    bad = 0
    for idx in map(tuple, nz[rng.choice(len(nz), 12, replace=False)]):
        op, om = occ.copy(), occ.copy()
        op[idx] += h
        om[idx] -= h
        F.map_load(t(op), None)
        lp, _ = loss(pose)
        F.map_load(t(om), None)
        lm, _ = loss(pose)
        fd = (lp - lm) / (2 * h)
        bad += abs(fd - go[idx]) > 2e-2 * abs(go[idx]) + 1e-3 * np.abs(go).max()
    F.map_load(t(occ), None)
    assert bad <= 1
    # pose, over rays that keep their hit sample at +-h
    _, o0 = loss(pose)
    k0 = o0["hitk"].cpu().numpy()
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        op, om = F.render(perturb(pose, e)), F.render(perturb(pose, -e))
        stable = (op["hitk"].cpu().numpy() == k0) & (om["hitk"].cpu().numpy() == k0)
        lp, _ = loss(perturb(pose, e), stable)
        lm, _ = loss(perturb(pose, -e), stable)
        fd = (lp - lm) / (2 * h)
        gs, _ = F.render_backward(pose, t((gD * stable).astype(np.float32)),
                                  t((gC * stable[..., None]).astype(np.float32)), None, None)
        assert gs[i] == pytest.approx(fd, rel=2e-2, abs=2e-3 * np.abs(g6).max()), (i, gs[i], fd)
    F.close()


def test_autograd_function(oracle_mod):
    from paper_2212_02988_gb300.autograd import render
    w = synth.ROOM64
    s = synth.Sequence(w)
    occ, rgb, vo, vr = s.settled_map()
    F, _ = make_pair(w, oracle_mod, map_arrays=(occ, rgb, vo, vr))
    pose = torch.tensor(s.pose7(5) * np.array([1, 1, 1, 1.3, 1.3, 1.3, 1.3]), dtype=torch.float64,
                        requires_grad=True)   # an unnormalised quaternion on purpose
    occ_t = t(occ).requires_grad_(True)
    rgb_t = t(rgb).requires_grad_(True)
    rng = np.random.default_rng(0)
    gD, gC = t(rng.normal(size=(w.height, w.width)).astype(np.float32)), \
        t(rng.normal(size=(w.height, w.width, 3)).astype(np.float32))
    d, c = render(pose, occ_t, rgb_t, F)
    (d * gD).sum().add((c * gC).sum()).backward()
    go = torch.zeros_like(occ_t)
    gr = torch.zeros_like(rgb_t)
    g6, g7 = F.render_backward(pose.detach().numpy(), gD, gC, go, gr)
    # two runs of the atomics-based scatter agree to FP32 summation order
    check_grads(occ_t.grad.cpu().numpy(), go.cpu().numpy(), "occ")
    check_grads(rgb_t.grad.cpu().numpy(), gr.cpu().numpy(), "rgb")
    np.testing.assert_allclose(pose.grad.numpy(), g7, rtol=1e-5, atol=1e-6 * np.abs(g7).max())
    # the quaternion gradient is the rotation gradient pulled back through
    # q -> R(q / |q|): central differences in q over rays keeping their hit sample
    h = 1e-4
    base = pose.detach().numpy()
    k0 = F.render(base)["hitk"]
    for j in range(4):
        e = np.zeros(7)
        e[3 + j] = h
        op, om = F.render(base + e), F.render(base - e)
        st = ((op["hitk"] == k0) & (om["hitk"] == k0)).float()
        wd, wc = gD * st, gC * st[..., None]
        fd = float(((op["depth"] - om["depth"]) * wd).sum() + ((op["rgb"] - om["rgb"]) * wc).sum()) / (2 * h)
        _, gm = F.render_backward(base, wd.contiguous(), wc.contiguous(), None, None)
        assert gm[3 + j] == pytest.approx(fd, rel=2e-2, abs=2e-3 * np.abs(g7[3:]).max()), (j, gm[3 + j], fd)
    F.close()


def test_autograd_loads_the_map_only_when_it_changed(oracle_mod):
    """A forward and its backward load the map once; an in-place update of
    the map tensors, or another map in the filter, makes the next forward
    load it again."""
    from paper_2212_02988_gb300.autograd import render
    w = synth.ROOM64
    s = synth.Sequence(w)
    occ, rgb, vo, vr = s.settled_map()
    F, _ = make_pair(w, oracle_mod, map_arrays=(occ, rgb, vo, vr))
    loads = []
    load = F.map_load
    F.map_load = lambda *a, **k: (loads.append(1), load(*a, **k))[1]
    pose = torch.tensor(s.pose7(5), dtype=torch.float64)
    occ_t = t(occ).requires_grad_(True)
    rgb_t = t(rgb).requires_grad_(True)
    first = None
    for it in range(3):
        d, c = render(pose, occ_t, rgb_t, F)
        (d.sum() + c.sum()).backward()
        assert len(loads) == it + 1
        if first is None:
            first = occ_t.grad.clone()
        with torch.no_grad():
            occ_t.sub_(1e-6 * torch.sign(occ_t.grad))   # an in-place step: the next forward reloads
        occ_t.grad = None
        rgb_t.grad = None
    F.map_load(t(occ), t(rgb))                           # another map in the filter
    d, c = render(pose, occ_t, rgb_t, F)
    assert len(loads) == 5
    # the gradient of the reloaded map is that of a fresh filter holding it
    G, _ = make_pair(w, oracle_mod, map_arrays=(occ_t.detach().cpu().numpy(), rgb, vo, vr))
    o2 = occ_t.detach().clone().requires_grad_(True)
    d2, c2 = render(pose, o2, rgb_t.detach().clone().requires_grad_(True), G)
    assert torch.equal(d, d2) and torch.equal(c, c2)
    assert first.abs().sum() > 0
    F.close()
    G.close()
