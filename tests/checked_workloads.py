"""Small workloads through every kernel family of the library, for the
bounds-check build's test (tests/test_gpu_checked.py).  Run as a script:

    [PRISM_CHECKED=1] python tests/checked_workloads.py OUT.npz

It loads whichever library the environment selects (paper_2212_02988_gb300
_lib: PRISM_CHECKED=1 loads libprism_checked.so), runs filter steps (predict,
localisation, map update, anchor render in the planned tile order), renders
of a ragged image with cameras inside and outside the grid, the render
adjoint, rollouts, a map-descent step and two streams through the server,
and writes every result and each handle's and the server's check word."""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import synth  # noqa: E402
from gpu_helpers import t  # noqa: E402


def random_field(n, seed):
    """A random near-tau occupancy field on an n^3 grid with random colours."""
    w = synth.tiny(n=n, width=83, height=61)
    rng = np.random.default_rng(seed)
    c = w.origin + (np.arange(n) + 0.5) * w.voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    occ = -0.3 * np.ones((n, n, n))
    for _ in range(6):
        ctr = rng.uniform(-1.5, 1.5, 3)
        occ = np.maximum(occ, rng.uniform(0.2, 0.6) - np.sqrt((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 +
                                                              (Z - ctr[2]) ** 2))
    occ = (occ + rng.normal(0, 0.02, occ.shape)).astype(np.float32)
    rgb = rng.uniform(0, 1, (n, n, n, 3)).astype(np.float32)
    return w, occ, rgb


def main(path):
    from paper_2212_02988_gb300 import Filter, _lib, config, make_state, state_arrays
    from paper_2212_02988_gb300.serve import Server
    out = {"checked_build": np.array(_lib.load().prism_checked_build())}
    words = []

    # filter steps from the prior map (the plan orders the anchor render from the second step on)
    for name, storage in (("room64_80x60", "f32"), ("room64_80x60", "bf16"), ("room128_320x240", "f32")):
        w = synth.PRESETS[name]
        s = synth.Sequence(w, n_frames=8)
        F = Filter(config(w.n, w.extent, w.width, w.height, storage=storage), make_state(s.pose7(0), s.velocity(0)),
                   device=0)
        F.map_load(*(t(np.asarray(a, np.float32)) for a in s.prior_map()))
        st = []
        for i in range(6):
            f = s.frame(i)
            st.append(state_arrays(F.step(s.imu_window(i) if i else None, w.dt, t(f["depth"]), t(f["rgb"]),
                                          want_state=True)))
        key = f"{name}_{storage}"
        out[f"{key}_pose"] = np.array([x["pose"] for x in st])
        out[f"{key}_cov"] = np.array([x["cov"] for x in st])
        m = F.map_store()
        out[f"{key}_occ"] = m["occ"].cpu().numpy()
        r = F.render(s.pose7(6))
        out[f"{key}_hitk"] = r["hitk"].cpu().numpy()
        # rollouts: two sequences of three frames
        wins = [[s.imu_window(i) for i in range(1, 4)], [s.imu_window(i) for i in range(3, 6)]]
        ro = F.rollout(wins, w.dt, hitk=True)
        out[f"{key}_roll_hitk"] = ro["hitk"].cpu().numpy()
        words.append(F.check_status())
        F.close()

    # ragged image, random field, cameras inside and outside the grid; the adjoint
    w, occ, rgb = random_field(24, 9)
    var = np.ones_like(occ)
    F = Filter(config(w.n, w.extent, w.width, w.height), None, device=0)
    F.map_load(t(occ), t(rgb), t(var), t(var))
    poses = [np.array([-1.7, 0.3, 0.1, 0.9, 0.1, -0.2, 0.3]), np.array([5.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]),
             np.array([0.0, 0.0, 0.0, 0.5, -0.5, 0.5, 0.5])]
    for j, p in enumerate(poses):
        r = F.render(p)
        out[f"ragged_hitk{j}"] = r["hitk"].cpu().numpy()
        out[f"ragged_depth{j}"] = r["depth"].cpu().numpy()
    g = torch.Generator(device="cpu").manual_seed(3)
    gd = torch.randn((w.height, w.width), generator=g).cuda()
    gc = torch.randn((w.height, w.width, 3), generator=g).cuda()
    go = torch.zeros((w.n,) * 3, device="cuda")
    gr = torch.zeros((w.n,) * 3 + (3,), device="cuda")
    g6, _ = F.render_backward(poses[0], gd, gc, go, gr)
    out["bwd_pose"] = g6
    out["bwd_occ"] = go.cpu().numpy()
    # one map-descent step over two frames rendered at two poses
    d = torch.stack([F.render(poses[0])["depth"], F.render(poses[2])["depth"]])
    c = torch.stack([F.render(poses[0])["rgb"], F.render(poses[2])["rgb"]])
    out["descent_loss"] = np.array(F.map_descent(np.stack([poses[0], poses[2]]), d, c, 0.02, 0.1, 1e-6, 1e-6))
    words.append(F.check_status())
    F.close()

    # two streams through the server
    specs = []
    for wk, seed in ((synth.tiny(n=32, width=48, height=40), 5), (synth.ROOM64, 6)):
        sq = synth.Sequence(wk, n_frames=5, seed=seed)
        specs.append((wk, sq))
    srv = Server(2 << 30, storage="f32")
    ids = [srv.open(config(wk.n, wk.extent, wk.width, wk.height), make_state(sq.pose7(0), sq.velocity(0)),
                    tuple(t(np.asarray(a, np.float32)) for a in sq.prior_map())) for wk, sq in specs]
    for i in range(4):
        for sid, (wk, sq) in zip(ids, specs):
            f = sq.frame(i)
            srv.submit(sid, sq.imu_window(i) if i else None, wk.dt, t(f["depth"]), t(f["rgb"]), tag=i)
    srv.drain()
    res = sorted(srv.poll(1024), key=lambda r: (r["stream"], r["tag"]))
    out["serve_pose"] = np.array([r["pose"] for r in res])
    words.append(srv.check_status())
    srv.destroy()

    out["words"] = np.array(words, dtype=np.uint64)
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
