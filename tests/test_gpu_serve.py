"""The multi-stream server (include/prism_serve.h) on the GPU.

Each stream's result in the server must be, bit for bit, the result of
prism_step on a single-stream handle with the same configuration and inputs
(the batched kernels run the same device bodies over the same virtual
grids), and therefore the same alone and in any mix of other streams.
Admission by budget: a stream that does not fit waits, with its requests,
until a closed stream's memory is released."""
import time

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import t

pytestmark = pytest.mark.gpu

MiB = 1 << 20


def frames_of(seq, n):
    out = []
    for i in range(n):
        f = seq.frame(i)
        out.append((seq.imu_window(i) if i else None, t(f["depth"]), t(f["rgb"])))
    return out


def stream_spec(w, seed, n_frames, start="prior"):
    from paper_2212_02988_gb300 import config, make_state
    s = synth.Sequence(w, n_frames=max(n_frames, 2) + 1, seed=seed)
    m = s.settled_map() if start == "settled" else s.prior_map()
    return {"w": w, "seq": s, "cfg": config(w.n, w.extent, w.width, w.height),
            "s1": make_state(s.pose7(0), s.velocity(0)), "map": tuple(t(np.asarray(a, np.float32)) for a in m),
            "frames": frames_of(s, n_frames)}


def run_filter(spec, storage):
    from paper_2212_02988_gb300 import Filter, config, state_arrays
    w = spec["w"]
    F = Filter(config(w.n, w.extent, w.width, w.height, storage=storage), spec["s1"], device=0)
    F.map_load(*spec["map"])
    out = []
    for imu, d, c in spec["frames"]:
        out.append(state_arrays(F.step(imu, w.dt, d, c, want_state=True)))
    m = F.map_store()
    F.close()
    return out, m


def run_server(specs, storage, order="interleaved", budget=8 << 30, **kw):
    from paper_2212_02988_gb300.serve import Server
    srv = Server(budget, storage=storage, **kw)
    ids = [srv.open(sp["cfg"], sp["s1"], sp["map"]) for sp in specs]
    n = max(len(sp["frames"]) for sp in specs)
    for i in range(n):
        for sid, sp in zip(ids, specs):
            if i < len(sp["frames"]):
                imu, d, c = sp["frames"][i]
                srv.submit(sid, imu, sp["w"].dt, d, c, tag=i)
    srv.drain()
    res = {sid: [] for sid in ids}
    for r in srv.poll(1024):
        res[r["stream"]].append(r)
    maps = [srv.map_store(sid, (sp["w"].n,) * 3) for sid, sp in zip(ids, specs)]
    st = srv.stats()
    srv.destroy()
    return [sorted(res[sid], key=lambda r: r["tag"]) for sid in ids], maps, st


def same_state(a, b):
    return (np.array_equal(a["pose"], b["pose"]) and np.array_equal(a["vel"], b["vel"])
            and np.array_equal(a["cov"], b["cov"]) and a["n_localised"] == b["n_localised"])


@pytest.fixture(scope="module")
def specs():
    tiny = synth.tiny(n=32, width=48, height=40)
    return [stream_spec(synth.ROOM64, 11, 5), stream_spec(synth.ROOM128, 12, 4, "settled"),
            stream_spec(tiny, 13, 6), stream_spec(synth.ROOM64, 14, 3)]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_server_matches_prism_step(specs, storage):
    results, maps, st = run_server(specs, storage)
    assert st["frames"] == sum(len(sp["frames"]) for sp in specs)
    assert st["max_batch"] >= 2                     # requests that arrive while batches run are batched
    for sp, res, m in zip(specs, results, maps):
        ref, ref_map = run_filter(sp, storage)
        assert len(res) == len(ref)
        for i, (r, q) in enumerate(zip(res, ref)):
            assert r["status"] == 0
            assert same_state(r, q), (sp["w"].name, i, r["pose"] - q["pose"])
        for k in ("occ", "rgb", "var_occ", "var_rgb"):
            assert torch.equal(m[k], ref_map[k]), k


def test_alone_and_in_the_mix_agree(specs):
    alone, alone_maps, _ = run_server(specs[1:2], "bf16")
    mix, mix_maps, st = run_server(specs[::-1], "bf16")
    k = len(specs) - 2                              # specs[1] in the reversed list
    assert st["max_batch"] > 1
    for a, b in zip(alone[0], mix[k]):
        assert same_state(a, b)
    for key in ("occ", "rgb", "var_occ", "var_rgb"):
        assert torch.equal(alone_maps[0][key], mix_maps[k][key])


def test_direct_launches_match_the_graph(specs):
    g, _, sg = run_server(specs[:2], "bf16", use_graph=True)
    d, _, sd = run_server(specs[:2], "bf16", use_graph=False)
    assert sg["graph_launches"] == sg["batches"] and sd["graph_launches"] == 0
    for ra, rb in zip(g, d):
        for a, b in zip(ra, rb):
            assert same_state(a, b)


def test_admission_waits_for_budget(specs):
    from paper_2212_02988_gb300.serve import Server
    a, b, c = specs[0], specs[3], specs[1]
    ba, bb, bc = (Server.stream_bytes(sp["cfg"], "bf16") for sp in (a, b, c))
    assert ba <= bc
    budget = bb + bc                                # a and b fit; c waits until a is released
    srv = Server(budget, storage="bf16")
    ia = srv.open(a["cfg"], a["s1"], a["map"])
    ib = srv.open(b["cfg"], b["s1"], b["map"])
    ic = srv.open(c["cfg"], c["s1"], c["map"])
    for sid, sp in ((ia, a), (ib, b), (ic, c)):
        for i, (imu, d, col) in enumerate(sp["frames"][:2]):
            srv.submit(sid, imu, sp["w"].dt, d, col, tag=i)
    got = []
    deadline = time.time() + 60
    while len(got) < 4 and time.time() < deadline:
        got += srv.poll(64, timeout_ms=200)
    st = srv.stats()
    assert st["streams_queued"] == 1 and st["streams_resident"] == 2
    assert {r["stream"] for r in got} == {ia, ib}
    assert st["bytes_in_use"] == ba + bb <= budget
    srv.close(ia)
    deadline = time.time() + 60
    while len([r for r in got if r["stream"] == ic]) < 2 and time.time() < deadline:
        got += srv.poll(64, timeout_ms=200)
    cres = sorted([r for r in got if r["stream"] == ic], key=lambda r: r["tag"])
    assert len(cres) == 2
    ref, _ = run_filter({**c, "frames": c["frames"][:2]}, "bf16")
    for r, q in zip(cres, ref):
        assert same_state(r, q)
    assert srv.stats()["bytes_peak"] <= budget
    srv.close(ib)
    srv.close(ic)
    srv.drain()
    deadline = time.time() + 30
    while srv.stats()["bytes_in_use"] and time.time() < deadline:
        time.sleep(0.05)
    assert srv.stats()["bytes_in_use"] == 0
    srv.destroy()


def test_submit_after_close_and_bad_arguments(specs):
    from paper_2212_02988_gb300.filter import PrismError
    from paper_2212_02988_gb300.serve import Server
    sp = specs[2]
    srv = Server(1 << 30, storage="f32")
    sid = srv.open(sp["cfg"], sp["s1"], sp["map"])
    imu, d, c = sp["frames"][0]
    with pytest.raises(PrismError):
        srv.submit(sid, imu, -1.0, d, c)           # dt must be > 0
    srv.close(sid)
    with pytest.raises(PrismError) as e:
        srv.submit(sid, imu, sp["w"].dt, d, c)
    assert e.value.status == -5
    too_big = Server(1 * MiB, storage="f32")
    with pytest.raises(PrismError) as e:
        too_big.open(specs[1]["cfg"], specs[1]["s1"])
    assert e.value.status == -2
    too_big.destroy()
    srv.destroy()
