"""CPU-side checks of the C ABI: libprism.so loads and exports every
function include/prism.h declares, the ctypes mirrors match the C struct
layouts, and prism_config_default carries the paper's constants."""
import ctypes as C
import json
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_02988_gb300 import build as B
    B.build()
    from paper_2212_02988_gb300 import _lib
    return _lib


def test_exports_every_declared_function(lib):
    names = lib.header_functions()
    assert len(names) >= 20
    L = lib.load()
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_struct_layouts_match_header(lib, tmp_path):
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "prism.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(prism_config), sizeof(prism_state), sizeof(prism_stats), sizeof(prism_timing));
  printf("%zu %zu %zu\\n", offsetof(prism_config, voxel), offsetof(prism_config, gravity), offsetof(prism_state, n_localised));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    a, b = subprocess.check_output([str(exe)], text=True).split("\n")[:2]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [C.sizeof(lib.Config), C.sizeof(lib.State), C.sizeof(lib.Stats), C.sizeof(lib.Timing)]
    assert offs == [lib.Config.voxel.offset, lib.Config.gravity.offset, lib.State.n_localised.offset]


def test_config_default_is_the_paper(lib):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    c = lib.Config()
    lib.load().prism_config_default(C.byref(c), 256, 6.4, 640, 480)
    assert c.voxel == pytest.approx(0.025)
    assert c.eps == pytest.approx(gold["eps_over_voxel"]["value"] * c.voxel)
    assert c.trunc == pytest.approx(gold["trunc_over_voxel"]["value"] * c.voxel)
    assert c.tau == gold["tau"]["value"]
    assert c.update_var == gold["sigma_update"]["value"] ** 2
    assert (c.init_occ, c.init_rgb) == (gold["init_occ"]["value"], gold["init_rgb"]["value"])
    assert list(c.sigma_vel) == [gold["sigma_vel_translation"]["value"], gold["sigma_vel_rotation"]["value"]]
    assert list(c.sigma_pose) == [gold["sigma_pose_translation"]["value"], gold["sigma_pose_rotation"]["value"]]
    assert (c.gate_geo, c.gate_rgb, c.b_geo, c.b_rgb, c.ema) == (
        gold["gate_geo"]["value"], gold["gate_rgb"]["value"], gold["b_geo"]["value"], gold["b_rgb"]["value"],
        gold["ema"]["value"])
    assert c.fx == 560.0 and c.cx == 319.5 and c.cy == 239.5
    assert c.skip_empty == 1
    # the paper's Adam (App. F.2), selected by optimiser = 1
    assert c.optimiser == 0 and c.adam_steps == 1000 and c.adam_pixels == 200
    assert c.adam_lr_t == 1e-3 and c.adam_lr_r == 3.6e-4 and c.adam_beta2 == 0.999 and c.adam_eps == 1e-8


def test_invalid_config_rejected_without_gpu_work(lib):
    L = lib.load()
    c = lib.Config()
    L.prism_config_default(C.byref(c), 64, 4.0, 80, 60)
    c.nx = 60                                   # not a multiple of 8
    h = C.c_void_p()
    assert L.prism_create_map(C.byref(c), None, None, C.byref(h)) == lib.EINVAL
    assert b"multiples of 8" in L.prism_last_error(None)
    c.nx, c.skip_empty = 64, 2
    assert L.prism_create_map(C.byref(c), None, None, C.byref(h)) == lib.EINVAL
    assert b"skip_empty" in L.prism_last_error(None)
    c.skip_empty, c.optimiser = 1, 2
    assert L.prism_create_map(C.byref(c), None, None, C.byref(h)) == lib.EINVAL
    assert b"optimiser" in L.prism_last_error(None)
    c.optimiser, c.adam_pixels = 1, 300                # more pixels a step than the kernel's block
    assert L.prism_create_map(C.byref(c), None, None, C.byref(h)) == lib.EINVAL
    assert b"adam_pixels" in L.prism_last_error(None)
    assert L.prism_destroy(None) == lib.EINVAL
    assert L.prism_status_string(lib.ENOTPD) == b"matrix not positive definite"


def test_product_path_does_not_touch_the_oracle():
    """The package and its C sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2212_02988_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text, f


def test_serve_struct_layouts_and_defaults(lib, tmp_path):
    src = tmp_path / "probe_serve.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "prism_serve.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(prism_serve_config), sizeof(prism_serve_result), sizeof(prism_serve_stats),
         offsetof(prism_serve_result, state), offsetof(prism_serve_stats, kernel_launches));
  return 0;
}
""")
    exe = tmp_path / "probe_serve"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]
    assert vals == [C.sizeof(lib.ServeConfig), C.sizeof(lib.ServeResult), C.sizeof(lib.ServeStats),
                    lib.ServeResult.state.offset, lib.ServeStats.kernel_launches.offset]
    c = lib.ServeConfig()
    lib.load().prism_serve_config_default(C.byref(c))
    assert (c.max_slots, c.storage, c.n_gn, c.max_inflight, c.use_graph) == (32, lib.STORAGE_BF16, 10, 2, 1)


def test_serve_stream_bytes_host_only(lib):
    """The admission footprint is computed on the host (no device needed):
    the six map planes dominate, bf16 halves them, and it grows with the
    image."""
    L = lib.load()

    def cfg(n, w, h):
        c = lib.Config()
        L.prism_config_default(C.byref(c), n, 6.4, w, h)
        return c

    def pad(x):
        return (x + 255) // 256 * 256

    c = cfg(256, 640, 480)
    f32 = L.prism_serve_stream_bytes(C.byref(c), lib.STORAGE_F32)
    b16 = L.prism_serve_stream_bytes(C.byref(c), lib.STORAGE_BF16)
    npad = 258 ** 3
    assert f32 - b16 == 6 * (pad(4 * npad) - pad(2 * npad))
    assert f32 > 6 * 4 * npad
    assert L.prism_serve_stream_bytes(C.byref(cfg(256, 320, 240)), lib.STORAGE_F32) < f32
    bad = cfg(60, 80, 60)
    assert L.prism_serve_stream_bytes(C.byref(bad), lib.STORAGE_F32) == -1
    assert L.prism_serve_stream_bytes(C.byref(c), 7) == -1


def test_serve_create_rejects_bad_config_without_gpu_work(lib):
    L = lib.load()
    c = lib.ServeConfig()
    L.prism_serve_config_default(C.byref(c))
    c.max_slots = 65
    h = C.c_void_p()
    assert L.prism_serve_create(C.byref(c), C.byref(h)) == lib.EINVAL
    assert b"max_slots" in L.prism_serve_last_error(None)
    c.max_slots, c.n_gn = 8, 63
    assert L.prism_serve_create(C.byref(c), C.byref(h)) == lib.EINVAL
    assert L.prism_serve_destroy(None) == lib.EINVAL


def test_entry_points_reject_a_null_handle_without_gpu_work(lib):
    """Every handle-taking entry answers PRISM_EINVAL for a NULL handle
    before touching the device (the check runs on a machine without a GPU)."""
    L = lib.load()
    f = C.c_float(0.0)
    st = lib.State()
    assert L.prism_step(None, None, 0, 0.1, C.byref(f), C.byref(f), None) == lib.EINVAL
    assert L.prism_step_host(None, None, 0, 0.1, C.byref(f), C.byref(f), C.byref(st)) == lib.EINVAL
    cnt = (C.c_int32 * 1)(0)
    dts = (C.c_double * 1)(0.1)
    assert L.prism_rollout(None, 1, 1, None, cnt, dts, None, None, None, None) == lib.EINVAL
    assert L.prism_predict(None, None, 0, 0.1) == lib.EINVAL
    assert L.prism_get_state(None, C.byref(st)) == lib.EINVAL
    assert b"NULL" in L.prism_last_error(None)


def test_noalloc_rejects_bad_arguments_without_gpu_work(lib):
    """The allocation-free entry checks its configuration, its size limit and
    its poses before any CUDA call (so this runs without a GPU): a frame just
    over the stated maximum, a NaN discontinuity threshold, a zero quaternion."""
    L = lib.load()
    c = lib.Config()
    L.prism_config_default(C.byref(c), 64, 4.0, 641, 480)
    pose = (C.c_double * 7)(0, 0, 0, 1, 0, 0, 0)
    img = (C.c_float * 4)()
    out = (C.c_double * 80)()
    args = lambda cfg, p: (C.byref(cfg), pose, img, img, p, img, img, None, out)
    assert L.prism_normal_equations_noalloc(*args(c, pose)) == lib.EINVAL
    assert b"at most 307200" in L.prism_noalloc_last_error()
    L.prism_config_default(C.byref(c), 64, 4.0, 640, 480)
    c.disc = float("nan")
    assert L.prism_normal_equations_noalloc(*args(c, pose)) == lib.EINVAL
    assert b"discontinuity" in L.prism_noalloc_last_error()
    c.disc = 0.1
    zero = (C.c_double * 7)(0, 0, 0, 0, 0, 0, 0)
    assert L.prism_normal_equations_noalloc(*args(c, zero)) == lib.EINVAL
    assert b"not finite" in L.prism_noalloc_last_error()


def test_noalloc_binding_checks_devices_before_any_call():
    """The binding refuses image tensors on different devices, or not on a
    CUDA device, before it reaches the library (CPU and meta tensors stand in
    for two devices here)."""
    import torch
    from paper_2212_02988_gb300.filter import _common_cuda_device
    a = torch.zeros(2, 2)
    m = torch.empty(2, 2, device="meta")
    with pytest.raises(ValueError, match="share one device"):
        _common_cuda_device((("anchor_depth", a), ("anchor_rgb", a), ("depth", m), ("rgb", a)))
    with pytest.raises(ValueError, match="CUDA tensors"):
        _common_cuda_device((("anchor_depth", a), ("depth", a)))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        _common_cuda_device((("anchor_depth", a), ("depth", None)))
