"""ctypes declarations of include/prism.h and include/prism_serve.h, and the
loader of libprism.so.

The library is built in-tree by paper_2212_02988_gb300.build; if it is
missing this module raises at load time — there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
# PRISM_CHECKED=1 in the environment loads the bounds-check build instead
# (libprism_checked.so, built beside it; prism_check_status in prism.h).
LIB_PATH = os.path.join(PKG, "libprism_checked.so" if os.environ.get("PRISM_CHECKED") == "1" else "libprism.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "prism.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(PKG), "include", "prism_serve.h")]

OK, EINVAL, ENOMEM, ECUDA, ENOTPD, ESTATE = 0, -1, -2, -3, -4, -5
STORAGE_F32, STORAGE_BF16 = 0, 1


class Config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("storage", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("n_gn", C.c_int32),
                ("skip_empty", C.c_int32), ("voxel", C.c_double), ("origin", C.c_double * 3),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("eps", C.c_double), ("tau", C.c_double), ("max_depth", C.c_double),
                ("trunc", C.c_double), ("prior_var", C.c_double), ("init_occ", C.c_double),
                ("init_rgb", C.c_double), ("update_var", C.c_double),
                ("sigma_vel", C.c_double * 2), ("sigma_pose", C.c_double * 2),
                ("b_geo", C.c_double), ("b_rgb", C.c_double), ("gate_geo", C.c_double),
                ("gate_rgb", C.c_double), ("floor_geo", C.c_double), ("floor_rgb", C.c_double),
                ("ema", C.c_double), ("disc", C.c_double), ("gravity", C.c_double),
                ("optimiser", C.c_int32), ("adam_steps", C.c_int32), ("adam_pixels", C.c_int32),
                ("adam_reserved", C.c_int32), ("adam_seed", C.c_uint64), ("adam_lr_t", C.c_double),
                ("adam_lr_r", C.c_double), ("adam_beta2", C.c_double), ("adam_eps", C.c_double)]


class State(C.Structure):
    _fields_ = [("t", C.c_double * 3), ("q", C.c_double * 4), ("v", C.c_double * 3),
                ("w", C.c_double * 3), ("cov", C.c_double * 144), ("n_localised", C.c_int32),
                ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("render_rays", "render_samples", "render_hits",
                                         "fuse_updates", "fuse_colour_updates", "track_pixels",
                                         "render_unique_corners", "kernel_launches")]


class Timing(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("predict_ms", "localise_ms", "fuse_ms", "render_ms",
                                          "anchor_ms")] + \
               [(n, C.c_int64) for n in ("predict_n", "localise_n", "fuse_n", "render_n", "anchor_n")] + \
               [("laplace_ms", C.c_double), ("laplace_n", C.c_int64)]


class ServeConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("storage", C.c_int32),
                ("n_gn", C.c_int32), ("max_inflight", C.c_int32), ("use_graph", C.c_int32),
                ("device", C.c_int32)]


class ServeResult(C.Structure):
    _fields_ = [("stream_id", C.c_int32), ("status", C.c_int32), ("tag", C.c_int64), ("batch", C.c_int64),
                ("batch_size", C.c_int32), ("reserved", C.c_int32), ("submit_s", C.c_double),
                ("done_s", C.c_double), ("latency_ms", C.c_double), ("state", State)]


class ServeStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("batches", "frames", "max_batch", "bytes_in_use", "bytes_peak",
                                         "budget")] + \
               [(n, C.c_int32) for n in ("streams_resident", "streams_queued", "streams_open", "reserved")] + \
               [(n, C.c_int64) for n in ("kernel_launches", "graph_launches")]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/prism.h and include/prism_serve.h declare."""
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(prism_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2212_02988_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P, vp, dp, fp = C.POINTER, C.c_void_p, C.POINTER(C.c_double), C.c_void_p
    H = vp
    st = C.c_int
    sig = {
        "prism_config_default": (None, [P(Config), C.c_int32, C.c_double, C.c_int32, C.c_int32]),
        "prism_create_map": (st, [P(Config), P(State), vp, P(H)]),
        "prism_destroy": (st, [H]),
        "prism_predict": (st, [H, dp, C.c_int32, C.c_double]),
        "prism_localise": (st, [H, fp, fp, P(State)]),
        "prism_update_map": (st, [H, fp, fp]),
        "prism_render": (st, [H, dp, fp, fp, vp, vp]),
        "prism_step": (st, [H, dp, C.c_int32, C.c_double, fp, fp, P(State)]),
        "prism_step_host": (st, [H, dp, C.c_int32, C.c_double, fp, fp, P(State)]),
        "prism_get_state": (st, [H, P(State)]),
        "prism_set_state": (st, [H, P(State)]),
        "prism_map_load": (st, [H, fp, fp, fp, fp]),
        "prism_map_store": (st, [H, fp, fp, fp, fp]),
        "prism_anchor_load": (st, [H, dp, fp, fp]),
        "prism_normal_equations": (st, [H, dp, fp, fp, dp]),
        "prism_get_stats": (st, [H, P(Stats)]),
        "prism_set_timing": (st, [H, C.c_int32]),
        "prism_set_detail_counters": (st, [H, C.c_int32]),
        "prism_set_cooperative": (st, [H, C.c_int32]),
        "prism_get_timing": (st, [H, P(Timing)]),
        "prism_timing_reset": (st, [H]),
        "prism_device_bytes": (C.c_int64, [H]),
        "prism_checked_build": (C.c_int32, []),
        "prism_check_status": (st, [H, P(C.c_uint64)]),
        "prism_last_error": (C.c_char_p, [H]),
        "prism_status_string": (C.c_char_p, [C.c_int32]),
        "prism_render_backward": (st, [H, dp, fp, fp, fp, fp, dp, dp]),
        "prism_rollout": (st, [H, C.c_int32, C.c_int32, dp, P(C.c_int32), dp, P(State), fp, fp, fp]),
        "prism_map_descent": (st, [H, C.c_int32, dp, fp, fp, C.c_double, C.c_double, C.c_double, C.c_double,
                                   dp]),
        "prism_normal_equations_noalloc": (st, [P(Config), dp, fp, fp, dp, fp, fp, vp, dp]),
        "prism_noalloc_last_error": (C.c_char_p, []),
        "prism_serve_config_default": (None, [P(ServeConfig)]),
        "prism_serve_stream_bytes": (C.c_int64, [P(Config), C.c_int32]),
        "prism_serve_create": (st, [P(ServeConfig), P(H)]),
        "prism_serve_destroy": (st, [H]),
        "prism_serve_open": (st, [H, P(Config), P(State), fp, fp, fp, fp, P(C.c_int32)]),
        "prism_serve_submit": (st, [H, C.c_int32, dp, C.c_int32, C.c_double, fp, fp, C.c_int64]),
        "prism_serve_close": (st, [H, C.c_int32]),
        "prism_serve_poll": (st, [H, P(ServeResult), C.c_int32, C.c_int32, P(C.c_int32)]),
        "prism_serve_drain": (st, [H, C.c_int32]),
        "prism_serve_get_stats": (st, [H, P(ServeStats)]),
        "prism_serve_check_status": (st, [H, P(C.c_uint64)]),
        "prism_serve_map_store": (st, [H, C.c_int32, fp, fp, fp, fp]),
        "prism_serve_last_error": (C.c_char_p, [H]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L
