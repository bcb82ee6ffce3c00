"""Python face of the serving ABI (include/prism_serve.h): argument
marshalling only.  The server, its admission queue, batching and completion
threads and the batched kernels all live in libprism.so.

    srv = Server(budget_bytes=32 << 30, storage="bf16")
    sid = srv.open(config(128, 6.4, 320, 240), make_state(pose7, vel6))
    srv.submit(sid, imu, dt, depth, rgb)        # frames: pinned host or CUDA tensors
    for r in srv.poll(timeout_ms=100): ...

Frames and initial maps are read asynchronously; this wrapper keeps a
reference to them until their result has been polled (for a map: until the
stream's first result), as the ABI requires.
"""
from __future__ import annotations

import ctypes as C
import itertools

import numpy as np
import torch

from . import _lib
from ._lib import Config, ServeConfig, ServeResult, ServeStats, State
from .filter import PrismError, state_arrays


def _fptr(t: torch.Tensor | None, shape, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


class Server:
    """A multi-stream PRISM filter server on one CUDA device."""

    def __init__(self, budget_bytes: int, max_slots: int = 32, storage: str = "bf16", n_gn: int = 10,
                 max_inflight: int = 2, use_graph: bool = True, device: int = 0):
        self.L = _lib.load()
        c = ServeConfig()
        self.L.prism_serve_config_default(C.byref(c))
        c.hbm_budget_bytes = int(budget_bytes)
        c.max_slots = max_slots
        c.storage = {"f32": _lib.STORAGE_F32, "bf16": _lib.STORAGE_BF16}[storage]
        c.n_gn = n_gn
        c.max_inflight = max_inflight
        c.use_graph = int(bool(use_graph))
        c.device = device
        self.cfg = c
        self.device = device
        h = C.c_void_p()
        with torch.cuda.device(device):
            st = self.L.prism_serve_create(C.byref(c), C.byref(h))
        if st != _lib.OK:
            raise PrismError(st, self.L.prism_serve_last_error(None).decode())
        self.h = h
        self._shapes = {}
        self._keep = {}          # tag -> tensors read by a pending request
        self._map_keep = {}      # stream id -> initial map tensors (until its first result)
        self._tags = itertools.count()
        self._user_tags = {}
        self._bufs = {}

    def _check(self, st):
        if st != _lib.OK:
            raise PrismError(st, self.L.prism_serve_last_error(self.h).decode())

    @staticmethod
    def stream_bytes(cfg: Config, storage: str = "bf16") -> int:
        s = {"f32": _lib.STORAGE_F32, "bf16": _lib.STORAGE_BF16}[storage]
        return int(_lib.load().prism_serve_stream_bytes(C.byref(cfg), s))

    def open(self, cfg: Config, s1: State | None = None, map_arrays=None) -> int:
        """New stream; map_arrays: optional (occ, rgb, var_occ, var_rgb) CUDA tensors."""
        n = (cfg.nz, cfg.ny, cfg.nx)
        ptrs = [None] * 4
        if map_arrays is not None:
            shapes = [n, n + (3,), n, n]
            ptrs = [_fptr(a, sh, nm) for a, sh, nm in zip(map_arrays, shapes, ("occ", "rgb", "var_occ", "var_rgb"))]
        sid = C.c_int32()
        self._check(self.L.prism_serve_open(self.h, C.byref(cfg), C.byref(s1) if s1 is not None else None,
                                            *ptrs, C.byref(sid)))
        self._shapes[sid.value] = (cfg.height, cfg.width)
        if map_arrays is not None:
            self._map_keep[sid.value] = tuple(map_arrays)
        return sid.value

    def submit(self, sid: int, imu, dt: float, depth: torch.Tensor, rgb: torch.Tensor, tag=None) -> int:
        """Queues one step; returns the internal tag its result carries."""
        H, W = self._shapes[sid]
        imu_a = None if imu is None else np.ascontiguousarray(imu, dtype=np.float64)
        n = 0 if imu_a is None else imu_a.shape[0]
        t = next(self._tags)
        dp = _fptr(depth, (H, W), "depth")
        cp = _fptr(rgb, (H, W, 3), "rgb")
        self._keep[t] = (depth, rgb)
        self._user_tags[t] = tag
        st = self.L.prism_serve_submit(self.h, sid, None if imu_a is None else
                                       imu_a.ctypes.data_as(C.POINTER(C.c_double)), n, float(dt), dp, cp, t)
        if st != _lib.OK:
            self._keep.pop(t)
            self._user_tags.pop(t)
            self._check(st)
        return t

    def poll(self, max_results: int = 256, timeout_ms: int = 0) -> list[dict]:
        buf = self._bufs.get(max_results)
        if buf is None:
            buf = self._bufs[max_results] = (ServeResult * max_results)()
        n = C.c_int32()
        self._check(self.L.prism_serve_poll(self.h, buf, max_results, timeout_ms, C.byref(n)))
        out = []
        for r in buf[:n.value]:
            self._keep.pop(r.tag, None)
            self._map_keep.pop(r.stream_id, None)
            d = {"stream": r.stream_id, "status": r.status, "tag": self._user_tags.pop(r.tag, None),
                 "batch": r.batch, "batch_size": r.batch_size, "submit_s": r.submit_s, "done_s": r.done_s,
                 "latency_ms": r.latency_ms}
            d.update(state_arrays(r.state))
            out.append(d)
        return out

    def close(self, sid: int):
        self._check(self.L.prism_serve_close(self.h, sid))

    def drain(self, timeout_ms: int = 120000):
        self._check(self.L.prism_serve_drain(self.h, timeout_ms))

    def stats(self) -> dict:
        s = ServeStats()
        self._check(self.L.prism_serve_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServeStats._fields_ if k != "reserved"}

    def check_status(self) -> int:
        """The bounds-check build's first index violation of any stream (0:
        none; always 0 in the plain build): prism_serve_check_status."""
        w = C.c_uint64(0)
        self._check(self.L.prism_serve_check_status(self.h, C.byref(w)))
        return int(w.value)

    def map_store(self, sid: int, shape) -> dict:
        nz, ny, nx = shape
        dev = torch.device("cuda", self.device)
        out = {"occ": torch.empty((nz, ny, nx), device=dev), "rgb": torch.empty((nz, ny, nx, 3), device=dev),
               "var_occ": torch.empty((nz, ny, nx), device=dev), "var_rgb": torch.empty((nz, ny, nx), device=dev)}
        self._check(self.L.prism_serve_map_store(self.h, sid, *(C.c_void_p(out[k].data_ptr())
                                                              for k in ("occ", "rgb", "var_occ", "var_rgb"))))
        return out

    def destroy(self):
        if self.h:
            self._check(self.L.prism_serve_destroy(self.h))
            self.h = None
            self._keep.clear()
            self._map_keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
