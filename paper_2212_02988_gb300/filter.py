"""Python face of the C ABI (include/prism.h): argument marshalling only.

Every method forwards to the prism_* entry of the same name; device arrays
are torch CUDA tensors (float32, contiguous), host arrays numpy.  All work
runs in libprism.so's kernels on the stream the filter was created with.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import Config, State, Stats, Timing


class PrismError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def config(n: int, extent: float, width: int, height: int, **overrides) -> Config:
    """prism_config_default plus field overrides (origin / sigma_* take sequences)."""
    c = Config()
    _lib.load().prism_config_default(C.byref(c), n, extent, width, height)
    for k, v in overrides.items():
        if k in ("origin", "sigma_vel", "sigma_pose"):
            for i, x in enumerate(v):
                getattr(c, k)[i] = x
        elif k == "storage" and isinstance(v, str):
            c.storage = {"f32": _lib.STORAGE_F32, "bf16": _lib.STORAGE_BF16}[v]
        else:
            setattr(c, k, v)
    return c


def make_state(pose7, vel6=None, cov=None, n_localised: int = 0) -> State:
    s = State()
    pose7 = np.asarray(pose7, dtype=np.float64)
    vel6 = np.zeros(6) if vel6 is None else np.asarray(vel6, dtype=np.float64)
    cov = np.eye(12) * 1e-8 if cov is None else np.asarray(cov, dtype=np.float64)
    for a in range(3):
        s.t[a], s.v[a], s.w[a] = pose7[a], vel6[a], vel6[3 + a]
    for a in range(4):
        s.q[a] = pose7[3 + a]
    for i in range(144):
        s.cov[i] = cov.flat[i]
    s.n_localised = n_localised
    return s


def state_arrays(s: State) -> dict:
    return {"pose": np.array(list(s.t) + list(s.q)), "vel": np.array(list(s.v) + list(s.w)),
            "cov": np.array(s.cov[:]).reshape(12, 12), "n_localised": int(s.n_localised)}


def _dptr(t: torch.Tensor | None, shape=None, dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _host_img(a, shape, name):
    """Pointer to a host float32 image: a contiguous numpy array or CPU tensor
    (pinned memory makes the library's copy asynchronous)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name} must be a contiguous float32 CPU tensor of shape {tuple(shape)}")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous or \
            tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous float32 array of shape {tuple(shape)}")
    return C.c_void_p(a.ctypes.data)


def _hptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _common_cuda_device(named) -> torch.device:
    """The one CUDA device that every (name, tensor) pair lives on; raises
    ValueError before any device work when they differ or are not CUDA."""
    devs = {}
    for name, x in named:
        if not isinstance(x, torch.Tensor):
            raise ValueError(f"{name} must be a CUDA tensor")
        devs.setdefault(x.device, name)
    if len(devs) != 1:
        raise ValueError("image tensors must share one device, got " +
                         ", ".join(f"{n} on {d}" for d, n in devs.items()))
    (d,) = devs
    if d.type != "cuda":
        raise ValueError(f"image tensors must be CUDA tensors, got {d}")
    return d


def normal_equations_noalloc(cfg: Config, anchor_pose7, anchor_depth, anchor_rgb, pose7, depth, rgb,
                             stream: torch.cuda.Stream | None = None) -> dict:
    """prism_normal_equations_noalloc: the normal equations of one pose with
    no device allocation (scratch in the library's static device array; see
    include/prism.h).  The four images must be CUDA tensors on one device;
    the call runs on that device, on `stream` (which must belong to it) or
    on that device's current stream."""
    d = _common_cuda_device((("anchor_depth", anchor_depth), ("anchor_rgb", anchor_rgb),
                             ("depth", depth), ("rgb", rgb)))
    if stream is not None and stream.device != d:
        raise ValueError(f"stream is on {stream.device}, the images on {d}")
    L = _lib.load()
    H, W = cfg.height, cfg.width
    ap = np.ascontiguousarray(anchor_pose7, dtype=np.float64)
    p = np.ascontiguousarray(pose7, dtype=np.float64)
    out = np.zeros(80)
    with torch.cuda.device(d):
        s = stream if stream is not None else torch.cuda.current_stream(d)
        st = L.prism_normal_equations_noalloc(
            C.byref(cfg), _hptr(ap), _dptr(anchor_depth, (H, W), name="anchor_depth"),
            _dptr(anchor_rgb, (H, W, 3), name="anchor_rgb"), _hptr(p), _dptr(depth, (H, W), name="depth"),
            _dptr(rgb, (H, W, 3), name="rgb"), C.c_void_p(s.cuda_stream), _hptr(out))
    if st != _lib.OK:
        raise PrismError(st, L.prism_noalloc_last_error().decode())
    return {"H": out[:36].reshape(6, 6), "g": out[36:42], "Ht": out[42:78].reshape(6, 6),
            "cost": out[78], "count": out[79]}


class Filter:
    """One PRISM filter (map + state + anchor) on one CUDA device."""

    def __init__(self, cfg: Config, s1: State | None = None, stream: torch.cuda.Stream | None = None,
                 device: int | None = None):
        self.L = _lib.load()
        self.cfg = cfg
        self.device = torch.cuda.current_device() if device is None else device
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = C.c_void_p()
            self._check(self.L.prism_create_map(C.byref(cfg), C.byref(s1) if s1 is not None else None,
                                                C.c_void_p(self.stream.cuda_stream), C.byref(h)), None)
        self.h = h
        self.W, self.H = cfg.width, cfg.height
        self.N = cfg.nx * cfg.ny * cfg.nz
        # Counts calls that may change the map (load, update, step, descent):
        # autograd.PrismRender reloads its map only when this or its tensors changed.
        self.map_version = 0

    # ------------------------------------------------------------- plumbing
    def _check(self, status: int, h):
        if status != _lib.OK:
            msg = self.L.prism_last_error(h).decode()
            raise PrismError(status, msg)

    def _img(self, depth, rgb):
        return (_dptr(depth, (self.H, self.W), name="depth"), _dptr(rgb, (self.H, self.W, 3), name="rgb"))

    def close(self):
        if getattr(self, "h", None):
            self._check(self.L.prism_destroy(self.h), None)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ the ABI
    def predict(self, imu: np.ndarray | None, dt: float):
        imu = np.zeros((0, 7)) if imu is None else np.ascontiguousarray(imu, dtype=np.float64)
        if imu.ndim != 2 or imu.shape[1] != 7:
            raise ValueError("imu must be (n, 7)")
        self._check(self.L.prism_predict(self.h, _hptr(imu) if len(imu) else None, len(imu), dt), self.h)

    def localise(self, depth, rgb, want_state: bool = True):
        d, c = self._img(depth, rgb)
        out = State() if want_state else None
        self._check(self.L.prism_localise(self.h, d, c, C.byref(out) if out is not None else None), self.h)
        return out

    def update_map(self, depth, rgb):
        d, c = self._img(depth, rgb)
        self.map_version += 1
        self._check(self.L.prism_update_map(self.h, d, c), self.h)

    def render(self, pose7=None, depth=None, rgb=None, mask=None, hitk=None, alloc: bool = True):
        """Render at pose7 (None: the state mean, which also sets the anchor).
        Missing outputs are allocated when alloc is True."""
        dev = torch.device("cuda", self.device)
        if alloc:
            depth = torch.empty((self.H, self.W), device=dev) if depth is None else depth
            rgb = torch.empty((self.H, self.W, 3), device=dev) if rgb is None else rgb
            mask = torch.empty((self.H, self.W), dtype=torch.uint8, device=dev) if mask is None else mask
            hitk = torch.empty((self.H, self.W), dtype=torch.int32, device=dev) if hitk is None else hitk
        p = None if pose7 is None else np.ascontiguousarray(pose7, dtype=np.float64)
        self._check(self.L.prism_render(self.h, _hptr(p), _dptr(depth, (self.H, self.W), name="depth"),
                                        _dptr(rgb, (self.H, self.W, 3), name="rgb"),
                                        _dptr(mask, (self.H, self.W), torch.uint8, "mask"),
                                        _dptr(hitk, (self.H, self.W), torch.int32, "hitk")), self.h)
        return {"depth": depth, "rgb": rgb, "mask": mask, "hitk": hitk}

    def step(self, imu, dt, depth, rgb, want_state: bool = False):
        imu = np.zeros((0, 7)) if imu is None else np.ascontiguousarray(imu, dtype=np.float64)
        d, c = self._img(depth, rgb)
        out = State() if want_state else None
        self.map_version += 1
        self._check(self.L.prism_step(self.h, _hptr(imu) if len(imu) else None, len(imu), dt, d, c,
                                      C.byref(out) if out is not None else None), self.h)
        return out

    def rollout(self, windows, dt, images: bool = True, hitk: bool = False, want_states: bool = True,
                out: dict | None = None) -> dict:
        """prism_rollout: predictive rollouts of candidate control sequences.
        windows: n_seq sequences of k IMU windows ((n, 7) arrays or None);
        dt: a scalar or an (n_seq, k) array of frame intervals.  Returns the
        predicted states ((n_seq, k) nested lists of State, or None) and,
        with images, depth (n_seq, k, H, W), rgb (n_seq, k, H, W, 3) and
        hitk (n_seq, k, H, W) when asked.  `out` may hold preallocated image
        tensors of those shapes."""
        n_seq, k = len(windows), len(windows[0])
        if n_seq == 0 or k == 0 or any(len(w) != k for w in windows):
            raise ValueError("windows must be n_seq >= 1 sequences of the same k >= 1 windows")
        rows, counts = [], np.zeros(n_seq * k, dtype=np.int32)
        for s_i, seq in enumerate(windows):
            for i, w in enumerate(seq):
                if w is None or len(w) == 0:
                    continue
                w = np.ascontiguousarray(w, dtype=np.float64)
                if w.ndim != 2 or w.shape[1] != 7:
                    raise ValueError("each IMU window must be (n, 7)")
                rows.append(w)
                counts[s_i * k + i] = len(w)
        imu = np.ascontiguousarray(np.concatenate(rows)) if rows else None
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n_seq, k)).ravel())
        dev = torch.device("cuda", self.device)
        out = dict(out or {})
        shp = (n_seq, k, self.H, self.W)
        if images:
            out.setdefault("depth", torch.empty(shp, device=dev))
            out.setdefault("rgb", torch.empty(shp + (3,), device=dev))
            if hitk:
                out.setdefault("hitk", torch.empty(shp, dtype=torch.int32, device=dev))
        recs = (State * (n_seq * k))() if want_states else None
        self._check(self.L.prism_rollout(self.h, n_seq, k, _hptr(imu), counts.ctypes.data_as(C.POINTER(C.c_int32)),
                                         _hptr(dts), recs,
                                         _dptr(out.get("depth"), shp, name="depth"),
                                         _dptr(out.get("rgb"), shp + (3,), name="rgb"),
                                         _dptr(out.get("hitk"), shp, torch.int32, "hitk")), self.h)
        out["states"] = None if recs is None else [[recs[s_i * k + i] for i in range(k)] for s_i in range(n_seq)]
        return out

    def step_host(self, imu, dt, depth, rgb, want_state: bool = False):
        """prism_step_host: the step with the frame in host memory (numpy or
        CPU tensors; pinned tensors make the upload asynchronous)."""
        imu = np.zeros((0, 7)) if imu is None else np.ascontiguousarray(imu, dtype=np.float64)
        d = _host_img(depth, (self.H, self.W), "depth")
        c = _host_img(rgb, (self.H, self.W, 3), "rgb")
        out = State() if want_state else None
        self.map_version += 1
        self._check(self.L.prism_step_host(self.h, _hptr(imu) if len(imu) else None, len(imu), dt, d, c,
                                           C.byref(out) if out is not None else None), self.h)
        return out

    def map_descent(self, poses, depth, rgb, sd: float, sc: float, lr_occ: float, lr_rgb: float,
                    want_loss: bool = True):
        """prism_map_descent: one gradient-descent step on the map means over
        n frames with known poses (n x 7), depth (n, H, W) and rgb (n, H, W, 3)
        CUDA tensors.  Returns the loss before the step (or None)."""
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 7)
        n = len(poses)
        d = _dptr(depth, (n, self.H, self.W), name="depth")
        c = _dptr(rgb, (n, self.H, self.W, 3), name="rgb")
        out = np.zeros(1) if want_loss else None
        self.map_version += 1
        self._check(self.L.prism_map_descent(self.h, n, _hptr(poses), d, c, sd, sc, lr_occ, lr_rgb,
                                             _hptr(out)), self.h)
        return float(out[0]) if want_loss else None

    def get_state(self) -> State:
        s = State()
        self._check(self.L.prism_get_state(self.h, C.byref(s)), self.h)
        return s

    def set_state(self, s: State):
        self._check(self.L.prism_set_state(self.h, C.byref(s)), self.h)

    def map_load(self, occ, rgb, var_occ=None, var_rgb=None):
        """Load map arrays (None leaves that part of the map unchanged)."""
        N = self.N
        f = lambda a, n, name: None if a is None else _dptr(a.reshape(-1), (n,), name=name)
        self.map_version += 1
        self._check(self.L.prism_map_load(self.h, f(occ, N, "occ"), f(rgb, 3 * N, "rgb"),
                                          f(var_occ, N, "var_occ"), f(var_rgb, N, "var_rgb")), self.h)

    def render_backward(self, pose7, grad_depth=None, grad_rgb=None, grad_occ=None, grad_rgb_map=None):
        """Adjoint of render(pose7); map gradients are accumulated into the given
        tensors (shapes of the map arrays).  Returns (grad_pose6, grad_pose7)."""
        p = np.ascontiguousarray(pose7, dtype=np.float64)
        g6, g7 = np.zeros(6), np.zeros(7)
        N = self.N
        self._check(self.L.prism_render_backward(
            self.h, _hptr(p), _dptr(grad_depth, (self.H, self.W), name="grad_depth"),
            _dptr(grad_rgb, (self.H, self.W, 3), name="grad_rgb"),
            None if grad_occ is None else _dptr(grad_occ.view(-1), (N,), name="grad_occ"),
            None if grad_rgb_map is None else _dptr(grad_rgb_map.view(-1), (3 * N,), name="grad_rgb_map"),
            _hptr(g6), _hptr(g7)), self.h)
        return g6, g7

    def render_backward_async(self, pose7, grad_depth=None, grad_rgb=None, grad_occ=None, grad_rgb_map=None):
        """render_backward without the host pose gradient (no synchronisation)."""
        p = np.ascontiguousarray(pose7, dtype=np.float64)
        N = self.N
        self._check(self.L.prism_render_backward(
            self.h, _hptr(p), _dptr(grad_depth, (self.H, self.W), name="grad_depth"),
            _dptr(grad_rgb, (self.H, self.W, 3), name="grad_rgb"),
            None if grad_occ is None else _dptr(grad_occ.view(-1), (N,), name="grad_occ"),
            None if grad_rgb_map is None else _dptr(grad_rgb_map.view(-1), (3 * N,), name="grad_rgb_map"),
            None, None), self.h)

    def map_store(self) -> dict:
        dev = torch.device("cuda", self.device)
        n = (self.cfg.nz, self.cfg.ny, self.cfg.nx)
        out = {"occ": torch.empty(n, device=dev), "rgb": torch.empty(n + (3,), device=dev),
               "var_occ": torch.empty(n, device=dev), "var_rgb": torch.empty(n, device=dev)}
        self._check(self.L.prism_map_store(self.h, *(C.c_void_p(out[k].data_ptr())
                                                      for k in ("occ", "rgb", "var_occ", "var_rgb"))),
                    self.h)
        return out

    def anchor_load(self, pose7, depth, rgb):
        p = np.ascontiguousarray(pose7, dtype=np.float64)
        d, c = self._img(depth, rgb)
        self._check(self.L.prism_anchor_load(self.h, _hptr(p), d, c), self.h)

    def normal_equations(self, pose7, depth, rgb) -> dict:
        p = np.ascontiguousarray(pose7, dtype=np.float64)
        d, c = self._img(depth, rgb)
        out = np.zeros(80)
        self._check(self.L.prism_normal_equations(self.h, _hptr(p), d, c, _hptr(out)), self.h)
        return {"H": out[:36].reshape(6, 6), "g": out[36:42], "Ht": out[42:78].reshape(6, 6),
                "cost": out[78], "count": out[79]}

    def stats(self) -> dict:
        s = Stats()
        self._check(self.L.prism_get_stats(self.h, C.byref(s)), self.h)
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_timing(self, enabled: bool = True):
        self._check(self.L.prism_set_timing(self.h, int(enabled)), self.h)

    def set_detail_counters(self, enabled: bool = True):
        self._check(self.L.prism_set_detail_counters(self.h, int(enabled)), self.h)

    def set_cooperative(self, enabled: bool = True):
        """The localisation's launch form: one cooperative launch for the
        Gauss-Newton passes after the first (default), or one launch per
        pass; the same bits either way."""
        self._check(self.L.prism_set_cooperative(self.h, int(enabled)), self.h)

    def timing(self) -> dict:
        t = Timing()
        self._check(self.L.prism_get_timing(self.h, C.byref(t)), self.h)
        return {k: getattr(t, k) for k, _ in Timing._fields_}

    def timing_reset(self):
        self._check(self.L.prism_timing_reset(self.h), self.h)

    def device_bytes(self) -> int:
        return int(self.L.prism_device_bytes(self.h))

    def check_status(self) -> int:
        """The bounds-check build's first index violation on this handle (0:
        none; always 0 in the plain build): prism_check_status."""
        w = C.c_uint64(0)
        self._check(self.L.prism_check_status(self.h, C.byref(w)), self.h)
        return int(w.value)
