"""ctypes binding of the PRISM FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, the package's smoke check and the benchmark's
CPU-baseline leg may import this module.  It loads oracle/liboracle.so,
building it with gcc on first use, and composes the C functions into the
filter step of the paper (Sec. 3.3, App. F):

    frame 1:  fuse at the given state s_1, render the anchor at s_1;
    frame t:  predict (App. E.1/E.2) -> localise (App. E.3, Sec. 4.1) ->
              fuse at the new mean (App. D) -> render the new anchor (App. B);
    rollout:  predict repeatedly from the belief with no observation, and
              render the map mean at each predicted pose mean (App. I).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prism_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GRAVITY = 9.81


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "prism_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("n_gn", C.c_int32),
                ("voxel", C.c_double), ("origin", C.c_double * 3),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("eps", C.c_double), ("tau", C.c_double), ("max_depth", C.c_double),
                ("trunc", C.c_double), ("prior_var", C.c_double), ("init_occ", C.c_double),
                ("update_var", C.c_double), ("sigma_vel", C.c_double * 2),
                ("sigma_pose", C.c_double * 2), ("b_geo", C.c_double), ("b_rgb", C.c_double),
                ("gate_geo", C.c_double), ("gate_rgb", C.c_double), ("floor_geo", C.c_double),
                ("floor_rgb", C.c_double), ("ema", C.c_double), ("disc", C.c_double),
                ("gravity", C.c_double), ("optimiser", C.c_int32), ("adam_steps", C.c_int32),
                ("adam_pixels", C.c_int32), ("adam_pad", C.c_int32), ("adam_seed", C.c_uint64),
                ("adam_lr_t", C.c_double), ("adam_lr_r", C.c_double), ("adam_beta2", C.c_double),
                ("adam_eps", C.c_double)]


class State(C.Structure):
    _fields_ = [("t", C.c_double * 3), ("q", C.c_double * 4), ("v", C.c_double * 3),
                ("w", C.c_double * 3), ("cov", C.c_double * 144), ("n_localised", C.c_int32),
                ("pad", C.c_int32)]


class Prior(C.Structure):
    _fields_ = [("t", C.c_double * 3), ("q", C.c_double * 4), ("v", C.c_double * 3),
                ("w", C.c_double * 3), ("cov", C.c_double * 144), ("cov_pp", C.c_double * 36),
                ("prec_pp", C.c_double * 36), ("D", C.c_double * 36), ("cov_vel", C.c_double * 36)]


class LocDiag(C.Structure):
    _fields_ = [("cost", C.c_double), ("n_pixels", C.c_double), ("xi", C.c_double * 6)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            dp, fp, u8p, i32p, i64p = (P(C.c_double), P(C.c_float), P(C.c_uint8), P(C.c_int32),
                                       P(C.c_int64))
            L.or_render.argtypes = [P(Params), dp, dp, dp, i32p, C.c_int32, dp, dp, u8p, i32p, i64p]
            L.or_render_backward.argtypes = [P(Params), dp, dp, dp, dp, dp, dp, dp, dp]
            L.or_depth_mask.argtypes = [P(Params), fp, u8p]
            L.or_anchor_normals.argtypes = [P(Params), fp, u8p, dp, fp, u8p]
            L.or_residuals.argtypes = [P(Params), dp, fp, fp, dp, fp, fp, dp, dp, i32p, u8p]
            L.or_normal_equations.argtypes = [P(Params), dp, fp, fp, dp, fp, fp, dp, dp, dp, dp]
            L.or_predict.argtypes = [P(Params), P(State), dp, C.c_int32, C.c_double, P(Prior)]
            L.or_localise.argtypes = [P(Params), P(Prior), P(State), fp, fp, fp, fp, P(State),
                                      P(LocDiag)]
            L.or_fuse.argtypes = [P(Params), dp, dp, dp, dp, dp, fp, fp]
            L.or_fuse.restype = C.c_int64
            L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.or_splitmix64.restype = C.c_uint64
            L.or_sample_pixel.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32]
            L.or_sample_pixel.restype = C.c_uint32
            L.or_adam.argtypes = [P(Params), P(Prior), dp, fp, fp, fp, fp, C.c_uint64, dp, dp]
            L.or_set_threads.argtypes = [C.c_int32]
            L.or_get_threads.restype = C.c_int32
            _lib = L
    return _lib


def params(w, **kw) -> Params:
    """Paper defaults (App. F.2, Tbl. transscales) for workload `w`."""
    p = Params()
    p.nx = p.ny = p.nz = w.n
    p.width, p.height = w.width, w.height
    p.n_gn = kw.pop("n_gn", 10)
    p.voxel = w.voxel
    for a in range(3):
        p.origin[a] = w.origin
    p.fx = p.fy = w.fx
    p.cx, p.cy = w.cx, w.cy
    p.eps = 0.4 * w.voxel
    p.tau = 0.0
    p.max_depth = 0.0
    p.trunc = 2.0 * w.voxel
    p.prior_var = 1e4
    p.init_occ = -0.001
    p.update_var = 1.0
    p.sigma_vel[0], p.sigma_vel[1] = 0.03, 0.03
    p.sigma_pose[0], p.sigma_pose[1] = 0.05, 0.02
    p.b_geo, p.b_rgb = 0.02, 0.1
    p.gate_geo, p.gate_rgb = 0.45, 0.15
    p.floor_geo, p.floor_rgb = 1e-3, 1e-2
    p.ema = 0.8
    p.disc = 0.1
    p.gravity = GRAVITY
    # App. F.2 pose optimiser (used when optimiser = 1)
    p.optimiser = 0
    p.adam_steps, p.adam_pixels = 1000, 200
    p.adam_seed = 0x5EED2212
    p.adam_lr_t, p.adam_lr_r = 1e-3, 3.6e-4
    p.adam_beta2, p.adam_eps = 0.999, 1e-8
    for k, v in kw.items():
        if k in ("origin", "sigma_vel", "sigma_pose"):
            for i, x in enumerate(v):
                getattr(p, k)[i] = x
        else:
            setattr(p, k, v)
    return p


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ wrappers
def set_threads(n: int) -> None:
    """Worker threads of the oracle's loops (n <= 0: every online processor,
    the default).  Results are bit-identical for any thread count."""
    lib().or_set_threads(int(n))


def threads() -> int:
    return int(lib().or_get_threads())


def render(p: Params, occ, rgb, pose7, pix=None):
    """Render at pose7 = (t, q).  Returns dict of depth, rgb, mask, hitk,
    n_samples; per pixel of `pix` (flat indices) if given, else (H, W)."""
    occ = _f64(occ)
    rgb = _f64(rgb)
    pose = _f64(pose7)
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int32)
        n = len(pix)
    else:
        n = p.width * p.height
    depth = np.zeros(n)
    col = np.zeros((n, 3))
    mask = np.zeros(n, np.uint8)
    hitk = np.zeros(n, np.int32)
    ns = np.zeros(1, np.int64)
    lib().or_render(C.byref(p), _p(occ, C.c_double), _p(rgb, C.c_double), _p(pose, C.c_double),
                    _p(pix, C.c_int32), n if pix is not None else 0, _p(depth, C.c_double),
                    _p(col, C.c_double), _p(mask, C.c_uint8), _p(hitk, C.c_int32),
                    _p(ns, C.c_int64))
    out = {"depth": depth, "rgb": col, "mask": mask, "hitk": hitk, "n_samples": int(ns[0])}
    if pix is None:
        out = {k: (v.reshape((p.height, p.width) + v.shape[1:]) if isinstance(v, np.ndarray) else v)
               for k, v in out.items()}
    return out


def render_backward(p: Params, occ, rgb, pose7, g_depth=None, g_rgb=None):
    """Gradients of sum(g_depth * depth) + sum(g_rgb * rgb) for the render at
    pose7: dict of occ (like occ), rgb (like rgb), pose (6: d/dt, d/dtheta for
    a world-frame left perturbation)."""
    occ, rgb, pose = _f64(occ), _f64(rgb), _f64(pose7)
    gd = None if g_depth is None else _f64(g_depth)
    gc = None if g_rgb is None else _f64(g_rgb)
    go = np.zeros_like(occ)
    gr = np.zeros_like(rgb)
    gp = np.zeros(6)
    lib().or_render_backward(C.byref(p), _p(occ, C.c_double), _p(rgb, C.c_double), _p(pose, C.c_double),
                             _p(gd, C.c_double), _p(gc, C.c_double), _p(go, C.c_double), _p(gr, C.c_double),
                             _p(gp, C.c_double))
    return {"occ": go, "rgb": gr, "pose": gp}


def depth_mask(p: Params, depth):
    d = _f32(depth)
    m = np.zeros(d.shape, np.uint8)
    lib().or_depth_mask(C.byref(p), _p(d, C.c_float), _p(m, C.c_uint8))
    return m


def anchor_normals(p: Params, depth):
    d = _f32(depth)
    m = depth_mask(p, d)
    n64 = np.zeros(d.shape + (3,))
    n32 = np.zeros(d.shape + (3,), np.float32)
    nv = np.zeros(d.shape, np.uint8)
    lib().or_anchor_normals(C.byref(p), _p(d, C.c_float), _p(m, C.c_uint8), _p(n64, C.c_double),
                            _p(n32, C.c_float), _p(nv, C.c_uint8))
    return {"mask": m, "n64": n64, "n32": n32, "valid": nv}


def normal_equations(p: Params, anchor_pose, a_depth, a_rgb, pose, o_depth, o_rgb):
    H = np.zeros(36)
    g = np.zeros(6)
    Ht = np.zeros(36)
    st = np.zeros(2)
    ap, cp = _f64(anchor_pose), _f64(pose)
    ad, ar, od, orr = _f32(a_depth), _f32(a_rgb), _f32(o_depth), _f32(o_rgb)
    rc = lib().or_normal_equations(C.byref(p), _p(ap, C.c_double), _p(ad, C.c_float),
                                   _p(ar, C.c_float), _p(cp, C.c_double), _p(od, C.c_float),
                                   _p(orr, C.c_float), _p(H, C.c_double), _p(g, C.c_double),
                                   _p(Ht, C.c_double), _p(st, C.c_double))
    if rc:
        raise RuntimeError(f"or_normal_equations failed: {rc}")
    return {"H": H.reshape(6, 6), "g": g, "Ht": Ht.reshape(6, 6), "cost": st[0], "count": st[1]}


def residuals(p: Params, anchor_pose, a_depth, a_rgb, pose, o_depth, o_rgb):
    """Per-pixel residuals (N, 4), Jacobians (N, 4, 6), association (N, 2), kept (N,)."""
    N = p.width * p.height
    r = np.zeros((N, 4))
    J = np.zeros((N, 4, 6))
    assoc = np.zeros((N, 2), np.int32)
    kept = np.zeros(N, np.uint8)
    ap, cp = _f64(anchor_pose), _f64(pose)
    ad, ar, od, orr = _f32(a_depth), _f32(a_rgb), _f32(o_depth), _f32(o_rgb)
    rc = lib().or_residuals(C.byref(p), _p(ap, C.c_double), _p(ad, C.c_float), _p(ar, C.c_float),
                            _p(cp, C.c_double), _p(od, C.c_float), _p(orr, C.c_float),
                            _p(r, C.c_double), _p(J, C.c_double), _p(assoc, C.c_int32),
                            _p(kept, C.c_uint8))
    if rc:
        raise RuntimeError(f"or_residuals failed: {rc}")
    return {"r": r, "J": J, "assoc": assoc, "kept": kept}


def make_state(pose7, vel6=None, cov=None, n_localised=0) -> State:
    s = State()
    pose7 = np.asarray(pose7, dtype=np.float64)
    for a in range(3):
        s.t[a] = pose7[a]
    for a in range(4):
        s.q[a] = pose7[3 + a]
    vel6 = np.zeros(6) if vel6 is None else np.asarray(vel6, dtype=np.float64)
    for a in range(3):
        s.v[a] = vel6[a]
        s.w[a] = vel6[3 + a]
    cov = np.eye(12) * 1e-8 if cov is None else np.asarray(cov, dtype=np.float64)
    for i in range(144):
        s.cov[i] = cov.flat[i]
    s.n_localised = n_localised
    return s


def state_arrays(s: State):
    return {"pose": np.array(list(s.t) + list(s.q)), "vel": np.array(list(s.v) + list(s.w)),
            "cov": np.array(s.cov[:]).reshape(12, 12), "n_localised": s.n_localised}


def prior_arrays(pr: Prior):
    g = lambda f, k: np.array(getattr(pr, f)[:]).reshape(k)
    return {"pose": np.array(list(pr.t) + list(pr.q)), "vel": np.array(list(pr.v) + list(pr.w)),
            "cov": g("cov", (12, 12)), "cov_pp": g("cov_pp", (6, 6)), "prec_pp": g("prec_pp", (6, 6)),
            "D": g("D", (6, 6)), "cov_vel": g("cov_vel", (6, 6))}


def predict(p: Params, s: State, imu, dt: float) -> Prior:
    imu = _f64(imu if imu is not None and len(imu) else np.zeros((0, 7)))
    pr = Prior()
    rc = lib().or_predict(C.byref(p), C.byref(s), _p(imu, C.c_double) if imu.size else None,
                          imu.shape[0], dt, C.byref(pr))
    if rc:
        raise RuntimeError(f"or_predict failed: {rc}")
    return pr


def localise(p: Params, pr: Prior, prev: State, a_depth, a_rgb, o_depth, o_rgb):
    out = State()
    dg = LocDiag()
    ad, ar, od, orr = _f32(a_depth), _f32(a_rgb), _f32(o_depth), _f32(o_rgb)
    rc = lib().or_localise(C.byref(p), C.byref(pr), C.byref(prev), _p(ad, C.c_float),
                           _p(ar, C.c_float), _p(od, C.c_float), _p(orr, C.c_float), C.byref(out),
                           C.byref(dg))
    if rc:
        raise RuntimeError(f"or_localise failed: {rc}")
    return out, {"cost": dg.cost, "n_pixels": dg.n_pixels, "xi": np.array(dg.xi[:])}


def splitmix64(seed: int, i: int) -> int:
    """Output i (0-based) of SplitMix64 started at state `seed`."""
    return int(lib().or_splitmix64(seed, i))


def sample_pixel(seed: int, i: int, n: int) -> int:
    return int(lib().or_sample_pixel(seed, i, n))


def adam(p: Params, pr: Prior, anchor_pose, a_depth, a_rgb, o_depth, o_rgb, counter0: int = 0,
         trace: bool = False):
    """The paper's pose optimiser from xi = 0 (App. F.2); returns xi, and the
    per-step xi (adam_steps x 6) when trace is set."""
    xi = np.zeros(6)
    tr = np.zeros((p.adam_steps, 6)) if trace else None
    anc = _f64(anchor_pose)
    ad, ar, od, orr = _f32(a_depth), _f32(a_rgb), _f32(o_depth), _f32(o_rgb)
    rc = lib().or_adam(C.byref(p), C.byref(pr), _p(anc, C.c_double), _p(ad, C.c_float), _p(ar, C.c_float),
                       _p(od, C.c_float), _p(orr, C.c_float), counter0, _p(xi, C.c_double), _p(tr, C.c_double))
    if rc:
        raise RuntimeError(f"or_adam failed ({rc})")
    return (xi, tr) if trace else xi


def rollout(p: Params, s: State, windows, dts, occ=None, rgb=None):
    """Predictive rollout from the filter belief (App. I, "Prediction and
    Control"; Fig. 1): each frame applies the transition of `predict`
    (App. E.1/E.2) with no observation, so its prior -- mean and the full
    12x12 covariance over pose and velocity -- is the next frame's state.
    With a map (occ, rgb) each frame also renders the map mean at the
    predicted pose mean (App. B).  windows: one IMU array (n x 7) or None per
    frame; dts: the frame intervals.  Returns the per-frame states (as
    state_arrays dicts) and the per-frame renders (empty without a map)."""
    states, images = [], []
    for imu, dt in zip(windows, dts):
        pr = prior_arrays(predict(p, s, imu, dt))
        s = make_state(pr["pose"], pr["vel"], pr["cov"], s.n_localised)
        states.append(state_arrays(s))
        if occ is not None:
            images.append(render(p, occ, rgb, pr["pose"]))
    return states, images


def map_loss_grad(p: Params, occ, rgb, poses, depths, rgbs, sd: float, sc: float):
    """The rendering loss of gradient-descent mapping (the alternative to the
    closed-form update, Sec. 4.4, Fig. sdfvsvi) and its gradient in the map
    means: sum over frames and over pixels where the render (App. B) hits and
    the observed depth is valid of (d - D)^2 / (2 sd^2) + |c - C|^2 / (2 sc^2),
    the gradient carried to the voxels by the render adjoint; plus the
    Gaussian prior of App. B, sum (mu - mu0)^2 / (2 prior_var).  Returns
    (loss, g_occ, g_rgb)."""
    occ, rgb = _f64(occ), _f64(rgb)
    g_occ, g_rgb = np.zeros_like(occ), np.zeros_like(rgb)
    loss = 0.0
    for pose, D, Cobs in zip(poses, depths, rgbs):
        r = render(p, occ, rgb, pose)
        D = np.asarray(D, dtype=np.float64)
        v = (r["mask"] > 0) & np.isfinite(D) & (D > 0)
        dd = np.where(v, r["depth"] - D, 0.0)
        dc = np.where(v[..., None], r["rgb"] - np.asarray(Cobs, dtype=np.float64), 0.0)
        loss += float(np.sum(dd * dd) / (2 * sd * sd) + np.sum(dc * dc) / (2 * sc * sc))
        b = render_backward(p, occ, rgb, pose, dd / (sd * sd), dc / (sc * sc))
        g_occ += b["occ"]
        g_rgb += b["rgb"]
    v0 = p.prior_var   # prior means: occupancy init_occ, colour 0 (App. F.2)
    loss += float(np.sum((occ - p.init_occ) ** 2) + np.sum(rgb ** 2)) / (2 * v0)
    g_occ += (occ - p.init_occ) / v0
    g_rgb += rgb / v0
    return loss, g_occ, g_rgb


def map_descent(p: Params, occ, rgb, poses, depths, rgbs, sd: float, sc: float, lr_occ: float,
                lr_rgb: float):
    """One step of gradient descent on map_loss_grad's loss:
    mu <- mu - lr g, lr_occ for occupancy and lr_rgb for colour.  Returns
    (occ', rgb', loss before the step)."""
    loss, g_occ, g_rgb = map_loss_grad(p, occ, rgb, poses, depths, rgbs, sd, sc)
    return _f64(occ) - lr_occ * g_occ, _f64(rgb) - lr_rgb * g_rgb, loss


def fuse(p: Params, m: dict, pose7, depth, rgb):
    """In-place FP64 map update; m holds occ, rgb, var_occ, var_rgb (float64)."""
    for k in ("occ", "rgb", "var_occ", "var_rgb"):
        assert m[k].dtype == np.float64 and m[k].flags.c_contiguous
    pose = _f64(pose7)
    d, c = _f32(depth), _f32(rgb)
    n = lib().or_fuse(C.byref(p), _p(m["occ"], C.c_double), _p(m["rgb"], C.c_double),
                      _p(m["var_occ"], C.c_double), _p(m["var_rgb"], C.c_double),
                      _p(pose, C.c_double), _p(d, C.c_float), _p(c, C.c_float))
    if n < 0:
        raise RuntimeError("or_fuse failed")
    return int(n)


def map64(occ, rgb, var_occ, var_rgb) -> dict:
    return {"occ": _f64(occ), "rgb": _f64(rgb), "var_occ": _f64(var_occ), "var_rgb": _f64(var_rgb)}


class Filter:
    """The oracle's filter over a sequence of frames (Sec. 3.3, App. F)."""

    def __init__(self, p: Params, map_arrays, s1: State):
        self.p = p
        self.m = map64(*map_arrays)
        self.s = s1
        self.anchor = None
        self.t = 0

    def step(self, depth, rgb, imu=None, dt=None):
        if self.t > 0:
            prior = predict(self.p, self.s, imu, dt)
            self.s, self.diag = localise(self.p, prior, self.s, self.anchor["depth"],
                                         self.anchor["rgb"], depth, rgb)
            self.prior = prior
        pose = np.array(list(self.s.t) + list(self.s.q))
        self.n_upd = fuse(self.p, self.m, pose, depth, rgb)
        r = render(self.p, self.m["occ"], self.m["rgb"], pose)
        # the anchor is the rendered observation, stored as the device stores it (FP32)
        self.anchor = {"depth": r["depth"].astype(np.float32), "rgb": r["rgb"].astype(np.float32),
                       "pose": pose, "n_samples": r["n_samples"]}
        self.t += 1
        return self.s
