"""Seeded analytic scenes: a closed room with axis-aligned boxes and spheres.

The scene is exact geometry, independent of any voxel map: frames are made
by intersecting camera rays with the primitives analytically, and a
"settled" voxel map (the map a long run of the filter converges to) is made
by sampling the scene's signed distance at voxel centres.  Neither uses any
part of the filter's own rendering or map-update arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .configs import Workload


@dataclass
class Patch:
    wall: int             # 0..5: -x, +x, -y, +y, -z, +z
    lo: np.ndarray        # (2,) in-plane lower corner (plane coords a, b)
    size: float
    colours: np.ndarray   # (8, 8, 3)


@dataclass
class Scene:
    lo: np.ndarray        # room interior lower corner
    hi: np.ndarray        # room interior upper corner
    wall_albedo: np.ndarray            # (6, 3)
    boxes_c: np.ndarray                # (nb, 3)
    boxes_h: np.ndarray                # (nb, 3) half extents
    boxes_albedo: np.ndarray           # (nb, 3)
    spheres_c: np.ndarray              # (ns, 3)
    spheres_r: np.ndarray              # (ns,)
    spheres_albedo: np.ndarray         # (ns, 3)
    patches: list = field(default_factory=list)

    # ----------------------------------------------------------------- colour
    def wall_colour(self, wall: np.ndarray, pts: np.ndarray) -> np.ndarray:
        """Albedo of wall points; `wall` gives the wall id of each point."""
        col = self.wall_albedo[wall].copy()
        axes = {0: (1, 2), 1: (1, 2), 2: (0, 2), 3: (0, 2), 4: (0, 1), 5: (0, 1)}
        for p in self.patches:
            sel = np.nonzero(wall == p.wall)[0]
            if sel.size == 0:
                continue
            a, b = axes[p.wall]
            ua = (pts[sel, a] - p.lo[0]) / p.size
            ub = (pts[sel, b] - p.lo[1]) / p.size
            inside = (ua >= 0) & (ua < 1) & (ub >= 0) & (ub < 1)
            ia = np.clip((ua[inside] * 8).astype(np.int64), 0, 7)
            ib = np.clip((ub[inside] * 8).astype(np.int64), 0, 7)
            col[sel[inside]] = p.colours[ia, ib]
        return col


def make_scene(w: Workload, rng: np.random.Generator, keep_clear: np.ndarray,
               clearance: float = 0.35) -> Scene:
    """Room filling the map cube up to a 3-voxel margin, plus w.n_prims
    primitives (sizes 0.2-1 m) kept `clearance` metres away from every
    point in `keep_clear` (the trajectory)."""
    m = 3.0 * w.voxel
    lo = np.full(3, w.origin + m)
    hi = np.full(3, w.origin + w.extent - m)
    wall_albedo = rng.uniform(0.2, 0.9, size=(6, 3))
    bc, bh, ba, sc, sr, sa = [], [], [], [], [], []
    tries = 0
    while len(bc) + len(sc) < w.n_prims and tries < 100000:
        tries += 1
        c = rng.uniform(lo, hi)
        alb = rng.uniform(0.05, 0.95, size=3)
        if rng.uniform() < 0.5:
            h = 0.5 * rng.uniform(0.2, 1.0, size=3)
            q = np.abs(keep_clear - c[None]) - h[None]
            d = np.linalg.norm(np.maximum(q, 0), axis=1) + np.minimum(q.max(axis=1), 0)
            if d.min() < clearance:
                continue
            bc.append(c); bh.append(h); ba.append(alb)
        else:
            r = 0.5 * rng.uniform(0.2, 1.0)
            d = np.linalg.norm(keep_clear - c[None], axis=1) - r
            if d.min() < clearance:
                continue
            sc.append(c); sr.append(r); sa.append(alb)
    patches = []
    if w.textured:
        axes = {0: (1, 2), 1: (1, 2), 2: (0, 2), 3: (0, 2), 4: (0, 1), 5: (0, 1)}
        for wall in range(6):
            a, b = axes[wall]
            for _ in range(6):
                size = rng.uniform(0.5, 1.2)
                plo = np.array([rng.uniform(lo[a], hi[a] - size), rng.uniform(lo[b], hi[b] - size)])
                patches.append(Patch(wall, plo, size, rng.uniform(0.0, 1.0, size=(8, 8, 3))))
    f = lambda x, k: np.array(x, dtype=np.float64).reshape(-1, k) if len(x) else np.zeros((0, k))
    return Scene(lo, hi, wall_albedo, f(bc, 3), f(bh, 3), f(ba, 3), f(sc, 3),
                 np.array(sr, dtype=np.float64), f(sa, 3), patches)


# ------------------------------------------------------------------ ray cast
def raycast(scene: Scene, w: Workload, R: np.ndarray, t: np.ndarray):
    """Exact z-depth and albedo for every pixel of a W x H pinhole camera at
    pose (R, t).  Rays are parameterised by camera-frame z-depth s:
    X(s) = t + s * R (x_n, y_n, 1), so the hit parameter is the z-depth."""
    u = np.arange(w.width, dtype=np.float64)
    v = np.arange(w.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - w.cx) / w.fx, (vv - w.cy) / w.fx, np.ones_like(uu)], axis=-1).reshape(-1, 3)
    d = dc @ R.T
    o = np.asarray(t, dtype=np.float64)
    n = d.shape[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        # room: exit distance from inside the box
        t_hi = (scene.hi[None] - o[None]) * inv
        t_lo = (scene.lo[None] - o[None]) * inv
        t_exit = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
        axis = np.argmin(t_exit, axis=1)
        best = t_exit[np.arange(n), axis]
        wall = 2 * axis + (d[np.arange(n), axis] > 0)
        kind = np.zeros(n, dtype=np.int64)          # 0 wall, 1 box, 2 sphere
        ident = wall.astype(np.int64)
        for i in range(scene.boxes_c.shape[0]):
            lo = scene.boxes_c[i] - scene.boxes_h[i]
            hi = scene.boxes_c[i] + scene.boxes_h[i]
            t1 = (lo[None] - o[None]) * inv
            t2 = (hi[None] - o[None]) * inv
            tn = np.nanmax(np.minimum(t1, t2), axis=1)
            tf = np.nanmin(np.maximum(t1, t2), axis=1)
            hit = (tn <= tf) & (tn > 0) & (tn < best)
            best = np.where(hit, tn, best)
            kind = np.where(hit, 1, kind)
            ident = np.where(hit, i, ident)
        for i in range(scene.spheres_c.shape[0]):
            oc = o - scene.spheres_c[i]
            a = np.einsum("ij,ij->i", d, d)
            b = 2.0 * d @ oc
            c = oc @ oc - scene.spheres_r[i] ** 2
            disc = b * b - 4 * a * c
            s = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
            hit = (disc >= 0) & (s > 0) & (s < best)
            best = np.where(hit, s, best)
            kind = np.where(hit, 2, kind)
            ident = np.where(hit, i, ident)
    pts = o[None] + best[:, None] * d
    col = np.zeros((n, 3))
    sel = kind == 0
    col[sel] = scene.wall_colour(ident[sel], pts[sel])
    sel = kind == 1
    col[sel] = scene.boxes_albedo[ident[sel]]
    sel = kind == 2
    col[sel] = scene.spheres_albedo[ident[sel]]
    depth = np.where(np.isfinite(best), best, 0.0)
    return depth.reshape(w.height, w.width), col.reshape(w.height, w.width, 3)


# --------------------------------------------------------------- settled map
def settled_map(scene: Scene, w: Workload, trunc_vox: float = 2.0,
                var_seen: float = 0.1, prior_var: float = 1e4, prior_occ: float = -0.001):
    """A voxel map as a long run of observation would leave it.

    occ  = -clamp(sdf, -trunc, trunc) where sdf >= -trunc (free space and the
           band behind each surface), the prior mean elsewhere;
    rgb  = albedo of the nearest surface where |sdf| <= trunc, 0 elsewhere;
    var  = var_seen where the value was set, the prior variance elsewhere.
    Returns float32 arrays occ (n,n,n), rgb (n,n,n,3), var_occ, var_rgb,
    indexed [k, j, i] (z, y, x)."""
    n = w.n
    vs = w.voxel
    trunc = trunc_vox * vs
    cen = w.origin + (np.arange(n) + 0.5) * vs
    Z, Y, X = np.meshgrid(cen, cen, cen, indexing="ij")
    # room: distance to the nearest wall, positive inside
    dl = np.stack([X - scene.lo[0], scene.hi[0] - X, Y - scene.lo[1], scene.hi[1] - Y,
                   Z - scene.lo[2], scene.hi[2] - Z]).astype(np.float32)
    wall = np.argmin(dl, axis=0)
    sdf = np.take_along_axis(dl, wall[None], axis=0)[0]
    del dl
    outside = (X < scene.lo[0]) | (X > scene.hi[0]) | (Y < scene.lo[1]) | (Y > scene.hi[1]) | \
              (Z < scene.lo[2]) | (Z > scene.hi[2])
    qx = np.maximum(np.maximum(scene.lo[0] - X, X - scene.hi[0]), 0)
    qy = np.maximum(np.maximum(scene.lo[1] - Y, Y - scene.hi[1]), 0)
    qz = np.maximum(np.maximum(scene.lo[2] - Z, Z - scene.hi[2]), 0)
    sdf = np.where(outside, -np.sqrt(qx * qx + qy * qy + qz * qz), sdf).astype(np.float32)
    owner = np.full((n, n, n), -1, dtype=np.int64)        # -1 wall, >=0 primitive
    prim_alb = []

    def box_of(lo_w, hi_w):
        a = np.clip(np.floor((lo_w - w.origin) / vs - 0.5).astype(int) - 1, 0, n)
        b = np.clip(np.ceil((hi_w - w.origin) / vs - 0.5).astype(int) + 2, 0, n)
        return a, b

    pid = 0
    for i in range(scene.boxes_c.shape[0]):
        c, h = scene.boxes_c[i], scene.boxes_h[i]
        a, b = box_of(c - h - trunc, c + h + trunc)
        sl = np.s_[a[2]:b[2], a[1]:b[1], a[0]:b[0]]
        q = np.stack([np.abs(X[sl] - c[0]) - h[0], np.abs(Y[sl] - c[1]) - h[1],
                      np.abs(Z[sl] - c[2]) - h[2]])
        d = np.sqrt(np.sum(np.maximum(q, 0) ** 2, axis=0)) + np.minimum(q.max(axis=0), 0)
        closer = d < sdf[sl]
        sdf[sl] = np.where(closer, d, sdf[sl])
        owner[sl] = np.where(closer, pid, owner[sl])
        prim_alb.append(scene.boxes_albedo[i]); pid += 1
    for i in range(scene.spheres_c.shape[0]):
        c, r = scene.spheres_c[i], scene.spheres_r[i]
        a, b = box_of(c - r - trunc, c + r + trunc)
        sl = np.s_[a[2]:b[2], a[1]:b[1], a[0]:b[0]]
        d = np.sqrt((X[sl] - c[0]) ** 2 + (Y[sl] - c[1]) ** 2 + (Z[sl] - c[2]) ** 2) - r
        closer = d < sdf[sl]
        sdf[sl] = np.where(closer, d, sdf[sl])
        owner[sl] = np.where(closer, pid, owner[sl])
        prim_alb.append(scene.spheres_albedo[i]); pid += 1
    seen = sdf >= -trunc
    band = np.abs(sdf) <= trunc
    occ = np.where(seen, -np.clip(sdf, -trunc, trunc), prior_occ).astype(np.float32)
    var_occ = np.where(seen, var_seen, prior_var).astype(np.float32)
    var_rgb = np.where(band, var_seen, prior_var).astype(np.float32)
    rgb = np.zeros((n, n, n, 3), dtype=np.float32)
    idx = np.nonzero(band)
    own = owner[idx]
    pts = np.stack([X[idx], Y[idx], Z[idx]], axis=1)
    col = np.zeros((len(own), 3))
    isw = own < 0
    if np.any(isw):
        col[isw] = scene.wall_colour(wall[idx][isw], pts[isw])
    if np.any(~isw):
        col[~isw] = np.asarray(prim_alb)[own[~isw]]
    rgb[idx] = col.astype(np.float32)
    return occ, rgb, var_occ, var_rgb
