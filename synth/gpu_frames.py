"""Batch generation of the synthetic RGB-D frames with torch on a GPU.

The same analytic ray cast as synth.scene.raycast (exact ray / box /
sphere / room intersections, wall checker patches, additive Gaussian noise),
vectorised over all pixels of a frame in torch so that a benchmark can make
hundreds of 640x480 frames in seconds.  Values agree with the numpy cast to
float rounding; the noise comes from a seeded torch generator, so these
frames are not bit-identical to Sequence.frame (tests use the numpy path).
"""
from __future__ import annotations

import torch

from ._rot import matrix_from_quat


def _wall_colour(scene, wall, pts, col):
    axes = {0: (1, 2), 1: (1, 2), 2: (0, 2), 3: (0, 2), 4: (0, 1), 5: (0, 1)}
    for p in scene.patches:
        a, b = axes[p.wall]
        ua = (pts[:, a] - float(p.lo[0])) / p.size
        ub = (pts[:, b] - float(p.lo[1])) / p.size
        inside = (wall == p.wall) & (ua >= 0) & (ua < 1) & (ub >= 0) & (ub < 1)
        ia = torch.clamp((ua * 8).long(), 0, 7)
        ib = torch.clamp((ub * 8).long(), 0, 7)
        pc = torch.as_tensor(p.colours, dtype=pts.dtype, device=pts.device)[ia, ib]
        col = torch.where(inside[:, None], pc, col)
    return col


@torch.no_grad()
def raycast_frames(seq, indices, device, noise: bool = True, seed: int = 0):
    """Frames `indices` of a synth.Sequence as (depth (n, H, W), rgb (n, H, W, 3))
    float32 tensors on `device`."""
    w, scene = seq.w, seq.scene
    dt = torch.float64
    u = torch.arange(w.width, device=device, dtype=dt)
    v = torch.arange(w.height, device=device, dtype=dt)
    vv, uu = torch.meshgrid(v, u, indexing="ij")
    dc = torch.stack([(uu - w.cx) / w.fx, (vv - w.cy) / w.fx, torch.ones_like(uu)], -1).reshape(-1, 3)
    lo_r = torch.as_tensor(scene.lo, dtype=dt, device=device)
    hi_r = torch.as_tensor(scene.hi, dtype=dt, device=device)
    wall_alb = torch.as_tensor(scene.wall_albedo, dtype=dt, device=device)
    bc = torch.as_tensor(scene.boxes_c, dtype=dt, device=device)
    bh = torch.as_tensor(scene.boxes_h, dtype=dt, device=device)
    ba = torch.as_tensor(scene.boxes_albedo, dtype=dt, device=device)
    sc = torch.as_tensor(scene.spheres_c, dtype=dt, device=device)
    sr = torch.as_tensor(scene.spheres_r, dtype=dt, device=device)
    sa = torch.as_tensor(scene.spheres_albedo, dtype=dt, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seq.seed) * 7919 + seed)
    depths, rgbs = [], []
    for i in indices:
        t, q = seq.pose(i)
        R = torch.as_tensor(matrix_from_quat(q), dtype=dt, device=device)
        o = torch.as_tensor(t, dtype=dt, device=device)
        d = dc @ R.T
        n = d.shape[0]
        inv = 1.0 / d
        t_hi = (hi_r - o) * inv
        t_lo = (lo_r - o) * inv
        t_exit = torch.where(d > 0, t_hi, torch.where(d < 0, t_lo, torch.full_like(d, float("inf"))))
        best, axis = torch.min(t_exit, dim=1)
        ar = torch.arange(n, device=device)
        wall = 2 * axis + (d[ar, axis] > 0).long()
        col = wall_alb[wall]
        is_wall = torch.ones(n, dtype=torch.bool, device=device)
        for k in range(bc.shape[0]):
            t1 = (bc[k] - bh[k] - o) * inv
            t2 = (bc[k] + bh[k] - o) * inv
            tn = torch.nan_to_num(torch.minimum(t1, t2), nan=-float("inf")).amax(1)
            tf = torch.nan_to_num(torch.maximum(t1, t2), nan=float("inf")).amin(1)
            hit = (tn <= tf) & (tn > 0) & (tn < best)
            best = torch.where(hit, tn, best)
            col = torch.where(hit[:, None], ba[k].expand(n, 3), col)
            is_wall = is_wall & ~hit
        for k in range(sc.shape[0]):
            oc = o - sc[k]
            a = (d * d).sum(1)
            b = 2.0 * d @ oc
            c = oc @ oc - sr[k] ** 2
            disc = b * b - 4 * a * c
            s = (-b - torch.sqrt(torch.clamp(disc, min=0))) / (2 * a)
            hit = (disc >= 0) & (s > 0) & (s < best)
            best = torch.where(hit, s, best)
            col = torch.where(hit[:, None], sa[k].expand(n, 3), col)
            is_wall = is_wall & ~hit
        pts = o + best[:, None] * d
        wcol = _wall_colour(scene, wall, pts, col)
        col = torch.where(is_wall[:, None], wcol, col)
        depth = torch.where(torch.isfinite(best), best, torch.zeros_like(best))
        if noise:
            valid = depth > 0
            depth = torch.where(valid, depth + w.depth_sigma * torch.randn(n, generator=gen, device=device,
                                                                              dtype=dt), depth)
            col = col + w.rgb_sigma * torch.randn(n, 3, generator=gen, device=device, dtype=dt)
        depths.append(depth.reshape(w.height, w.width).float())
        rgbs.append(col.reshape(w.height, w.width, 3).float())
    return torch.stack(depths), torch.stack(rgbs)


__all__ = ["raycast_frames"]
