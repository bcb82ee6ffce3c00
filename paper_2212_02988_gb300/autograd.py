"""The render as a torch.autograd.Function (App. B: the emission is
differentiable), over libprism.so's forward and hand-written adjoint.

    depth, rgb = render(pose7, occ, rgb_map, filt)

pose7 is a CPU float64 tensor (t, q); occ (nz, ny, nx) and rgb_map
(nz, ny, nx, 3) are CUDA float32 tensors that become the means of filt's
map (its variances are left as they are), so give it a Filter of its own
(not one that tracks a sequence).  The map is loaded only when it has to
be: when occ or rgb_map is another tensor or has been modified in place
since it was loaded, or when filt's map was changed in between (a step,
update or load).  So a forward and its backward load it once, and a
training loop that updates the map in place loads it once per iteration.
Backward re-marches the rays (nothing is stored) and returns gradients for
pose7 (with respect to t and the quaternion as given), occ and rgb_map.
The hit sample of each ray is held fixed, as for any first-hit renderer.
"""
from __future__ import annotations

import numpy as np
import torch


def _ensure_map(filt, occ, rgb_map):
    """Load (occ, rgb_map) into filt unless they are already its map."""
    key = (occ.data_ptr(), occ._version, rgb_map.data_ptr(), rgb_map._version, tuple(occ.shape))
    if getattr(filt, "_autograd_map", None) == (filt.map_version, key):
        return False
    filt.map_load(occ.detach().contiguous(), rgb_map.detach().contiguous())
    filt._autograd_map = (filt.map_version, key)
    return True


class PrismRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pose7, occ, rgb_map, filt):
        _ensure_map(filt, occ, rgb_map)
        out = filt.render(pose7.detach().cpu().double().numpy(), mask=None, hitk=None, alloc=False,
                          depth=torch.empty((filt.H, filt.W), device=occ.device),
                          rgb=torch.empty((filt.H, filt.W, 3), device=occ.device))
        ctx.filt = filt
        ctx.save_for_backward(pose7, occ, rgb_map)
        return out["depth"], out["rgb"]

    @staticmethod
    def backward(ctx, g_depth, g_rgb):
        pose7, occ, rgb_map = ctx.saved_tensors
        filt = ctx.filt
        # the map as it was at forward time (reloaded only if filt has held another since)
        _ensure_map(filt, occ, rgb_map)
        go = torch.zeros_like(occ) if ctx.needs_input_grad[1] else None
        gr = torch.zeros_like(rgb_map) if ctx.needs_input_grad[2] else None
        _, g7 = filt.render_backward(pose7.detach().cpu().double().numpy(),
                                     None if g_depth is None else g_depth.contiguous(),
                                     None if g_rgb is None else g_rgb.contiguous(), go, gr)
        gp = torch.from_numpy(np.asarray(g7)).to(pose7.dtype) if ctx.needs_input_grad[0] else None
        return gp, go, gr, None


def render(pose7, occ, rgb_map, filt):
    return PrismRender.apply(pose7, occ, rgb_map, filt)
