"""torch.autograd binding of the trajectory loss (Sec. III-B / III-C, Eq. 1-4).

The forward runs dc_loss_traj without the gradient and keeps only the nearest-neighbour
indices; the backward calls dc_loss_traj_bwd, which recomputes the sampled points from the
stored draws instead of storing them.
"""
from __future__ import annotations

import torch

from . import _lib


class DCLoss(torch.autograd.Function):
    """(L_total, loss_frames): L_total = sum_t w_t L_t and L_t(verts[t]), both computed by the
    library; differentiable with respect to verts only. Frames whose entry of frame_w is 0
    are skipped (their L_t is reported as the constant 0 and gets no gradient)."""

    @staticmethod
    def forward(ctx, verts, faces, draws, targets, mode=_lib.BIDIR_MEAN, face_mask=None,
                frame_w=None):
        verts = verts.detach().contiguous()
        r = _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode, grad=False, total=True,
                              nn=True, face_mask=face_mask, frame_w=frame_w)
        ctx.mode = mode
        ctx.face_mask = face_mask
        ctx.frame_w = frame_w
        ctx.set_materialize_grads(False)
        nn_ba = r["nn_ba"] if r["nn_ba"] is not None else r["nn_ab"]
        ctx.save_for_backward(verts, faces, draws, targets, r["nn_ab"], nn_ba)
        return r["loss_total"].reshape(()), r["loss_frames"]

    @staticmethod
    def backward(ctx, grad_total, grad_frames):
        verts, faces, draws, targets, nn_ab, nn_ba = ctx.saved_tensors
        if grad_total is None and grad_frames is None:
            return None, None, None, None, None, None, None
        # the library forms g_t = w_t grad_total + grad_frames[t] itself
        gt = None if grad_total is None else grad_total.detach().reshape(1).float().contiguous()
        gf = None if grad_frames is None else grad_frames.detach().float().contiguous()
        g = _lib.dc_loss_traj_bwd(verts, faces, draws, targets, nn_ab,
                                  nn_ba if ctx.mode == _lib.BIDIR_MEAN else None, gf,
                                  mode=ctx.mode, face_mask=ctx.face_mask, frame_w=ctx.frame_w,
                                  grad_total=gt)
        return g, None, None, None, None, None, None


def loss_traj(verts, faces, draws, targets, mode=_lib.BIDIR_MEAN, frame_w=None,
              face_mask=None):
    """Differentiable sum_t w_t L_t (w_t = 1 by default) and the per-frame losses, both from
    the library. face_mask [F] (optional): sample only the faces with a nonzero entry. Frames
    of weight 0 do no work in either direction (their L_t is reported as 0)."""
    fw = None
    if frame_w is not None:
        fw = torch.as_tensor(frame_w, dtype=torch.float32, device=verts.device).contiguous()
    return DCLoss.apply(verts, faces, draws, targets, mode, face_mask, fw)


class DiffCloudLoss(torch.nn.Module):
    """The loss as a module: loss(verts) -> (sum_t w_t L_t, per-frame L_t), differentiable in
    verts [T, V, 3]. Every call draws fresh samples (n per frame, from its own seeded
    generator), as a sampler inside an optimisation loop does; the draws of the last call
    are kept in `last_draws`.

    faces [F, 3] int32, targets [T, M, 3] float32 on the device; mode BIDIR_MEAN (Eq. 1) or
    UNIDIR_SUM (Eq. 2); frame_w [T] optional (frames of weight 0 cost nothing); face_mask [F]
    optional (sample only these faces)."""

    def __init__(self, faces, targets, n: int, mode=_lib.BIDIR_MEAN, frame_w=None,
                 face_mask=None, seed: int = 0):
        super().__init__()
        self.faces, self.targets, self.n, self.mode = faces, targets, int(n), mode
        self.frame_w, self.face_mask = frame_w, face_mask
        self.gen = torch.Generator(device="cpu").manual_seed(seed)
        self.last_draws = None

    def forward(self, verts):
        T = verts.shape[0]
        draws = torch.rand((T, self.n, 3), generator=self.gen).clamp_(max=1 - 2 ** -24)
        self.last_draws = draws.to(verts.device)
        return loss_traj(verts.float().contiguous(), self.faces, self.last_draws, self.targets,
                         mode=self.mode, frame_w=self.frame_w, face_mask=self.face_mask)
