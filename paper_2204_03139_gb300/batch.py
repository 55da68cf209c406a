"""Batched loss over many trajectories of uneven sizes (one launch sequence, CUDA graph).

Every frame of every trajectory becomes one dc_frame; dc_batch_plan lays them out in one
workspace, and dc_batch_run issues the whole sequence -- area CDFs, sampling, ONE persistent
Chamfer launch whose work split covers all frames, neighbour recovery, losses and the vertex
gradients -- reading only device memory, so it can be replayed from a CUDA graph.

The plain per-frame form (`per_frame_loss`) is the comparison point: the same kernels, one
dc_loss_traj call per frame, no graph.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class DeviceTrajectory:
    """Device tensors of one trajectory. Frames may be ragged: draws and targets are flat
    [sum_t N_t, 3] / [sum_t M_t, 3] with host offsets n_off / m_off ([T+1])."""

    verts: torch.Tensor    # [T, V, 3] float32
    faces: torch.Tensor    # [F, 3] int32
    draws: torch.Tensor    # [sum N_t, 3] float32
    targets: torch.Tensor  # [sum M_t, 3] float32
    n_off: np.ndarray
    m_off: np.ndarray
    face_mask: torch.Tensor | None = None  # [F] uint8: sample only faces with a nonzero entry

    @property
    def T(self):
        return int(self.verts.shape[0])

    @staticmethod
    def from_host(tr, device) -> "DeviceTrajectory":
        return DeviceTrajectory(torch.from_numpy(tr.verts).to(device),
                                torch.from_numpy(tr.faces).to(device),
                                torch.from_numpy(tr.draws).to(device),
                                torch.from_numpy(tr.targets).to(device),
                                np.asarray(tr.n_off, np.int64), np.asarray(tr.m_off, np.int64),
                                _device_mask(getattr(tr, "face_mask", None), device))

    def pairs(self) -> int:
        return int(np.sum(np.diff(self.n_off) * np.diff(self.m_off)))


def _device_mask(m, device):
    return None if m is None else torch.from_numpy(np.ascontiguousarray(m, np.uint8)).to(device)


# numpy view of the C struct dc_frame (include/diffcloud.h), 96 bytes per frame
FRAME_DTYPE = np.dtype([("verts", "u8"), ("faces", "u8"), ("face_mask", "u8"), ("draws", "u8"),
                        ("targets", "u8"),
                        ("V", "i4"), ("F", "i4"), ("N", "i4"), ("M", "i4"), ("weight", "f4"),
                        ("tag", "i4"), ("loss", "u8"), ("grad_verts", "u8"), ("nn_ab", "u8"),
                        ("nn_ba", "u8")])
assert FRAME_DTYPE.itemsize == ctypes.sizeof(_lib.dc_frame)
for _name, _ in _lib.dc_frame._fields_:
    assert FRAME_DTYPE.fields[_name][1] == getattr(_lib.dc_frame, _name).offset


class BatchedLoss:
    """Loss (and vertex gradients) of a list of trajectories in one planned launch sequence.

    After run(): loss_frames[k] [T_k] and grad_verts[k] [T_k, V_k, 3] hold each trajectory's
    per-frame losses and gradients (gradient of sum_t w_t L_t), and the returned tensor is the
    weighted total over all trajectories.
    """

    def __init__(self, trajs, mode=_lib.BIDIR_MEAN, weights=None, grad=True, graph=False,
                 nn=False, stream=None, tune=False, shape=None, outputs=None,
                 async_plan=False):
        """tune=True: plan with the shape the autotuner found fastest for this batch's size
        bucket (timing every shape first if the bucket has no entry); shape: plan with this
        shape (autotune.SHAPES); otherwise the library's default. outputs: per trajectory a
        (loss_frames [T], grad_verts [T, V, 3] or None) pair of device tensors to write into
        instead of new ones. async_plan: upload the plan from pinned staging memory without
        waiting for the stream (the staging stays referenced by this object)."""
        from . import autotune

        self.trajs = list(trajs)
        self.mode = mode
        dev = self.trajs[0].verts.device
        self.device = dev
        # the stream the plan is uploaded on and the batch runs on (default: current stream)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        if tune and shape is None:
            shape = autotune.best_batch(self.trajs, mode, dev)
            if shape is None:
                shape = autotune.tune_batch(self.trajs, mode=mode, weights=weights,
                                            grad=grad)["best"]
        self.shape = shape
        # outputs and workspace belong to the batch's stream (the caching allocator reuses
        # memory per stream); the plan keeps the shape it was made with
        with torch.cuda.stream(self.stream), autotune.tuned(shape):
            self._build(mode, weights, grad, nn, outputs, async_plan)
        if graph:
            self._capture()

    def _build(self, mode, weights, grad, nn, outputs=None, async_plan=False):
        dev = self.device
        nfr = sum(t.T for t in self.trajs)
        # the dc_frame table, filled column by column (one row per frame)
        tab = np.zeros(nfr, dtype=FRAME_DTYPE)
        self.loss_frames, self.grad_verts, self.nn_ab, self.nn_ba = [], [], [], []
        k = 0
        for i, tr in enumerate(self.trajs):
            T, V, F = tr.T, int(tr.verts.shape[1]), int(tr.faces.shape[0])
            if outputs is not None and outputs[i] is not None:
                lf, gv = outputs[i]
                if lf.dtype != torch.float32 or tuple(lf.shape) != (T,) or not lf.is_contiguous():
                    raise ValueError("outputs: loss_frames must be a contiguous [T] float32 tensor")
                if grad and (gv is None or tuple(gv.shape) != (T, V, 3) or
                             gv.dtype != torch.float32 or not gv.is_contiguous()):
                    raise ValueError("outputs: grad_verts must be a contiguous [T, V, 3] "
                                     "float32 tensor")
            else:
                lf = torch.empty(T, dtype=torch.float32, device=dev)
                gv = torch.empty((T, V, 3), dtype=torch.float32, device=dev) if grad else None
            nab = torch.empty(int(tr.n_off[-1]), dtype=torch.int32, device=dev) if nn else None
            nba = (torch.empty(int(tr.m_off[-1]), dtype=torch.int32, device=dev)
                   if nn and mode == _lib.BIDIR_MEAN else None)
            self.loss_frames.append(lf)
            self.grad_verts.append(gv)
            self.nn_ab.append(nab)
            self.nn_ba.append(nba)
            n_off = np.asarray(tr.n_off, np.int64)
            m_off = np.asarray(tr.m_off, np.int64)
            t = np.arange(T, dtype=np.int64)
            row = tab[k:k + T]
            row["verts"] = tr.verts.data_ptr() + 12 * V * t
            row["faces"] = tr.faces.data_ptr()
            if tr.face_mask is not None:
                if tr.face_mask.dtype != torch.uint8 or tr.face_mask.numel() != F:
                    raise ValueError("face_mask must be a uint8 tensor with one entry per face")
                row["face_mask"] = tr.face_mask.data_ptr()
            row["draws"] = tr.draws.data_ptr() + 12 * n_off[:-1]
            row["targets"] = tr.targets.data_ptr() + 12 * m_off[:-1]
            row["V"], row["F"] = V, F
            row["N"] = np.diff(n_off)
            row["M"] = np.diff(m_off)
            row["weight"] = 1.0 if weights is None or weights[i] is None else weights[i]
            row["tag"] = i
            row["loss"] = lf.data_ptr() + 4 * t
            if grad:
                row["grad_verts"] = gv.data_ptr() + 12 * V * t
            if nab is not None:
                row["nn_ab"] = nab.data_ptr() + 4 * n_off[:-1]
            if nba is not None:
                row["nn_ba"] = nba.data_ptr() + 4 * m_off[:-1]
            k += T
        self._table = tab
        self.frames = tab.ctypes.data_as(ctypes.POINTER(_lib.dc_frame))
        L = _lib.lib()
        nb = int(L.dc_batch_workspace_size(self.frames, nfr))
        if nb == 0:
            raise _lib.DCError(_lib.DC_EINVAL, "bad batch sizes")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.total = torch.empty(1, dtype=torch.float32, device=dev)
        self.workspace_bytes = nb
        self.n_frames = nfr
        if async_plan:
            sb = int(L.dc_batch_plan_bytes(self.frames, nfr, mode))
            if sb == 0:
                raise _lib.DCError(_lib.DC_EINVAL, "bad batch sizes")
            self._staging = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
            _lib._check(L.dc_batch_plan_async(self.frames, nfr, mode,
                                              ctypes.c_void_p(self.ws.data_ptr()), nb,
                                              ctypes.c_void_p(self._staging.data_ptr()), sb,
                                              ctypes.c_void_p(self.stream.cuda_stream)))
        else:
            _lib._check(L.dc_batch_plan(self.frames, nfr, mode,
                                        ctypes.c_void_p(self.ws.data_ptr()), nb,
                                        ctypes.c_void_p(self.stream.cuda_stream)))
        self.graph = None

    def _launch(self):
        _lib._check(_lib.lib().dc_batch_run(ctypes.c_void_p(self.ws.data_ptr()),
                                            ctypes.c_void_p(self.total.data_ptr()),
                                            ctypes.c_void_p(self.stream.cuda_stream)))

    def _capture(self):
        # one eager run first: per-device one-time set-up happens outside the capture
        self._launch()
        torch.cuda.synchronize(self.device)
        s = torch.cuda.Stream(self.device)
        s.wait_stream(self.stream)
        g = torch.cuda.CUDAGraph()
        launch_stream = self.stream
        self.stream = s
        try:
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    self._launch()
        finally:
            self.stream = launch_stream
        self.stream.wait_stream(s)
        self.graph = g

    def run(self, check: bool = False) -> torch.Tensor:
        if self.graph is not None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
        else:
            self._launch()
        if check:
            _lib.check_ws(self.ws)
        return self.total

    def pairs(self) -> int:
        return sum(t.pairs() for t in self.trajs)


def per_frame_loss(trajs, mode=_lib.BIDIR_MEAN, grad=True):
    """The plain per-frame form: one dc_loss_traj call per frame, no graph, one stream.
    Returns (per-trajectory loss_frames, per-trajectory grad_verts)."""
    losses, grads = [], []
    for tr in trajs:
        T, V = tr.T, int(tr.verts.shape[1])
        lf = torch.empty(T, dtype=torch.float32, device=tr.verts.device)
        gv = torch.empty((T, V, 3), dtype=torch.float32, device=tr.verts.device) if grad else None
        for t in range(T):
            n0, n1 = int(tr.n_off[t]), int(tr.n_off[t + 1])
            m0, m1 = int(tr.m_off[t]), int(tr.m_off[t + 1])
            out = {"loss_frames": lf[t:t + 1]}
            if grad:
                out["grad_verts"] = gv[t:t + 1]
            _lib.dc_loss_traj(tr.verts[t:t + 1], tr.faces, tr.draws[n0:n1].unsqueeze(0),
                              tr.targets[m0:m1].unsqueeze(0), mode=mode, grad=grad, total=False,
                              nn=False, out=out)
        losses.append(lf)
        grads.append(gv)
    return losses, grads
