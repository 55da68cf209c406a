"""Pipelined loss + gradient for a stream of independent trajectories of one shape.

Each submitted step copies its inputs from (pinned) host memory to the device, runs
dc_loss_traj with the vertex gradient, and copies the gradient and the losses back to host
memory. Three CUDA streams overlap consecutive steps: while step k computes, step k+1's
inputs are copied in and step k-1's results are copied out. Events order every reuse of a
device buffer slot (inputs are overwritten only after the computation that read them, outputs
only after the copy that read them), so any number of steps can be in flight up to `depth`.

This is the shape of workloads that evaluate many independent trajectories: scoring many
candidate parameter sets, many sampling seeds, or a queue of requests of the same size.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


class LossPipeline:
    """Slots of device buffers for trajectories of T frames, V vertices, F faces, N samples
    and M targets per frame; `depth` steps may be in flight at once."""

    def __init__(self, T, V, F, N, M, device="cuda:0", mode=_lib.BIDIR_MEAN, depth=2,
                 grad=True):
        self.device = torch.device(device)
        self.mode, self.grad, self.depth = mode, grad, depth
        self.shape = (T, V, F, N, M)
        dev = self.device
        f32 = dict(dtype=torch.float32, device=dev)
        self._in = [dict(verts=torch.empty((T, V, 3), **f32),
                         faces=torch.empty((F, 3), dtype=torch.int32, device=dev),
                         draws=torch.empty((T, N, 3), **f32),
                         targets=torch.empty((T, M, 3), **f32)) for _ in range(depth)]
        self._out = [dict(loss_total=torch.empty(1, **f32), loss_frames=torch.empty(T, **f32),
                          grad_verts=torch.empty((T, V, 3), **f32) if grad else None)
                     for _ in range(depth)]
        self._s_in = torch.cuda.Stream(dev)
        self._s_run = torch.cuda.Stream(dev)
        self._s_out = torch.cuda.Stream(dev)
        self._ran = [None] * depth      # computation of the slot's last step finished
        self._copied = [None] * depth   # results of the slot's last step are on the host
        self._k = 0

    def submit(self, verts, faces, draws, targets, grad_out=None, loss_out=None,
               frames_out=None) -> torch.cuda.Event:
        """Queue one step. Inputs are host tensors (pinned for asynchronous copies) of the
        pipeline's shape; results go to the given host tensors (pinned): grad_out [T,V,3],
        loss_out [1], frames_out [T] (each optional). Returns an event that completes when
        the results are on the host; the caller must not touch the host tensors before."""
        s = self._k % self.depth
        self._k += 1
        d, o = self._in[s], self._out[s]
        with torch.cuda.stream(self._s_in):
            if self._ran[s] is not None:  # the slot's inputs were read by its last computation
                self._s_in.wait_event(self._ran[s])
            d["verts"].copy_(verts, non_blocking=True)
            d["faces"].copy_(faces, non_blocking=True)
            d["draws"].copy_(draws, non_blocking=True)
            d["targets"].copy_(targets, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(self._s_in)
        with torch.cuda.stream(self._s_run):
            self._s_run.wait_event(ready)
            if self._copied[s] is not None:  # the slot's outputs were read by the last copy
                self._s_run.wait_event(self._copied[s])
            _lib.dc_loss_traj(d["verts"], d["faces"], d["draws"], d["targets"], mode=self.mode,
                              grad=self.grad, nn=False, out=o)
            ran = torch.cuda.Event()
            ran.record(self._s_run)
            self._ran[s] = ran
        with torch.cuda.stream(self._s_out):
            self._s_out.wait_event(ran)
            if grad_out is not None and self.grad:
                grad_out.copy_(o["grad_verts"], non_blocking=True)
            if loss_out is not None:
                loss_out.copy_(o["loss_total"], non_blocking=True)
            if frames_out is not None:
                frames_out.copy_(o["loss_frames"], non_blocking=True)
            done = torch.cuda.Event()
            done.record(self._s_out)
            self._copied[s] = done
        return done

    def status(self) -> int:
        """Synchronise and return the first device-side error of the pipeline's calls."""
        with torch.cuda.stream(self._s_run):  # the workspace belongs to the compute stream
            ws = _lib.workspace(_lib.dc_workspace_size(*self.shape), self.device)
        return _lib.ws_status(ws, self._s_run)

    @staticmethod
    def pinned(shape, dtype=torch.float32) -> torch.Tensor:
        return torch.empty(shape, dtype=dtype).pin_memory()

    @staticmethod
    def pin(a) -> torch.Tensor:
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


class BatchPipeline:
    """Pipelined loss + gradient for a stream of batches of one structure: the same list of
    trajectories (frame counts, vertex and face counts, per-frame sample and target counts),
    new values every step. Each of `depth` slots holds device inputs for the whole batch and
    a batch plan over them (`batch.BatchedLoss`, replayed from a CUDA graph); three streams
    overlap consecutive batches as in `LossPipeline`, so that while batch k computes, batch
    k+1's inputs are copied in and batch k-1's gradients and losses copied out.

    `shapes` lists per trajectory (V, F, n_off, m_off): vertex and face counts and the host
    offsets of its frames' samples and targets ([T+1] each; T = len(n_off) - 1)."""

    def __init__(self, shapes, device="cuda:0", mode=_lib.BIDIR_MEAN, depth=2, grad=True,
                 weights=None, shape=None, graph=True):
        from .batch import BatchedLoss, DeviceTrajectory

        self.device = torch.device(device)
        self.depth, self.grad = depth, grad
        dev = self.device
        self._s_in = torch.cuda.Stream(dev)
        self._s_run = torch.cuda.Stream(dev)
        self._s_out = torch.cuda.Stream(dev)
        self._slots = []
        for _ in range(depth):
            trajs = []
            for V, F, n_off, m_off in shapes:
                n_off = np.asarray(n_off, np.int64)
                m_off = np.asarray(m_off, np.int64)
                T = len(n_off) - 1
                # zero-filled, so the plan's first (capturing) run reads defined values
                trajs.append(DeviceTrajectory(
                    torch.zeros((T, V, 3), dtype=torch.float32, device=dev),
                    torch.zeros((F, 3), dtype=torch.int32, device=dev),
                    torch.zeros((int(n_off[-1]), 3), dtype=torch.float32, device=dev),
                    torch.zeros((int(m_off[-1]), 3), dtype=torch.float32, device=dev),
                    n_off, m_off))
            plan = BatchedLoss(trajs, mode=mode, weights=weights, grad=grad, graph=graph,
                               stream=self._s_run, shape=shape)
            self._slots.append({"trajs": trajs, "plan": plan, "ran": None, "copied": None})
        self._k = 0

    def submit(self, inputs, grads_out=None, total_out=None, frames_out=None):
        """Queue one batch. `inputs` lists per trajectory (verts [T,V,3], faces [F,3],
        draws [sum N,3], targets [sum M,3]) host tensors (pinned for asynchronous copies);
        results go to the given pinned host tensors: grads_out (per trajectory [T,V,3]),
        total_out [1], frames_out (per trajectory [T]), each optional. Returns an event that
        completes when the results are on the host; the caller must not touch the input or
        output host tensors before (the copies read and write them asynchronously)."""
        s = self._slots[self._k % self.depth]
        self._k += 1
        with torch.cuda.stream(self._s_in):
            if s["ran"] is not None:  # the slot's inputs were read by its last computation
                self._s_in.wait_event(s["ran"])
            for d, (v, f, x, y) in zip(s["trajs"], inputs):
                d.verts.copy_(v, non_blocking=True)
                d.faces.copy_(f, non_blocking=True)
                d.draws.copy_(x, non_blocking=True)
                d.targets.copy_(y, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(self._s_in)
        plan = s["plan"]
        with torch.cuda.stream(self._s_run):
            self._s_run.wait_event(ready)
            if s["copied"] is not None:  # the slot's outputs were read by the last copy
                self._s_run.wait_event(s["copied"])
            plan.run()
            ran = torch.cuda.Event()
            ran.record(self._s_run)
            s["ran"] = ran
        with torch.cuda.stream(self._s_out):
            self._s_out.wait_event(ran)
            if grads_out is not None and self.grad:
                for h, g in zip(grads_out, plan.grad_verts):
                    h.copy_(g, non_blocking=True)
            if frames_out is not None:
                for h, lf in zip(frames_out, plan.loss_frames):
                    h.copy_(lf, non_blocking=True)
            if total_out is not None:
                total_out.copy_(plan.total, non_blocking=True)
            done = torch.cuda.Event()
            done.record(self._s_out)
            s["copied"] = done
        return done

    def status(self) -> int:
        """Synchronise and return the first device-side error of the slots' last runs."""
        torch.cuda.synchronize(self.device)
        for s in self._slots:
            rc = _lib.ws_status(s["plan"].ws, self._s_run)
            if rc != _lib.DC_OK:
                return rc
        return _lib.DC_OK
