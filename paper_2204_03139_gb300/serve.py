"""Serving loss-and-gradient requests from many concurrent parameter-inference optimisations.

Each request is one trajectory (its own mesh resolution, frame count and cloud sizes) whose
loss and vertex gradient a caller's optimiser needs (the inner step of Sec. III-C, repeated by
every optimisation). The server batches continuously:

  - admission: requests wait in arrival order until their device memory (inputs, outputs and
    their share of a batch workspace) fits in the HBM budget; their inputs are then copied to
    the device once, on a copy stream, and stay resident until the result is delivered;
  - time slicing: an admitted request is cut into items of consecutive frames of at most
    `item_pairs` point pairs, so that a long request cannot hold the GPU for its whole
    duration (one persistent Chamfer launch occupies every SM until it ends);
  - batching: whenever one of the compute streams is free, admitted items of the same mode, up
    to `max_batch_pairs`, go into one planned launch sequence (dc_batch_plan / dc_batch_run):
    one persistent Chamfer launch covers all their frames, whatever their sizes. Requests are
    served shortest remaining work first (a short request passes a long one; long ones run
    one after another instead of sharing the GPU and all finishing late), except that a
    request waiting longer than `max_wait_s` goes first, so that long ones never starve;
  - overlap: batches on different streams run at the same time while new requests are
    admitted and copied in. A batch's plan is uploaded from pinned staging memory without
    waiting for its stream, and every item writes its frames' losses and gradients straight
    into its request's device buffers; when a request's last item finishes, the library forms
    its total (dc_loss_total, the same fixed order as one dc_loss_traj call) and the results
    go back to pinned host memory by copies that an event completes, so the scheduler thread
    never waits for the device. Finished requests resolve their futures and release their
    memory, which admits the next requests.

Every result equals the one the request gets alone (same kernels; only the order of the
per-slice loss partial sums may differ, within float32 rounding).
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from .batch import BatchedLoss, DeviceTrajectory


@dataclass
class Result:
    loss_frames: np.ndarray          # [T] L_t
    loss_total: float                # sum_t w_t L_t
    grad_verts: np.ndarray | None    # [T, V, 3] gradient of sum_t w_t L_t
    latency_s: float                 # completion - arrival
    batch_id: int
    batch_requests: int


@dataclass(eq=False)  # identity comparison: the fields hold arrays and tensors
class _Request:
    rid: int
    traj: object
    mode: int
    weights: np.ndarray | None
    grad: bool
    arrival: float
    nbytes: int
    future: Future
    dev: DeviceTrajectory | None = None
    ready: torch.cuda.Event | None = None
    host: tuple = field(default_factory=tuple)
    loss_dev: torch.Tensor | None = None   # [T] on the device, written item by item
    grad_dev: torch.Tensor | None = None   # [T, V, 3]
    w_dev: torch.Tensor | None = None      # [T] frame weights (None: all ones)
    w_host: torch.Tensor | None = None     # their pinned host copy, alive until the copy ran
    total_dev: torch.Tensor | None = None  # [1] sum_t w_t L_t, formed by the library
    out_host: tuple = field(default_factory=tuple)  # pinned (loss, grad, total) copies
    fin: torch.cuda.Event | None = None    # the host copies of the results are complete
    left: int = 0                          # items not finished yet
    batches: set = field(default_factory=set)
    last_batch: int = 0
    last_batch_items: int = 0              # items in the batch that finished the request
    failed: bool = False


@dataclass(eq=False)
class _Item:
    req: _Request
    a: int             # first frame
    b: int             # one past the last frame
    dev: DeviceTrajectory
    pairs: int


def form_batch(items, now: float, cap: float, max_items: int, max_wait_s: float):
    """The items of the next batch, from admitted items (objects with .req (having .arrival)
    and .pairs). Requests are taken shortest remaining work first, those that waited longer
    than max_wait_s first of all (oldest first), so that long requests cannot starve; each
    request's items in order, until the batch holds `cap` pairs or `max_items` items (the
    first item is always taken). Returns (items, pairs)."""
    reqs, items_of = {}, collections.defaultdict(list)
    for it in items:
        reqs[id(it.req)] = it.req
        items_of[id(it.req)].append(it)
    remaining = {k: sum(it.pairs for it in v) for k, v in items_of.items()}

    def priority(k):
        r = reqs[k]
        if now - r.arrival > max_wait_s:
            return (0, r.arrival, 0)
        return (1, remaining[k], r.arrival)

    take, pairs = [], 0
    for k in sorted(reqs, key=priority):
        for it in items_of[k]:
            if take and (len(take) >= max_items or pairs + it.pairs > cap):
                return take, pairs
            take.append(it)
            pairs += it.pairs
    return take, pairs


def _slice(d: DeviceTrajectory, a: int, b: int) -> DeviceTrajectory:
    """Frames [a, b) of a device trajectory (views, no copies)."""
    n0, n1 = int(d.n_off[a]), int(d.n_off[b])
    m0, m1 = int(d.m_off[a]), int(d.m_off[b])
    return DeviceTrajectory(d.verts[a:b], d.faces, d.draws[n0:n1], d.targets[m0:m1],
                            d.n_off[a:b + 1] - n0, d.m_off[a:b + 1] - m0, d.face_mask)


def _frames_of(traj):
    """dc_frame array with sizes only (no pointers): enough for dc_batch_workspace_size."""
    n = np.diff(np.asarray(traj.n_off))
    m = np.diff(np.asarray(traj.m_off))
    fr = (_lib.dc_frame * traj.T)()
    for t in range(traj.T):
        fr[t].V, fr[t].F, fr[t].N, fr[t].M = traj.V, traj.F, int(n[t]), int(m[t])
        fr[t].grad_verts = 1  # counted as having a gradient
    return fr


def request_bytes(traj, grad: bool = True) -> int:
    """Device bytes a request holds while admitted: inputs, outputs, workspace share."""
    inputs = (traj.verts.nbytes + traj.faces.nbytes + traj.draws.nbytes + traj.targets.nbytes
              + traj.F)  # and the face mask, if any
    outputs = 4 * traj.T + (traj.verts.nbytes if grad else 0)
    ws = int(_lib.lib().dc_batch_workspace_size(_frames_of(traj), traj.T))
    if ws == 0:
        raise _lib.DCError(_lib.DC_EINVAL, "request sizes are invalid")
    return inputs + outputs + ws + 64 * 1024


class Server:
    """Continuous-batching loss+gradient server on one GPU."""

    def __init__(self, device="cuda:0", hbm_budget: int = 120 << 30, streams: int = 2,
                 max_batch_items: int = 512, max_batch_pairs: int = 16 * 10**9,
                 item_pairs: int = 16 * 10**9, max_wait_s: float = 0.2):
        """max_batch_pairs: batch size when the queue is short; under load batches grow up
        to 8x that. item_pairs: the time slice a long request is cut into."""
        self.device = torch.device(device)
        self.budget = int(hbm_budget)
        self.max_batch_items = max_batch_items
        self.max_batch_pairs = max_batch_pairs
        self.item_pairs = item_pairs
        self.max_wait_s = max_wait_s
        self._copy = torch.cuda.Stream(self.device)
        self._streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self._busy = [None] * streams
        self._cv = threading.Condition()
        self._waiting: collections.deque = collections.deque()
        self._admitted: list = []
        self._used = 0
        self._next_id = 0
        self._next_batch = 0
        self._closing = False
        self.completed: list[tuple[int, float, int, int]] = []  # (rid, latency, pairs, batch)
        self.batch_sizes: list[int] = []
        self.host_launch_s: list[float] = []  # scheduler host time to plan and launch a batch
        self._finishing: list = []
        self._thread = threading.Thread(target=self._loop, name="diffcloud-serve", daemon=True)
        self._thread.start()

    # ---- client side ----
    def submit(self, traj, mode: int = _lib.BIDIR_MEAN, weights=None, grad: bool = True) -> Future:
        """Queue one trajectory (workloads.Trajectory or anything with verts, faces, draws,
        targets, n_off, m_off as numpy arrays). Returns a Future of Result."""
        fut: Future = Future()
        try:
            nbytes = request_bytes(traj, grad)
        except Exception as e:  # invalid sizes
            fut.set_exception(e)
            return fut
        if nbytes > self.budget:
            fut.set_exception(_lib.DCError(
                _lib.DC_ENOSPC, f"request needs {nbytes} bytes, the HBM budget is {self.budget}"))
            return fut
        w = None if weights is None else np.asarray(weights, np.float32)
        with self._cv:
            if self._closing:
                fut.set_exception(RuntimeError("server is closed"))
                return fut
            r = _Request(self._next_id, traj, mode, w, grad, time.perf_counter(), nbytes, fut)
            self._next_id += 1
            self._waiting.append(r)
            self._cv.notify()
        return fut

    def close(self, wait: bool = True):
        with self._cv:
            self._closing = True
            self._cv.notify()
        if wait:
            self._thread.join()

    def stats(self) -> dict:
        lat = np.array([c[1] for c in self.completed]) if self.completed else np.zeros(0)
        hl = np.array(self.host_launch_s) if self.host_launch_s else np.zeros(0)
        return {"requests": len(self.completed),
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
                "mean_batch_requests": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0,
                "batches": len(self.batch_sizes),
                "host_ms_per_batch": float(hl.mean() * 1e3) if hl.size else None,
                "host_ms_per_batch_p99": float(np.percentile(hl, 99) * 1e3) if hl.size else None}

    # ---- scheduler thread ----
    def _loop(self):
        torch.cuda.set_device(self.device)
        # the scheduler's own allocations and copies go on the copy stream, never on the
        # legacy default stream
        torch.cuda.set_stream(self._copy)
        while True:
            with self._cv:
                idle = (not self._waiting and not self._admitted and not self._finishing
                        and all(b is None for b in self._busy))
                if idle and self._closing:
                    return
                if idle:
                    self._cv.wait(timeout=0.05)
                    continue
            try:
                self._admit()
                self._launch()
                progressed = self._complete()
                progressed = self._finish() or progressed
            except Exception as e:  # fail the affected requests, keep serving
                self._fail_all(e)
                progressed = True
            if not progressed:
                time.sleep(5e-5)

    def _admit(self):
        while True:
            with self._cv:
                if not self._waiting or self._used + self._waiting[0].nbytes > self.budget:
                    return
                r = self._waiting.popleft()
                self._used += r.nbytes
            tr = r.traj
            # pinned host copies, kept on the trajectory object for repeated submissions
            host = getattr(tr, "_dc_pinned", None)
            if host is None:
                arrays = [tr.verts, tr.faces, tr.draws, tr.targets]
                if getattr(tr, "face_mask", None) is not None:
                    arrays.append(np.asarray(tr.face_mask, np.uint8))
                host = tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                             for a in arrays)
                try:
                    tr._dc_pinned = host
                except AttributeError:
                    pass
            with torch.cuda.stream(self._copy):
                dv = [h.to(self.device, non_blocking=True) for h in host]
                r.ready = torch.cuda.Event()
                r.ready.record(self._copy)
            r.host = host  # pinned buffers live until the copy has finished
            r.dev = DeviceTrajectory(dv[0], dv[1], dv[2], dv[3], np.asarray(tr.n_off, np.int64),
                                     np.asarray(tr.m_off, np.int64),
                                     dv[4] if len(dv) > 4 else None)
            with torch.cuda.stream(self._copy):
                r.loss_dev = torch.empty(tr.T, dtype=torch.float32, device=self.device)
                r.grad_dev = (torch.empty(tr.verts.shape, dtype=torch.float32, device=self.device)
                              if r.grad else None)
                r.total_dev = torch.empty(1, dtype=torch.float32, device=self.device)
                if r.weights is not None:
                    # pinned, so the copy does not wait for the stream; the request keeps the
                    # host buffer until its results are back
                    r.w_host = torch.from_numpy(
                        np.ascontiguousarray(r.weights, np.float32)).pin_memory()
                    r.w_dev = r.w_host.to(self.device, non_blocking=True)
            # cut into items of consecutive frames of at most item_pairs pairs
            per = np.diff(r.dev.n_off) * np.diff(r.dev.m_off)
            a = 0
            items = []
            while a < tr.T:
                b, acc = a, 0
                while b < tr.T and (b == a or acc + per[b] <= self.item_pairs):
                    acc += int(per[b])
                    b += 1
                items.append(_Item(r, a, b, _slice(r.dev, a, b), acc))
                a = b
            r.left = len(items)
            self._admitted.extend(items)

    def _launch(self):
        for s_idx, busy in enumerate(self._busy):
            if busy is not None or not self._admitted:
                continue
            mode = self._admitted[0].req.mode
            # small batches while few requests wait (latency), larger ones when many do
            # (fewer launches per pair)
            waiting = len({id(it.req) for it in self._admitted})
            cap = self.max_batch_pairs * max(1, min(8, waiting // 8))
            take, pairs = form_batch([it for it in self._admitted if it.req.mode == mode],
                                     time.perf_counter(), cap, self.max_batch_items,
                                     self.max_wait_s)
            for it in take:
                self._admitted.remove(it)
            stream = self._streams[s_idx]
            for r in {id(it.req): it.req for it in take}.values():
                stream.wait_event(r.ready)
            t_host = time.perf_counter()
            weights, outs = [], []
            for it in take:
                w = it.req.weights
                weights.append(w[it.a:it.b] if w is not None else np.ones(it.b - it.a, np.float32))
                outs.append((it.req.loss_dev[it.a:it.b],
                             it.req.grad_dev[it.a:it.b] if it.req.grad_dev is not None else None))
            any_grad = any(it.req.grad for it in take)
            if any_grad:  # a batch either computes every frame's gradient or none
                outs = [(lf, gv) if gv is not None else (lf, torch.empty(
                    (lf.shape[0],) + tuple(it.dev.verts.shape[1:]), dtype=torch.float32,
                    device=self.device)) for (lf, gv), it in zip(outs, take)]
            b = BatchedLoss([it.dev for it in take], mode=mode, weights=weights, grad=any_grad,
                            stream=stream, outputs=outs, async_plan=True)
            b.run()
            self.host_launch_s.append(time.perf_counter() - t_host)
            done = torch.cuda.Event()
            done.record(stream)
            self._busy[s_idx] = (b, done, take, self._next_batch, pairs)
            self.batch_sizes.append(len(take))
            self._next_batch += 1

    def _complete(self) -> bool:
        progressed = False
        for s_idx, busy in enumerate(self._busy):
            if busy is None:
                continue
            b, done, take, bid, _ = busy
            if not done.query():
                continue
            # the batch's stream is idle: reading its status waits for nothing
            status = _lib.ws_status(b.ws, b.stream)
            for it in take:
                r = it.req
                if status != _lib.DC_OK:
                    r.failed = True
                r.batches.add(bid)
                r.last_batch = bid
                r.last_batch_items = len(take)
                r.left -= 1
                if r.left == 0:
                    self._finalize(r, b.stream, status)
            self._busy[s_idx] = None
            progressed = True
        return progressed

    def _finalize(self, r, stream, status):
        """The request's last item is done (every earlier one too): on the batch's stream, the
        library forms the total and the results are copied to pinned host memory; an event
        marks their arrival, which _finish waits for without blocking."""
        if r.failed:
            r.future.set_exception(_lib.DCError(status, "device-side error in batch"))
            self._release(r)
            return
        with torch.cuda.stream(stream):
            _lib.dc_loss_total(r.loss_dev, r.w_dev, out=r.total_dev)
            h_loss = torch.empty(r.loss_dev.shape, dtype=torch.float32, pin_memory=True)
            h_total = torch.empty(1, dtype=torch.float32, pin_memory=True)
            h_loss.copy_(r.loss_dev, non_blocking=True)
            h_total.copy_(r.total_dev, non_blocking=True)
            h_grad = None
            if r.grad_dev is not None:
                h_grad = torch.empty(r.grad_dev.shape, dtype=torch.float32, pin_memory=True)
                h_grad.copy_(r.grad_dev, non_blocking=True)
            r.fin = torch.cuda.Event()
            r.fin.record(stream)
        r.out_host = (h_loss, h_grad, h_total)
        self._finishing.append(r)

    def _finish(self) -> bool:
        progressed = False
        for r in list(self._finishing):
            if not r.fin.query():
                continue
            self._finishing.remove(r)
            h_loss, h_grad, h_total = r.out_host
            lat = time.perf_counter() - r.arrival
            r.future.set_result(Result(h_loss.numpy(), float(h_total[0]),
                                       h_grad.numpy() if h_grad is not None else None, lat,
                                       r.last_batch, r.last_batch_items))
            self.completed.append((r.rid, lat, r.dev.pairs(), r.last_batch))
            self._release(r)
            progressed = True
        return progressed

    def _release(self, r):
        r.dev = None
        r.host = ()
        r.loss_dev = r.grad_dev = r.total_dev = r.w_dev = r.w_host = None
        with self._cv:
            self._used -= r.nbytes

    def _fail_all(self, e):
        reqs = {}
        for s_idx, busy in enumerate(self._busy):
            if busy is not None:
                for it in busy[2]:
                    reqs[id(it.req)] = it.req
                self._busy[s_idx] = None
        for it in self._admitted:
            reqs[id(it.req)] = it.req
        self._admitted.clear()
        for r in self._finishing:
            reqs[id(r)] = r
        self._finishing.clear()
        for r in reqs.values():
            if not r.future.done():
                r.future.set_exception(e)
            with self._cv:
                self._used -= r.nbytes


def serve_plain(requests, device="cuda:0", mode: int = _lib.BIDIR_MEAN):
    """The plain per-request form, for comparison: each request in arrival order, copied in,
    computed with dc_loss_traj (uniform trajectories) on one stream, copied out. Requests are
    (arrival_s, traj) pairs; returns the per-request latencies (s) measured from arrival."""
    dev = torch.device(device)
    t0 = time.perf_counter()
    lat = []
    for arrival, tr in requests:
        now = time.perf_counter() - t0
        if now < arrival:
            time.sleep(arrival - now)
        v = torch.from_numpy(tr.verts).to(dev)
        f = torch.from_numpy(tr.faces).to(dev)
        d = torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).to(dev)
        y = torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).to(dev)
        m = getattr(tr, "face_mask", None)
        m = None if m is None else torch.from_numpy(np.asarray(m, np.uint8)).to(dev)
        r = _lib.dc_loss_traj(v, f, d, y, mode=mode, face_mask=m)
        r["grad_verts"].cpu()
        float(r["loss_total"][0])
        lat.append(time.perf_counter() - t0 - arrival)
    return lat
