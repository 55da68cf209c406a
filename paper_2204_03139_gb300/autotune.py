"""Autotuner of the nearest-neighbour search's engine and tile shape.

The shapes it chooses between:
  ("tensor", 0)  the tensor-core filter on warp-level MMAs (frames of at most 524 288
                 points per side; the library's default for calls of 1e9 pairs and more);
  ("tcgen05", 0) the same filter on tcgen05 MMAs;
  ("direct", w)  the CUDA-core direct form with CTAs of w = 1, 2 or 4 warps (w x 512 sim
                 points held in registers; wide CTAs amortise the target staging and the
                 column merges, narrow ones split small problems into enough work items).
tune() times every shape on the caller's own inputs and records the fastest per size bucket
in a JSON cache (path from DC_AUTOTUNE_CACHE, default ~/.cache/diffcloud/autotune.json);
best() looks a bucket up; tuned() sets a shape around a block of calls (and of batch plans,
which keep the shape they were planned with); tune_batch() does the same for a list of
trajectories planned as one batch.
"""
from __future__ import annotations

import contextlib
import json
import math
import os
import threading

import torch

from . import _lib

SHAPES = (("tensor", 0), ("tcgen05", 0), ("direct", 1), ("direct", 2), ("direct", 4))
_ENGINES = {"tcgen05": _lib.ENGINE_TCGEN05, "tensor": _lib.ENGINE_TENSOR,
            "direct": _lib.ENGINE_DIRECT}
WIDTHS = (1, 2, 4)
_lock = threading.Lock()
_cache: dict | None = None


def cache_path() -> str:
    return os.environ.get("DC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "diffcloud",
                                       "autotune.json"))


def _load() -> dict:
    global _cache
    if _cache is None:
        try:
            with open(cache_path()) as f:
                _cache = json.load(f)
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _save():
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(_cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _lg(x) -> int:
    return int(math.floor(math.log2(max(1, x))))


def bucket(T: int, N: int, M: int, mode: int, device=None) -> str:
    """Size bucket: device, mode, and powers of two of frames, sim points and targets."""
    name = torch.cuda.get_device_name(device)
    return f"{name}|m{mode}|T{_lg(T)}|N{_lg(N)}|M{_lg(M)}"


def batch_bucket(trajs, mode: int, device=None) -> str:
    """Size bucket of a batch: frames, mean points per side and total pairs (powers of two)."""
    frames = sum(t.T for t in trajs)
    n = sum(int(t.n_off[-1]) for t in trajs) / max(frames, 1)
    m = sum(int(t.m_off[-1]) for t in trajs) / max(frames, 1)
    pairs = sum(t.pairs() for t in trajs)
    name = torch.cuda.get_device_name(device)
    return f"{name}|batch|m{mode}|F{_lg(frames)}|N{_lg(n)}|M{_lg(m)}|P{_lg(pairs)}"


def _norm(shape):
    """A shape as (engine name, warps); an int w means ("direct", w)."""
    if shape is None:
        return None
    if isinstance(shape, int):
        return ("direct", shape)
    e, w = shape
    return (str(e), int(w))


def best(T: int, N: int, M: int, mode: int = _lib.BIDIR_MEAN, device=None):
    with _lock:
        s = _load().get(bucket(T, N, M, mode, device))
    return None if s is None else _norm(s)


@contextlib.contextmanager
def tuned(shape):
    """Use `shape` (("tcgen05", 0), ("tensor", 0), ("direct", w), or an int w for the direct
    engine; None leaves the current setting) for the calls and plans in the block."""
    shape = _norm(shape)
    if shape is None:
        yield
        return
    old = _lib.tune_get()
    _lib.tune_set(shape[1] if shape[0] == "direct" else 0, _ENGINES[shape[0]])
    try:
        yield
    finally:
        _lib.tune_set(*old)


def _time(fn, dev, reps: int) -> float:
    fn()  # warm-up
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps


def tune(verts, faces, draws, targets, mode: int = _lib.BIDIR_MEAN, reps: int = 3,
         save: bool = True, shapes=SHAPES) -> dict:
    """Time dc_loss_traj (forward + gradient) at every shape on these inputs; record and
    return {"best": shape, "ms": {shape: ms}}."""
    dev = verts.device
    T, N, M = verts.shape[0], draws.shape[1], targets.shape[1]
    times = {}
    for sh in shapes:
        with tuned(sh):
            times[sh] = _time(lambda: _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode),
                              dev, reps)
    s_best = min(times, key=times.get)
    with _lock:
        _load()[bucket(T, N, M, mode, dev)] = list(s_best)
        if save:
            _save()
    return {"best": s_best, "ms": times}


def tune_batch(trajs, mode: int = _lib.BIDIR_MEAN, weights=None, grad: bool = True,
               reps: int = 2, save: bool = True, shapes=SHAPES) -> dict:
    """Plan the batch of DeviceTrajectory objects at every shape, time its run, record the
    fastest for the batch's size bucket and return {"best": shape, "ms": {shape: ms}}."""
    from .batch import BatchedLoss

    dev = trajs[0].verts.device
    times = {}
    for sh in shapes:
        with tuned(sh):
            b = BatchedLoss(trajs, mode=mode, weights=weights, grad=grad)
        times[sh] = _time(b.run, dev, reps)
        del b
    s_best = min(times, key=times.get)
    with _lock:
        _load()[batch_bucket(trajs, mode, dev)] = list(s_best)
        if save:
            _save()
    return {"best": s_best, "ms": times}


def best_batch(trajs, mode: int = _lib.BIDIR_MEAN, device=None):
    with _lock:
        s = _load().get(batch_bucket(trajs, mode, device))
    return None if s is None else _norm(s)


def loss_traj(verts, faces, draws, targets, mode: int = _lib.BIDIR_MEAN, **kw):
    """dc_loss_traj at the tuned shape of its size bucket (tuning the bucket first if it has
    no entry yet)."""
    T, N, M = verts.shape[0], draws.shape[1], targets.shape[1]
    s = best(T, N, M, mode, verts.device)
    if s is None:
        s = tune(verts, faces, draws, targets, mode)["best"]
    with tuned(s):
        return _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode, **kw)
