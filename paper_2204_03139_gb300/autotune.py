"""Autotuner of the Chamfer kernel's tile shape.

The tile shape is the number of warps per Chamfer CTA (1, 2 or 4; each warp holds 512 sim
points). The best width depends on the problem size: wide CTAs amortise the target staging
and the column merges, narrow ones split small problems into enough work items. tune() times
every width on the caller's own inputs and records the fastest per size bucket in a JSON cache
(path from DC_AUTOTUNE_CACHE, default ~/.cache/diffcloud/autotune.json); best() looks a
bucket up; tuned() sets the width around a block of calls.
"""
from __future__ import annotations

import contextlib
import json
import math
import os
import threading

import torch

from . import _lib

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


def bucket(T: int, N: int, M: int, mode: int, device=None) -> str:
    """Size bucket: device, mode, and powers of two of frames, sim points and targets."""
    name = torch.cuda.get_device_name(device)
    lg = lambda x: int(math.floor(math.log2(max(1, x))))  # noqa: E731
    return f"{name}|m{mode}|T{lg(T)}|N{lg(N)}|M{lg(M)}"


def best(T: int, N: int, M: int, mode: int = _lib.BIDIR_MEAN, device=None) -> int | None:
    with _lock:
        return _load().get(bucket(T, N, M, mode, device))


@contextlib.contextmanager
def tuned(warps: int | None):
    """Use CTA width `warps` (None: leave the current setting) for the calls in the block."""
    if warps is None:
        yield
        return
    old = _lib.tune_get()
    _lib.tune_set(warps)
    try:
        yield
    finally:
        _lib.tune_set(old)


def tune(verts, faces, draws, targets, mode: int = _lib.BIDIR_MEAN, reps: int = 3,
         save: bool = True) -> dict:
    """Time dc_loss_traj (forward + gradient) at every width on these inputs; record and
    return {"best": w, "ms": {w: ms}}."""
    dev = verts.device
    T, N, M = verts.shape[0], draws.shape[1], targets.shape[1]
    times = {}
    for w in WIDTHS:
        with tuned(w):
            _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode)  # warm-up
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode)
            b.record()
            torch.cuda.synchronize(dev)
            times[w] = a.elapsed_time(b) / reps
    w_best = min(times, key=times.get)
    with _lock:
        _load()[bucket(T, N, M, mode, dev)] = w_best
        if save:
            _save()
    return {"best": w_best, "ms": times}


def loss_traj(verts, faces, draws, targets, mode: int = _lib.BIDIR_MEAN, **kw):
    """dc_loss_traj at the tuned width of its size bucket (tuning the bucket first if it has
    no entry yet)."""
    T, N, M = verts.shape[0], draws.shape[1], targets.shape[1]
    w = best(T, N, M, mode, verts.device)
    if w is None:
        w = tune(verts, faces, draws, targets, mode)["best"]
    with tuned(w):
        return _lib.dc_loss_traj(verts, faces, draws, targets, mode=mode, **kw)
