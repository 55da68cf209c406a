"""Parity helpers: oracle-side input sanitising and GPU-vs-oracle comparisons.

Tolerances (written once, used by every parity test):
  - face picks and nearest-neighbour indices: bit-exact, except draws within WINDOW of a
    CDF boundary (in units of the total area), whose face may go either way;
  - loss: relative error <= LOSS_RTOL per frame and in total;
  - vertex gradient: relative L2 error <= GRAD_RTOL over the whole tensor.
"""
from __future__ import annotations

import copy

import numpy as np

import oracle

WINDOW = 1e-6
LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4


def frame_margins(verts_t, faces, draws_t, face_mask=None):
    """Oracle face picks and CDF margins of one frame's draws (no Chamfer needed)."""
    one = np.zeros((1, 3), np.float32)
    r = oracle.frame(verts_t, faces, draws_t, one, mode=oracle.UNIDIR_SUM, grads=False,
                     face_mask=face_mask)
    return r["face_idx"], r["margin"]


def nudge_draws(traj, window: float = WINDOW):
    """Copy of `traj` whose draws within `window` of a CDF boundary (per the oracle) are
    moved to the middle of their face's CDF interval, so that no face pick is ill-posed.
    Returns (trajectory, number of draws moved). Uses the oracle only."""
    tr = copy.copy(traj)
    tr.draws = traj.draws.copy()
    moved = 0
    mask = getattr(traj, "face_mask", None)
    for t in range(traj.T):
        d = tr.draws[traj.n_off[t]:traj.n_off[t + 1]]
        fi, mg = frame_margins(traj.verts[t], traj.faces, d, mask)
        bad = np.nonzero(mg < window)[0]
        if bad.size:
            cdf = oracle.area_cdf(oracle.face_areas(traj.verts[t], traj.faces, mask))
            A = cdf[-1]
            f = fi[bad]
            lo = np.where(f > 0, cdf[np.maximum(f - 1, 0)], 0.0)
            d[bad, 0] = ((lo + cdf[f]) / (2 * A)).astype(np.float32)
            moved += bad.size
    return tr, moved


def expected_moves(traj, window: float = WINDOW) -> float:
    """How many draws nudge_draws is expected to move: a uniform r_f falls within `window` of
    one of the frame's interior CDF boundaries with probability 2 window (F+ - 1), where F+
    counts the faces of positive area weight (faces outside a subset add no boundary)."""
    mask = getattr(traj, "face_mask", None)
    e = 0.0
    for t in range(traj.T):
        a = oracle.face_areas(traj.verts[t], traj.faces, mask)
        e += traj.n(t) * 2.0 * window * max(int(np.count_nonzero(a > 0)) - 1, 0)
    return e


def check_moves(traj, moved: int, window: float = WINDOW):
    """The number of draws nudge_draws moved is near its expectation: far fewer would mean a
    margin that comes out too large (draws on a boundary left in place), far more one that
    comes out too small (draws moved for nothing). Poisson-distributed, so 3x either way is
    many standard deviations once the expectation reaches a few tens."""
    e = expected_moves(traj, window)
    assert moved <= 3.0 * e + 6.0, f"{moved} draws moved, {e:.1f} expected"
    if e >= 20.0:
        assert moved >= e / 3.0, f"{moved} draws moved, {e:.1f} expected"
    return e


def nudged(traj, window: float = WINDOW):
    """nudge_draws with its count of moved draws checked against the expectation."""
    tr, moved = nudge_draws(traj, window)
    check_moves(traj, moved, window)
    return tr


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def check_face_picks(gpu_face, orc_face, margin, window: float = WINDOW):
    """Bit-exact outside the window. Returns the indices that differ (all inside it)."""
    gpu_face = np.asarray(gpu_face)
    diff = np.nonzero(gpu_face != orc_face)[0]
    outside = diff[margin[diff] >= window]
    assert outside.size == 0, (
        f"{outside.size} face picks differ outside the {window} window: "
        f"{[(int(i), int(gpu_face[i]), int(orc_face[i]), float(margin[i])) for i in outside[:5]]}")
    return diff


def check_nn(gpu_ab, orc_ab, gpu_ba=None, orc_ba=None, moved_rows=()):
    """Bit-exact neighbours. Rows whose sampled point legitimately differs (face pick inside
    the window) are exempt, and so are target-side indices that point at such a row."""
    moved = np.zeros(len(orc_ab), bool)
    moved[np.asarray(moved_rows, dtype=np.int64)] = True
    gpu_ab = np.asarray(gpu_ab)
    bad = np.nonzero((gpu_ab != orc_ab) & ~moved)[0]
    assert bad.size == 0, (f"{bad.size} sim->target neighbours differ: "
                           f"{[(int(i), int(gpu_ab[i]), int(orc_ab[i])) for i in bad[:5]]}")
    if orc_ba is not None:
        gpu_ba = np.asarray(gpu_ba)
        d = np.nonzero(gpu_ba != orc_ba)[0]
        ok = moved[np.clip(gpu_ba[d], 0, len(moved) - 1)] | moved[orc_ba[d]]
        assert np.all(ok & (gpu_ba[d] >= 0)), (
            f"{int((~ok).sum())} target->sim neighbours differ: "
            f"{[(int(j), int(gpu_ba[j]), int(orc_ba[j])) for j in d[~ok][:5]]}")


def check_loss(gpu, orc, rtol: float = LOSS_RTOL, what: str = "loss"):
    gpu = np.asarray(gpu, np.float64)
    orc = np.asarray(orc, np.float64)
    err = np.abs(gpu - orc) / np.maximum(np.abs(orc), 1e-300)
    assert np.all(err <= rtol), f"{what}: max relative error {err.max():.3e} > {rtol}"
    return float(err.max())


def check_grad(gpu, orc, rtol: float = GRAD_RTOL):
    e = rel_l2(gpu, orc)
    assert e <= rtol, f"vertex gradient: relative L2 error {e:.3e} > {rtol}"
    return e
