"""FP64 CPU oracle of the DiffCloud loss (ctypes binding of diffcloud_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the bench's CPU
baseline leg, never by the library. It shares no code with the CUDA path; both read the same
seeded inputs from `workloads`.

Functions follow the paper: face areas and area-weighted pick (Sec. III-B), barycentric
point (Eq. 3), Chamfer loss (Eq. 1, Eq. 2), gradient scatter (Eq. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diffcloud_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

BIDIR_MEAN = 0  # Eq. 1
UNIDIR_SUM = 1  # Eq. 2

OK, EINVAL, EDEGENERATE = 0, -1, -2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        _lib.orc_frame.restype = I
        _lib.orc_frame.argtypes = [P, P, P, I, I, P, I, P, I, I, D, I] + [P] * 16
        _lib.orc_chamfer.restype = I
        _lib.orc_chamfer.argtypes = [P, I, P, I, I, D, P, P]
        _lib.orc_nn_pair.restype = None
        _lib.orc_nn_pair.argtypes = [P, I, P, I, P, P, P, P, P, P]
        _lib.orc_face_areas.restype = None
        _lib.orc_face_areas.argtypes = [P, P, I, P]
        _lib.orc_mask_areas.restype = None
        _lib.orc_mask_areas.argtypes = [P, P, I]
        _lib.orc_area_cdf.restype = None
        _lib.orc_area_cdf.argtypes = [P, I, P]
        _lib.orc_pick_face.restype = I
        _lib.orc_pick_face.argtypes = [P, I, ctypes.c_float, P]
        _lib.orc_bary.restype = None
        _lib.orc_bary.argtypes = [ctypes.c_float, ctypes.c_float, P]
        _lib.orc_num_threads.restype = I
        _lib.orc_set_num_threads.restype = None
        _lib.orc_set_num_threads.argtypes = [I]
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle returned {code}")
        self.code = code


def face_areas(verts, faces, face_mask=None) -> np.ndarray:
    """Face areas; with a mask, the area weights of faces outside the subset are 0."""
    v, f = _c(verts, np.float32), _c(faces, np.int32)
    out = np.empty(f.shape[0], np.float64)
    lib().orc_face_areas(_p(v), _p(f), f.shape[0], _p(out))
    if face_mask is not None:
        m = _c(face_mask, np.uint8)
        lib().orc_mask_areas(_p(out), _p(m), f.shape[0])
    return out


def area_cdf(area) -> np.ndarray:
    a = _c(area, np.float64)
    out = np.empty_like(a)
    lib().orc_area_cdf(_p(a), a.size, _p(out))
    return out


def pick_face(cdf, r: float) -> tuple[int, float]:
    c = _c(cdf, np.float64)
    m = np.zeros(1, np.float64)
    f = lib().orc_pick_face(_p(c), c.size, ctypes.c_float(r), _p(m))
    return int(f), float(m[0])


def bary(r1: float, r2: float) -> np.ndarray:
    w = np.empty(3, np.float64)
    lib().orc_bary(ctypes.c_float(r1), ctypes.c_float(r2), _p(w))
    return w


def frame(verts, faces, draws, tgt, mode: int = BIDIR_MEAN, gscale: float = 1.0,
          exact64: bool = False, details: bool = True, grads: bool = True,
          face_mask=None) -> dict:
    """One frame: loss, gradients and every intermediate (see orc_frame). face_mask [F]:
    sample only the faces with a nonzero entry."""
    v, f = _c(verts, np.float32), _c(faces, np.int32)
    fm = None if face_mask is None else _c(face_mask, np.uint8)
    if fm is not None and fm.shape != (f.shape[0],):
        raise ValueError("face_mask must have one entry per face")
    d, y = _c(draws, np.float32), _c(tgt, np.float32)
    V, F, N, M = v.shape[0], f.shape[0], d.shape[0], y.shape[0]
    out = {"loss": np.zeros(1), "loss_exact": np.full(1, np.nan)}
    if grads:
        out["grad_verts"] = np.empty((V, 3))
        out["grad_points"] = np.empty((N, 3))
        out["grad_targets"] = np.empty((M, 3))
    if details:
        out.update(face_idx=np.empty(N, np.int32), margin=np.empty(N), bary=np.empty((N, 3)),
                   x64=np.empty((N, 3)), x32=np.empty((N, 3), np.float32))
    out.update(nn_ab=np.empty(N, np.int32), d_ab=np.empty(N, np.float32),
               d2_ab=np.empty(N, np.float32), nn_ba=np.empty(M, np.int32),
               d_ba=np.empty(M, np.float32), d2_ba=np.empty(M, np.float32))
    g = out.get
    rc = lib().orc_frame(_p(v), _p(f), _p(fm), V, F, _p(d), N, _p(y), M, int(mode),
                         float(gscale),
                         int(exact64), _p(out["loss"]), _p(out["loss_exact"]),
                         _p(g("grad_verts")), _p(g("face_idx")), _p(g("margin")),
                         _p(g("bary")), _p(g("x64")), _p(g("x32")), _p(out["nn_ab"]),
                         _p(out["d_ab"]), _p(out["d2_ab"]), _p(out["nn_ba"]), _p(out["d_ba"]),
                         _p(out["d2_ba"]), _p(g("grad_points")), _p(g("grad_targets")))
    if rc != OK:
        raise OracleError(rc)
    out["loss"] = float(out["loss"][0])
    out["loss_exact"] = float(out["loss_exact"][0])
    return out


def chamfer(a, b, mode: int = BIDIR_MEAN, gscale: float = 1.0) -> tuple[float, np.ndarray]:
    """Chamfer loss of two clouds (Eq. 1 / Eq. 2) and its gradient w.r.t. the first."""
    a, b = _c(a, np.float32), _c(b, np.float32)
    loss = np.zeros(1)
    ga = np.empty(a.shape)
    rc = lib().orc_chamfer(_p(a), a.shape[0], _p(b), b.shape[0], int(mode), float(gscale),
                           _p(loss), _p(ga))
    if rc != OK:
        raise OracleError(rc)
    return float(loss[0]), ga


def nn_pair(a, b) -> dict:
    a, b = _c(a, np.float32), _c(b, np.float32)
    n, m = a.shape[0], b.shape[0]
    o = {k: np.empty(n, t) for k, t in (("nn_ab", np.int32), ("d_ab", np.float32),
                                          ("d2_ab", np.float32))}
    o.update({k: np.empty(m, t) for k, t in (("nn_ba", np.int32), ("d_ba", np.float32),
                                               ("d2_ba", np.float32))})
    lib().orc_nn_pair(_p(a), n, _p(b), m, _p(o["nn_ab"]), _p(o["d_ab"]), _p(o["d2_ab"]),
                      _p(o["nn_ba"]), _p(o["d_ba"]), _p(o["d2_ba"]))
    return o


def loss_traj(traj, mode: int = BIDIR_MEAN, weights=None, gscale=None, frames=None,
              details: bool = False, grads: bool = True) -> dict:
    """Per-frame oracle over a (possibly ragged) workloads.Trajectory.

    L = sum_t w_t L_t (weights default to 1); grad_verts[t] = gscale[t] dL_t/dverts[t] with
    gscale defaulting to the weights. `frames` restricts the run to a subset of frames
    (the others are reported as NaN)."""
    T = traj.T
    w = np.ones(T) if weights is None else np.asarray(weights, np.float64)
    gs = w if gscale is None else np.asarray(gscale, np.float64)
    frames = range(T) if frames is None else frames
    loss_frames = np.full(T, np.nan)
    grad = np.full((T, traj.V, 3), np.nan) if grads else None
    per = {}
    for t in frames:
        r = frame(traj.verts[t], traj.faces, traj.frame_draws(t), traj.frame_targets(t),
                  mode=mode, gscale=float(gs[t]), details=details, grads=grads,
                  face_mask=getattr(traj, "face_mask", None))
        loss_frames[t] = r["loss"]
        if grads:
            grad[t] = r["grad_verts"]
        per[t] = r
    total = float(np.nansum(w * loss_frames))
    return {"loss_frames": loss_frames, "loss_total": total, "grad_verts": grad, "frames": per}


def time_pairs(traj, seconds: float = 10.0, mode: int = BIDIR_MEAN) -> dict:
    """Time the oracle on whole frames of `traj` until `seconds` have passed (at least one
    frame). Returns the unique pairs processed, the elapsed time and the thread count."""
    t0 = time.perf_counter()
    pairs, frames = 0, 0
    for t in range(traj.T):
        frame(traj.verts[t], traj.faces, traj.frame_draws(t), traj.frame_targets(t), mode=mode,
              details=False)
        pairs += traj.n(t) * traj.m(t)
        frames += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"pairs": pairs, "frames": frames, "seconds": el, "pairs_per_s": pairs / el,
            "threads": num_threads()}
