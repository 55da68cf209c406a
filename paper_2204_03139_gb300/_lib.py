"""ctypes binding of libdiffcloud.so: the C-ABI entry points under the same names.

Argument marshalling only: tensors in, device pointers and the current CUDA stream out to
the library, outputs and workspaces allocated with torch. Every step of the loss runs in the
library's CUDA kernels; there is no other code path. If the library has not been built this
module raises at first use.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

DC_OK, DC_EINVAL, DC_EDEGENERATE, DC_ECUDA, DC_ETIMEOUT, DC_EDEVICE, DC_ENOSPC = (
    0, -1, -2, -3, -4, -5, -6)
BIDIR_MEAN, UNIDIR_SUM = 0, 1
_NAMES = {0: "DC_OK", -1: "DC_EINVAL", -2: "DC_EDEGENERATE", -3: "DC_ECUDA",
          -4: "DC_ETIMEOUT", -5: "DC_EDEVICE", -6: "DC_ENOSPC"}

_lib = None
_lock = threading.Lock()


class DCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


ENGINE_AUTO, ENGINE_DIRECT, ENGINE_TENSOR, ENGINE_TCGEN05 = 0, 1, 2, 3


class dc_tune(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("engine", ctypes.c_int32)]


class dc_frame(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("faces", ctypes.c_void_p),
                ("face_mask", ctypes.c_void_p), ("draws", ctypes.c_void_p),
                ("targets", ctypes.c_void_p),
                ("V", ctypes.c_int32), ("F", ctypes.c_int32), ("N", ctypes.c_int32),
                ("M", ctypes.c_int32), ("weight", ctypes.c_float), ("tag", ctypes.c_int32),
                ("loss", ctypes.c_void_p), ("grad_verts", ctypes.c_void_p),
                ("nn_ab", ctypes.c_void_p), ("nn_ba", ctypes.c_void_p)]


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libdiffcloud.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(
                    f"{_build.LIB} is missing: build it with `python -c \"import "
                    f"__graft_entry__ as g; g.build()\"` (nvcc, sm_103a)")
            L = ctypes.CDLL(_build.LIB)
            P, I, S, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
            sig = {
                "dc_workspace_size": (S, [I, I, I, I, I]),
                "dc_sample": (I, [P, P, P, P, I, I, I, I, P, P, P, P, S, P]),
                "dc_area_cdf": (I, [P, P, P, I, I, I, P, P, S, P]),
                "dc_chamfer_fwd": (I, [P, P, I, I, I, I, P, P, P, P, S, P]),
                "dc_chamfer_bwd": (I, [P, P, P, P, I, I, I, I, P, P, P]),
                "dc_loss_traj": (I, [P, P, P, P, P, I, I, I, I, I, I, P, P, P, P, P, P, P, S,
                                     P]),
                "dc_loss_traj_bwd": (I, [P, P, P, P, P, I, I, I, I, I, I, P, P, P, P, P, P, P,
                                         S, P]),
                "dc_batch_workspace_size": (S, [P, I]),
                "dc_batch_plan": (I, [P, I, I, P, S, P]),
                "dc_batch_plan_bytes": (S, [P, I, I]),
                "dc_batch_plan_async": (I, [P, I, I, P, S, P, S, P]),
                "dc_loss_total": (I, [P, P, I, P, P]),
                "dc_batch_run": (I, [P, P, P]),
                "dc_ws_status": (I, [P, P]),
                "dc_last_error": (ctypes.c_char_p, []),
                "dc_launch_count": (ctypes.c_longlong, []),
                "dc_prof_start": (I, [I]),
                "dc_prof_stop": (I, [ctypes.POINTER(F), ctypes.POINTER(I)]),
                "dc_loss_traj_noalloc": (I, [P, P, P, P, P, I, I, I, I, I, I, P, P, P, P, P, P,
                                             P, P]),
                "dc_tune_set": (I, [P]),
                "dc_test_inject_stall": (I, []),
                "dc_fp32_fma_rate": (I, [I, I, ctypes.POINTER(ctypes.c_double), P]),
                "dc_tune_get": (I, [P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().dc_last_error().decode()


def _check(rc: int):
    if rc != DC_OK:
        raise DCError(rc, last_error())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(t: torch.Tensor):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("tensors must be on a CUDA device")
    return t.device


def _need(t, name, dtype, shape, dev):
    """t must be a contiguous `dtype` tensor of exactly `shape` on `dev`: the kernels read
    every element through raw device pointers, so anything else would make them read host
    memory or past the end of the buffer."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device != dev:
        raise ValueError(f"{name} must be on {dev} (it is on {t.device})")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype} (it is {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)} (it has {tuple(t.shape)})")
    return t


def _cloud(t, name, dev, T=None):
    """A [T, n, 3] float32 cloud; returns n."""
    if not isinstance(t, torch.Tensor) or t.dim() != 3 or t.shape[2] != 3:
        raise ValueError(f"{name} must be a [T, n, 3] tensor")
    _need(t, name, torch.float32, (t.shape[0] if T is None else T, t.shape[1], 3), dev)
    return t.shape[1]


def _check_mesh(verts, faces, draws=None, targets=None, face_mask=None, frame_w=None,
                nn_ab=None, nn_ba=None, grad_frames=None):
    """Validate the tensors of a trajectory call; returns (device, T, V, F, N, M, mask)."""
    dev = _dev(verts)
    if verts.dim() != 3 or verts.shape[2] != 3:
        raise ValueError("verts must be a [T, V, 3] tensor")
    T, V = verts.shape[0], verts.shape[1]
    _need(verts, "verts", torch.float32, (T, V, 3), dev)
    if not isinstance(faces, torch.Tensor) or faces.dim() != 2 or faces.shape[1] != 3:
        raise ValueError("faces must be an [F, 3] tensor")
    F = faces.shape[0]
    _need(faces, "faces", torch.int32, (F, 3), dev)
    N = _cloud(draws, "draws", dev, T) if draws is not None else 0
    M = _cloud(targets, "targets", dev, T) if targets is not None else 0
    if frame_w is not None:
        _need(frame_w, "frame_w", torch.float32, (T,), dev)
    if grad_frames is not None:
        _need(grad_frames, "grad_frames", torch.float32, (T,), dev)
    if nn_ab is not None:
        _need(nn_ab, "nn_ab", torch.int32, (T, N), dev)
    if nn_ba is not None:
        _need(nn_ba, "nn_ba", torch.int32, (T, M), dev)
    return dev, T, V, F, N, M, _mask(face_mask, F, dev)


def _mask(m, F, dev=None):
    """face_mask: None, or a contiguous uint8 (or bool) tensor of one entry per face on the
    call's device."""
    if m is None:
        return None
    if m.dtype == torch.bool:
        m = m.to(torch.uint8)
    if (m.dtype != torch.uint8 or not m.is_contiguous() or not m.is_cuda or m.numel() != F
            or (dev is not None and m.device != dev)):
        raise ValueError("face_mask must be a contiguous uint8 CUDA tensor with one entry per "
                         "face, on the device of verts")
    return m


# one workspace per (device, stream): calls on one stream are ordered, so they may share it
_ws_cache: dict = {}


def workspace(nbytes: int, device) -> torch.Tensor:
    key = (torch.device(device).index, torch.cuda.current_stream(device).cuda_stream)
    ws = _ws_cache.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _ws_cache[key] = ws
    return ws


def ws_status(ws: torch.Tensor, stream=None) -> int:
    """Device-side status of the calls issued on `stream` (default: current) with ws."""
    s = _stream(ws.device) if stream is None else ctypes.c_void_p(stream.cuda_stream)
    return int(lib().dc_ws_status(_ptr(ws), s))


def check_ws(ws: torch.Tensor):
    rc = ws_status(ws)
    if rc != DC_OK:
        raise DCError(rc, "device-side error recorded in the workspace")


def dc_workspace_size(T, V, F, N, M) -> int:
    return int(lib().dc_workspace_size(T, V, F, N, M))


def dc_area_cdf(verts, faces, face_mask=None, check=False):
    """Per-frame area CDF (Sec. III-B): [T, F] float32 inclusive prefix sums of the face areas
    (0 outside face_mask); the last entry of each row is the frame's total area."""
    dev, T, V, F, _, _, fm = _check_mesh(verts, faces, face_mask=face_mask)
    cdf = torch.empty((T, F), dtype=torch.float32, device=dev)
    nb = dc_workspace_size(T, V, F, 1, 0)
    if nb == 0:
        raise DCError(DC_EINVAL, "bad sizes")
    ws = workspace(nb, dev)
    _check(lib().dc_area_cdf(_ptr(verts), _ptr(faces), _ptr(fm), T, V, F, _ptr(cdf), _ptr(ws),
                             ws.numel(), _stream(dev)))
    if check:
        check_ws(ws)
    return cdf


def dc_sample(verts, faces, draws, face_idx=True, bary=True, check=False, face_mask=None):
    """Area-weighted sampling (Sec. III-B, Eq. 3). verts [T,V,3], faces [F,3], draws [T,N,3];
    face_mask [F] (optional): sample only the faces with a nonzero entry.
    Returns points [T,N,3], face_idx [T,N] and bary [T,N,3] (or None)."""
    dev, T, V, F, N, _, fm = _check_mesh(verts, faces, draws=draws, face_mask=face_mask)
    pts = torch.empty((T, N, 3), dtype=torch.float32, device=dev)
    fi = torch.empty((T, N), dtype=torch.int32, device=dev) if face_idx else None
    bc = torch.empty((T, N, 3), dtype=torch.float32, device=dev) if bary else None
    nb = dc_workspace_size(T, V, F, N, 0)
    if nb == 0:
        raise DCError(DC_EINVAL, "bad sizes")
    ws = workspace(nb, dev)
    _check(lib().dc_sample(_ptr(verts), _ptr(faces), _ptr(fm), _ptr(draws), T, V, F, N,
                           _ptr(pts), _ptr(fi), _ptr(bc), _ptr(ws), ws.numel(), _stream(dev)))
    if check:
        check_ws(ws)
    return pts, fi, bc


def dc_chamfer_fwd(a, b, mode=BIDIR_MEAN, check=False):
    """Chamfer distance per frame (Eq. 1 / Eq. 2). a [T,N,3], b [T,M,3].
    Returns loss [T], nn_ab [T,N], nn_ba [T,M] (None in Eq. 2)."""
    dev = _dev(a)
    N = _cloud(a, "a", dev)
    T = a.shape[0]
    M = _cloud(b, "b", dev, T)
    loss = torch.empty(T, dtype=torch.float32, device=dev)
    nn_ab = torch.empty((T, N), dtype=torch.int32, device=dev)
    nn_ba = torch.empty((T, M), dtype=torch.int32, device=dev) if mode == BIDIR_MEAN else None
    nb = dc_workspace_size(T, 1, 1, N, M)
    if nb == 0:
        raise DCError(DC_EINVAL, "bad sizes")
    ws = workspace(nb, dev)
    _check(lib().dc_chamfer_fwd(_ptr(a), _ptr(b), T, N, M, mode, _ptr(loss), _ptr(nn_ab),
                                _ptr(nn_ba), _ptr(ws), ws.numel(), _stream(dev)))
    if check:
        check_ws(ws)
    return loss, nn_ab, nn_ba


def dc_chamfer_bwd(a, b, nn_ab, nn_ba, grad_loss, mode=BIDIR_MEAN):
    """Gradient of sum_t g_t L_t w.r.t. a. Returns grad_a [T,N,3]."""
    dev = _dev(a)
    N = _cloud(a, "a", dev)
    T = a.shape[0]
    M = _cloud(b, "b", dev, T)
    _need(nn_ab, "nn_ab", torch.int32, (T, N), dev)
    if mode == BIDIR_MEAN:
        _need(nn_ba, "nn_ba", torch.int32, (T, M), dev)
    _need(grad_loss, "grad_loss", torch.float32, (T,), dev)
    g = torch.empty_like(a)
    _check(lib().dc_chamfer_bwd(_ptr(a), _ptr(b), _ptr(nn_ab),
                                _ptr(nn_ba if mode == BIDIR_MEAN else None), T, N, M, mode,
                                _ptr(grad_loss), _ptr(g), _stream(dev)))
    return g


def dc_loss_traj(verts, faces, draws, targets, mode=BIDIR_MEAN, frame_w=None, grad=True,
                 total=True, nn=True, check=False, out=None, face_mask=None):
    """The whole loss over a trajectory (Sec. III-B, Eq. 1-4).

    verts [T,V,3], faces [F,3], draws [T,N,3], targets [T,M,3] (CUDA, contiguous); face_mask
    [F] (optional): sample only the faces with a nonzero entry; frame_w [T] float32 (optional).
    Returns a dict with loss_total [1] (or None), loss_frames [T], grad_verts [T,V,3] (or
    None), nn_ab [T,N], nn_ba [T,M] (or None). `out` may supply preallocated outputs."""
    dev, T, V, F, N, M, fm = _check_mesh(verts, faces, draws, targets, face_mask, frame_w)
    o = out if out is not None else {}
    lt = o.get("loss_total") if total else None
    if total and lt is None:
        lt = torch.empty(1, dtype=torch.float32, device=dev)
    lf = o.get("loss_frames")
    if lf is None:
        lf = torch.empty(T, dtype=torch.float32, device=dev)
    gv = o.get("grad_verts") if grad else None
    if grad and gv is None:
        gv = torch.empty((T, V, 3), dtype=torch.float32, device=dev)
    nab = nba = None
    if nn:
        nab = o.get("nn_ab")
        if nab is None:
            nab = torch.empty((T, N), dtype=torch.int32, device=dev)
        if mode == BIDIR_MEAN:
            nba = o.get("nn_ba")
            if nba is None:
                nba = torch.empty((T, M), dtype=torch.int32, device=dev)
    if lt is not None:
        _need(lt, "loss_total", torch.float32, (1,), dev)
    _need(lf, "loss_frames", torch.float32, (T,), dev)
    if gv is not None:
        _need(gv, "grad_verts", torch.float32, (T, V, 3), dev)
    if nab is not None:
        _need(nab, "nn_ab", torch.int32, (T, N), dev)
    if nba is not None:
        _need(nba, "nn_ba", torch.int32, (T, M), dev)
    nb = dc_workspace_size(T, V, F, N, M)
    if nb == 0:
        raise DCError(DC_EINVAL, "bad sizes")
    ws = o.get("ws")
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, dev)
    _check(lib().dc_loss_traj(_ptr(verts), _ptr(faces), _ptr(fm), _ptr(draws), _ptr(targets), T,
                              V, F, N, M, mode, _ptr(frame_w), _ptr(lt), _ptr(lf), _ptr(gv),
                              _ptr(nab), _ptr(nba), _ptr(ws), ws.numel(), _stream(dev)))
    if check:
        check_ws(ws)
    return {"loss_total": lt, "loss_frames": lf, "grad_verts": gv, "nn_ab": nab, "nn_ba": nba}


def dc_loss_traj_bwd(verts, faces, draws, targets, nn_ab, nn_ba, grad_frames=None,
                     mode=BIDIR_MEAN, check=False, grad_verts=None, face_mask=None,
                     frame_w=None, grad_total=None):
    """Vertex gradient of an objective J(L_total, L_1..L_T), recomputing the samples from the
    draws. The library forms g_t = dJ/dL_t = w_t grad_total + grad_frames[t] (w_t from
    frame_w, default 1; a missing grad_total or grad_frames counts as 0; a frame of weight 0
    gets g_t = 0, as its forward L_t is the constant 0)."""
    dev, T, V, F, N, M, fm = _check_mesh(
        verts, faces, draws, targets, face_mask, frame_w, nn_ab,
        nn_ba if mode == BIDIR_MEAN else None, grad_frames)
    if grad_total is None and grad_frames is None:
        raise ValueError("grad_total or grad_frames is required")
    if grad_total is not None:
        _need(grad_total, "grad_total", torch.float32, (1,), dev)
    gv = grad_verts if grad_verts is not None else torch.empty_like(verts)
    _need(gv, "grad_verts", torch.float32, (T, V, 3), dev)
    nb = dc_workspace_size(T, V, F, N, M)
    if nb == 0:
        raise DCError(DC_EINVAL, "bad sizes")
    ws = workspace(nb, dev)
    _check(lib().dc_loss_traj_bwd(_ptr(verts), _ptr(faces), _ptr(fm), _ptr(draws), _ptr(targets),
                                  T, V, F, N, M, mode, _ptr(nn_ab),
                                  _ptr(nn_ba if mode == BIDIR_MEAN else None), _ptr(frame_w),
                                  _ptr(grad_total), _ptr(grad_frames), _ptr(gv), _ptr(ws),
                                  ws.numel(), _stream(dev)))
    if check:
        check_ws(ws)
    return gv


def dc_loss_total(loss_frames, frame_w=None, out=None):
    """sum_t w_t L_t of per-frame losses on the device, in the library's fixed order."""
    dev = _dev(loss_frames)
    T = loss_frames.numel()
    _need(loss_frames, "loss_frames", torch.float32, (T,), dev)
    if frame_w is not None:
        _need(frame_w, "frame_w", torch.float32, (T,), dev)
    lt = out if out is not None else torch.empty(1, dtype=torch.float32, device=dev)
    _need(lt, "loss_total", torch.float32, (1,), dev)
    _check(lib().dc_loss_total(_ptr(loss_frames), _ptr(frame_w), T, _ptr(lt), _stream(dev)))
    return lt


def launch_count() -> int:
    return int(lib().dc_launch_count())


def prof_start(cap: int):
    _check(lib().dc_prof_start(cap))


def prof_stop() -> tuple[float, int]:
    ms = ctypes.c_float(0.0)
    n = ctypes.c_int(0)
    _check(lib().dc_prof_stop(ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def dc_loss_traj_noalloc(verts, faces, draws, targets, mode=BIDIR_MEAN, frame_w=None,
                         grad=True, check=False, face_mask=None):
    """dc_loss_traj on the library's built-in 16 MiB scratch array instead of a workspace,
    for callers that cannot allocate device memory when they need the loss. The outputs are
    allocated here for convenience; a caller that cannot allocate passes its own buffers to
    the C function directly. check=True reads the device-side status the call wrote."""
    dev, T, V, F, N, M, fm = _check_mesh(verts, faces, draws, targets, face_mask, frame_w)
    lt = torch.empty(1, dtype=torch.float32, device=dev)
    lf = torch.empty(T, dtype=torch.float32, device=dev)
    gv = torch.empty((T, V, 3), dtype=torch.float32, device=dev) if grad else None
    nab = torch.empty((T, N), dtype=torch.int32, device=dev)
    nba = torch.empty((T, M), dtype=torch.int32, device=dev) if mode == BIDIR_MEAN else None
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().dc_loss_traj_noalloc(_ptr(verts), _ptr(faces), _ptr(fm), _ptr(draws),
                                      _ptr(targets), T, V, F, N, M, mode, _ptr(frame_w),
                                      _ptr(lt), _ptr(lf), _ptr(gv), _ptr(nab), _ptr(nba),
                                      _ptr(st), _stream(dev)))
    if check:
        code = int(st.item())
        if code != DC_OK:
            raise DCError(code, "device-side error reported by dc_loss_traj_noalloc")
    return {"loss_total": lt, "loss_frames": lf, "grad_verts": gv, "nn_ab": nab, "nn_ba": nba}


def tune_set(warps_per_cta: int = 0, engine: int = ENGINE_AUTO):
    """Nearest-neighbour engine (ENGINE_AUTO, ENGINE_DIRECT, ENGINE_TENSOR or ENGINE_TCGEN05)
    and the direct engine's CTA width (1, 2 or 4 warps; 0: automatic) for every later call
    and plan."""
    t = dc_tune(int(warps_per_cta), int(engine))
    _check(lib().dc_tune_set(ctypes.byref(t)))


def tune_get() -> tuple[int, int]:
    """(warps_per_cta, engine) currently set."""
    t = dc_tune(0, 0)
    _check(lib().dc_tune_get(ctypes.byref(t)))
    return int(t.warps_per_cta), int(t.engine)


def fp32_fma_rate(packed: bool, iters: int = 20000, device=None) -> float:
    """Measured FP32 FMA throughput of the device in flop/s (scalar or packed f32x2 FMAs)."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    r = ctypes.c_double(0.0)
    with torch.cuda.device(dev):
        _check(lib().dc_fp32_fma_rate(int(bool(packed)), int(iters), ctypes.byref(r),
                                      _stream(dev)))
    return float(r.value)


def test_inject_stall():
    """Make the next Chamfer launch's bounded waits give up (DC_ETIMEOUT), for tests."""
    _check(lib().dc_test_inject_stall())
