"""The C-ABI library builds, loads and exports every entry point include/diffcloud.h declares,
and rejects bad host-side arguments before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "diffcloud.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2204_03139_gb300 import _lib, build

    if build.stale():
        try:
            build.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    return _lib.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dc_sample", "dc_chamfer_fwd", "dc_chamfer_bwd", "dc_loss_traj",
              "dc_loss_traj_bwd", "dc_workspace_size", "dc_batch_plan", "dc_batch_run",
              "dc_ws_status", "dc_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_workspace_size(L):
    assert L.dc_workspace_size(0, 1, 1, 1, 1) == 0
    assert L.dc_workspace_size(1, 1, 1, 0, 1) == 0
    a = L.dc_workspace_size(1, 625, 1152, 2048, 2048)
    b = L.dc_workspace_size(40, 2500, 4802, 10000, 10000)
    c = L.dc_workspace_size(100, 10000, 19602, 32768, 32768)
    assert 0 < a < b < c
    assert a % 256 == 0 and b % 256 == 0 and c % 256 == 0
    # at least the padded point buffers: 16 B points + 16 B picks + 8 B minima per row
    assert c >= 100 * 32768 * (16 + 16 + 8)
    # far beyond 32-bit offsets is refused
    assert L.dc_workspace_size(100000, 3, 1, 1 << 20, 1 << 20) == 0


FAKE = ctypes.c_void_p(0x100000)  # never dereferenced: validation fails first


def test_host_side_validation(L):
    from paper_2204_03139_gb300 import _lib

    rc = L.dc_loss_traj(None, FAKE, None, FAKE, FAKE, 1, 3, 1, 4, 4, 0, None, None,
                        FAKE, None, None, None, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL and "NULL" in _lib.last_error()
    rc = L.dc_loss_traj(FAKE, FAKE, None, FAKE, FAKE, 1, 3, 1, 0, 4, 0, None, None,
                        FAKE, None, None, None, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL
    rc = L.dc_loss_traj(FAKE, FAKE, None, FAKE, FAKE, 1, 3, 1, 4, 4, 7, None, None,
                        FAKE, None, None, None, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL and "mode" in _lib.last_error()
    # workspace too small / misaligned
    rc = L.dc_loss_traj(FAKE, FAKE, None, FAKE, FAKE, 1, 3, 1, 4, 4, 0, None, None,
                        FAKE, None, None, None, FAKE, 16, None)
    assert rc == _lib.DC_ENOSPC
    rc = L.dc_loss_traj(FAKE, FAKE, None, FAKE, FAKE, 1, 3, 1, 4, 4, 0, None, None,
                        FAKE, None, None, None, ctypes.c_void_p(0x100010), 1 << 30, None)
    assert rc == _lib.DC_EINVAL and "aligned" in _lib.last_error()
    # misaligned data pointer
    rc = L.dc_chamfer_fwd(ctypes.c_void_p(0x100002), FAKE, 1, 4, 4, 0, FAKE, None, None, FAKE,
                          1 << 20, None)
    assert rc == _lib.DC_EINVAL
    rc = L.dc_chamfer_bwd(FAKE, FAKE, FAKE, None, 1, 4, 4, 0, FAKE, FAKE, None)
    assert rc == _lib.DC_EINVAL and "nn_ba" in _lib.last_error()
    rc = L.dc_sample(FAKE, FAKE, None, FAKE, 1, 3, 1, -1, FAKE, None, None, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL


NOALLOC_SCRATCH_BYTES = 16 << 20  # the built-in scratch of dc_loss_traj_noalloc


def test_noalloc_rejects_problems_beyond_its_scratch(L):
    """dc_loss_traj_noalloc refuses a problem whose workspace exceeds its built-in scratch
    before it looks at any pointer or makes any CUDA call: every pointer here is NULL, so a
    regression of that order would fail with DC_EINVAL instead, and nothing would launch."""
    from paper_2204_03139_gb300 import _lib

    # 512 frames of 10 000 x 10 000: the sampled points alone (16 B each, before any other
    # region) take 82 MB, more than four times the scratch, whatever the engine's layout
    T, V, F, N, M = 512, 2500, 4802, 10000, 10000
    assert T * N * 16 > 4 * NOALLOC_SCRATCH_BYTES
    rc = L.dc_loss_traj_noalloc(None, None, None, None, None, T, V, F, N, M, 0,
                                None, None, None, None, None, None, None, None)
    assert rc == _lib.DC_ENOSPC
    assert "built-in scratch" in _lib.last_error()
    # one that fits gets as far as the pointer checks
    rc = L.dc_loss_traj_noalloc(None, None, None, None, None, 1, 625, 1152, 2048, 2048, 0,
                                None, None, None, None, None, None, None, None)
    assert rc == _lib.DC_EINVAL and "NULL" in _lib.last_error()


def test_loss_traj_bwd_needs_an_upstream_gradient(L):
    from paper_2204_03139_gb300 import _lib

    rc = L.dc_loss_traj_bwd(FAKE, FAKE, None, FAKE, FAKE, 1, 3, 1, 4, 4, 0, FAKE, FAKE,
                            None, None, None, FAKE, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL and "grad_total or grad_frames" in _lib.last_error()


def test_binding_validates_tensors():
    """The Python binding refuses tensors of the wrong device, dtype, shape or layout before
    any pointer reaches the library (checked with CPU tensors, which are refused first)."""
    import torch

    from paper_2204_03139_gb300 import _lib

    v = torch.zeros((2, 3, 3))
    f = torch.zeros((1, 3), dtype=torch.int32)
    with pytest.raises(ValueError):
        _lib._check_mesh(v, f)
    meta = torch.device("meta")
    vm = torch.zeros((2, 3, 3), device=meta)
    with pytest.raises(ValueError):  # not CUDA
        _lib._check_mesh(vm, f.to(meta))


def test_batch_validation(L):
    from paper_2204_03139_gb300 import _lib

    fr = (_lib.dc_frame * 2)()
    for k in range(2):
        fr[k].verts = fr[k].faces = fr[k].draws = fr[k].targets = 0x100000
        fr[k].V, fr[k].F, fr[k].N, fr[k].M = 3, 1, 5, 7
        fr[k].weight = 1.0
    assert L.dc_batch_workspace_size(fr, 2) > 0
    fr[1].M = 0
    assert L.dc_batch_workspace_size(fr, 2) == 0
    rc = L.dc_batch_plan(fr, 2, 0, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL and "frame 1" in _lib.last_error()
    fr[1].M = 7
    fr[0].targets = None
    rc = L.dc_batch_plan(fr, 2, 0, FAKE, 1 << 20, None)
    assert rc == _lib.DC_EINVAL
    rc = L.dc_batch_run(ctypes.c_void_p(0x200000), None, None)
    assert rc == _lib.DC_EINVAL and "plan" in _lib.last_error()


def test_product_path_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2204_03139_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "liboracle" not in src and "diffcloud_oracle" not in src, f
