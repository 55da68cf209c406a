"""dc_loss_traj_noalloc, the entry point for callers that cannot allocate device memory when
they need the loss (a plug-in whose host framework owns all device memory, a real-time loop
that forbids allocator calls after start-up). It runs on the library's built-in scratch
array; here it is checked, through the C ABI, against dc_loss_traj with a workspace, on two
calls in a row (the scratch keeps the previous call's contents). This file sorts last so
that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import parity
import workloads as W

pytestmark = pytest.mark.gpu

NOALLOC_SCRATCH_BYTES = 16 << 20  # the built-in scratch of dc_loss_traj_noalloc


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _inputs(dev, tr):
    return (torch.from_numpy(tr.verts).to(dev), torch.from_numpy(tr.faces).to(dev),
            torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).to(dev),
            torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).to(dev))


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_workspace_entry_point_twice(mode):
    from paper_2204_03139_gb300 import _lib

    dev = _dev()
    cases = [W.single_frame(), W.trajectory_50x50(T=3, n=4000, m=3000)]
    for tr in cases:
        v, f, d, y = _inputs(dev, tr)
        ref = _lib.dc_loss_traj(v, f, d, y, mode=mode, check=True)
        for _ in range(2):  # two calls in a row on the shared scratch
            got = _lib.dc_loss_traj_noalloc(v, f, d, y, mode=mode, check=True)
            torch.cuda.synchronize()
            parity.check_loss(got["loss_frames"].cpu().numpy(), ref["loss_frames"].cpu().numpy())
            parity.check_loss(got["loss_total"].cpu().numpy(), ref["loss_total"].cpu().numpy())
            parity.check_grad(got["grad_verts"].cpu().numpy(), ref["grad_verts"].cpu().numpy())
            np.testing.assert_array_equal(got["nn_ab"].cpu().numpy(), ref["nn_ab"].cpu().numpy())
            if mode == 0:
                np.testing.assert_array_equal(got["nn_ba"].cpu().numpy(),
                                              ref["nn_ba"].cpu().numpy())


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2204_03139_gb300 import _lib

    _dev()
    L = _lib.lib()
    # The pointers below are not device memory: the call must fail on the size check before
    # any launch. So the problem is sized on the host first, well beyond the scratch, and the
    # test refuses to make the call if it is not.
    T, V, F, N, M = 16, 2500, 4802, 10000, 10000
    while _lib.dc_workspace_size(T, V, F, N, M) <= 4 * NOALLOC_SCRATCH_BYTES:
        T *= 2
    assert _lib.dc_workspace_size(T, V, F, N, M) > 4 * NOALLOC_SCRATCH_BYTES
    fake = ctypes.c_void_p(0x100000)
    rc = L.dc_loss_traj_noalloc(fake, fake, None, fake, fake, T, V, F, N, M, 0,
                                None, None, fake, None, None, None, None, None)
    assert rc == _lib.DC_ENOSPC
    assert "built-in scratch" in _lib.last_error()


def test_noalloc_reports_device_errors_in_status():
    from paper_2204_03139_gb300 import _lib

    dev = _dev()
    v = torch.zeros((1, 3, 3), device=dev)
    f = torch.tensor([[0, 1, 2]], dtype=torch.int32, device=dev)
    d = torch.full((1, 4, 3), 0.5, device=dev)
    y = torch.zeros((1, 4, 3), device=dev)
    with pytest.raises(_lib.DCError) as e:
        _lib.dc_loss_traj_noalloc(v, f, d, y, check=True)
    assert e.value.code == _lib.DC_EDEGENERATE
