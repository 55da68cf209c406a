"""dc_loss_traj_noalloc, the entry point for callers that cannot allocate device memory when
they need the loss (a plug-in whose host framework owns all device memory, a real-time loop
that forbids allocator calls after start-up). It runs on the library's built-in scratch
array; here it is checked, through the C ABI, against dc_loss_traj with a workspace, on two
calls in a row (the scratch keeps the previous call's contents). This file sorts last so
that a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

import parity
import workloads as W

pytestmark = pytest.mark.gpu


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
    """Two calls in a row per case, the larger problem first, so that the smaller one runs on
    scratch still holding the larger one's data; then the smaller one again with other draws
    and targets and a frame of weight 0. Each result equals dc_loss_traj's on a workspace of
    its own."""
    from paper_2204_03139_gb300 import _lib

    dev = _dev()
    big = W.trajectory_50x50(T=3, n=4000, m=3000)
    small = W.single_frame()
    other = W.lift_trajectory(5, 25, 2, 2048, 2048, name="other")
    cases = [(big, None), (small, None), (other, [0.0, 1.0]), (big, [1.0, 0.0, 2.0])]
    for tr, w in cases:
        v, f, d, y = _inputs(dev, tr)
        fw = None if w is None else torch.tensor(w, dtype=torch.float32, device=dev)
        fresh = torch.empty(_lib.dc_workspace_size(tr.T, tr.V, tr.F, tr.n(0), tr.m(0)),
                            dtype=torch.uint8, device=dev)
        ref = _lib.dc_loss_traj(v, f, d, y, mode=mode, frame_w=fw, check=True,
                                out={"ws": fresh})
        for _ in range(2):  # two calls in a row on the shared scratch
            got = _lib.dc_loss_traj_noalloc(v, f, d, y, mode=mode, frame_w=fw, check=True)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got["loss_frames"].cpu().numpy(),
                                          ref["loss_frames"].cpu().numpy())
            parity.check_loss(got["loss_total"].cpu().numpy(), ref["loss_total"].cpu().numpy())
            parity.check_grad(got["grad_verts"].cpu().numpy(), ref["grad_verts"].cpu().numpy())
            # neighbours of the frames that ran (a skipped frame's are not written)
            live = [t for t in range(tr.T) if w is None or w[t] != 0.0]
            np.testing.assert_array_equal(got["nn_ab"].cpu().numpy()[live],
                                          ref["nn_ab"].cpu().numpy()[live])
            if mode == 0:
                np.testing.assert_array_equal(got["nn_ba"].cpu().numpy()[live],
                                              ref["nn_ba"].cpu().numpy()[live])
            if w is not None:
                dead = [t for t in range(tr.T) if w[t] == 0.0]
                assert np.all(got["loss_frames"].cpu().numpy()[dead] == 0.0)
                assert np.all(got["grad_verts"].cpu().numpy()[dead] == 0.0)


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
