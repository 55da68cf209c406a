"""Batched frames of uneven sizes in one launch sequence (and its CUDA-graph replay) against
the FP64 oracle and against the plain per-frame form (GB300 only)."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def trajs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tr = W.batched_uneven(n_traj=4, grid=(12, 30), T=(3, 5), m=(300, 3000))
    return [parity.nudged(t) for t in tr]


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_oracle(trajs, graph, mode):
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    dts = [DeviceTrajectory.from_host(t, DEV) for t in trajs]
    weights = [np.linspace(0.5, 1.5, t.T) for t in trajs]
    b = BatchedLoss(dts, mode=mode, weights=weights, grad=True, graph=graph, nn=True)
    for _ in range(2):  # replays give the same answer
        total = b.run(check=True)
        torch.cuda.synchronize()
    ref_total = 0.0
    for k, t in enumerate(trajs):
        ref = oracle.loss_traj(t, mode=mode, weights=weights[k])
        parity.check_loss(b.loss_frames[k].cpu().numpy(), ref["loss_frames"])
        parity.check_grad(b.grad_verts[k].cpu().numpy(), ref["grad_verts"])
        for f in range(t.T):
            n0, n1 = t.n_off[f], t.n_off[f + 1]
            per = ref["frames"][f]
            nba = None
            if mode == 0:
                nba = b.nn_ba[k][t.m_off[f]:t.m_off[f + 1]].cpu().numpy()
            parity.check_nn(b.nn_ab[k][n0:n1].cpu().numpy(), per["nn_ab"], nba,
                            per["nn_ba"] if mode == 0 else None)
        ref_total += ref["loss_total"]
    parity.check_loss([float(total[0])], [ref_total], what="batch total")


def test_batch_skips_zero_weight_frames(trajs):
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    dts = [DeviceTrajectory.from_host(t, DEV) for t in trajs]
    weights = [np.where(np.arange(t.T) % 2 == 0, 0.0, 1.0) for t in trajs]
    b = BatchedLoss(dts, weights=weights, grad=True)
    b.run(check=True)
    torch.cuda.synchronize()
    for k, t in enumerate(trajs):
        live = [f for f in range(t.T) if weights[k][f] != 0.0]
        dead = [f for f in range(t.T) if weights[k][f] == 0.0]
        ref = oracle.loss_traj(t, weights=weights[k], frames=live)
        lf = b.loss_frames[k].cpu().numpy()
        gv = b.grad_verts[k].cpu().numpy()
        parity.check_loss(lf[live], ref["loss_frames"][live])
        parity.check_grad(gv[live], ref["grad_verts"][live])
        assert np.all(lf[dead] == 0.0) and np.all(gv[dead] == 0.0)


def test_batch_with_face_subsets(trajs):
    """Each trajectory samples its own face subset (alternate trajectories: the upper half of
    the cloth, or every face); the batch matches the oracle with the same masks."""
    import copy

    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    mtr = []
    for k, t in enumerate(trajs):
        t = copy.copy(t)
        n = int(round(t.V ** 0.5))
        t.face_mask = W.upper_half_mask(n) if k % 2 == 0 else None
        mtr.append(parity.nudged(t))
    b = BatchedLoss([DeviceTrajectory.from_host(t, DEV) for t in mtr], grad=True)
    b.run(check=True)
    torch.cuda.synchronize()
    for k, t in enumerate(mtr):
        ref = oracle.loss_traj(t)
        parity.check_loss(b.loss_frames[k].cpu().numpy(), ref["loss_frames"])
        parity.check_grad(b.grad_verts[k].cpu().numpy(), ref["grad_verts"])


def test_batch_equals_per_frame_form(trajs):
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory, per_frame_loss

    dts = [DeviceTrajectory.from_host(t, DEV) for t in trajs]
    b = BatchedLoss(dts, grad=True, graph=True)
    b.run(check=True)
    lf, gv = per_frame_loss(dts)
    torch.cuda.synchronize()
    for k in range(len(dts)):
        # the same kernels; the loss partial sums may be cut into different slices
        np.testing.assert_allclose(b.loss_frames[k].cpu().numpy(), lf[k].cpu().numpy(),
                                   rtol=1e-6)
        assert parity.rel_l2(b.grad_verts[k].cpu().numpy(), gv[k].cpu().numpy()) < 1e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_engines_agree(trajs, mode):
    """One batch plan per engine (warp-level MMA filter, tcgen05 filter, direct form): the
    neighbours and per-frame losses agree bit for bit, gradients to float rounding of the
    scatter order, and the tcgen05 plan matches the oracle."""
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    dts = [DeviceTrajectory.from_host(t, DEV) for t in trajs]
    outs = {}
    for sh in (("tensor", 0), ("tcgen05", 0), ("direct", 2)):
        b = BatchedLoss(dts, mode=mode, grad=True, graph=True, nn=True, shape=sh)
        b.run(check=True)
        torch.cuda.synchronize()
        outs[sh[0]] = b
    ref = outs["direct"]
    for eng in ("tensor", "tcgen05"):
        b = outs[eng]
        for k in range(len(dts)):
            np.testing.assert_array_equal(b.loss_frames[k].cpu().numpy(),
                                          ref.loss_frames[k].cpu().numpy())
            np.testing.assert_array_equal(b.nn_ab[k].cpu().numpy(), ref.nn_ab[k].cpu().numpy())
            if mode == 0:
                np.testing.assert_array_equal(b.nn_ba[k].cpu().numpy(),
                                              ref.nn_ba[k].cpu().numpy())
            assert parity.rel_l2(b.grad_verts[k].cpu().numpy(),
                                 ref.grad_verts[k].cpu().numpy()) < 1e-6
    for k, t in enumerate(trajs):
        o = oracle.loss_traj(t, mode=mode)
        parity.check_loss(outs["tcgen05"].loss_frames[k].cpu().numpy(), o["loss_frames"])


@pytest.mark.timeout(180)
@pytest.mark.parametrize("shape", [("tensor", 0), ("tcgen05", 0)])
def test_bounded_waits_with_units_handed_out_on_demand(shape):
    """1000 frames of 2048 points (8000 tensor-core units, many more than CTAs): the passes
    hand out whole units from a counter. A launch whose first chunk is never requested in
    any CTA must end with DC_ETIMEOUT, the next run of the same plan must give the normal
    result, and its per-frame losses equal the direct engine's."""
    from paper_2204_03139_gb300 import _lib
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    trs = [W.lift_trajectory(W.SEED_BASE + 900 + k, 12, 100, 2048, 2048, name=f"d{k}")
           for k in range(10)]
    b = BatchedLoss([DeviceTrajectory.from_host(t, DEV) for t in trs], grad=True, shape=shape)
    good = b.run(check=True).cpu().numpy().copy()
    _lib.test_inject_stall()
    b.run()
    torch.cuda.synchronize()
    assert _lib.ws_status(b.ws, b.stream) == _lib.DC_ETIMEOUT
    again = b.run(check=True).cpu().numpy()
    np.testing.assert_array_equal(again, good)
    # and in this mode the filter's per-frame losses equal the direct engine's bit for bit
    ref = BatchedLoss([DeviceTrajectory.from_host(t, DEV) for t in trs], grad=True,
                      shape=("direct", 2))
    ref.run(check=True)
    torch.cuda.synchronize()
    for k in range(len(trs)):
        np.testing.assert_array_equal(b.loss_frames[k].cpu().numpy(),
                                      ref.loss_frames[k].cpu().numpy())


@pytest.mark.slow
def test_batched_uneven_full_size_sampled_frames():
    """All 64 trajectories of the uneven workload (grids 15x15..80x80, 20..100 frames, 2 000 to
    30 000 points per frame) in one batch, as the bench runs it; the oracle checks the first,
    middle and last frame of three trajectories."""
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    trajs = [parity.nudged(t) for t in W.batched_uneven()]
    dts = [DeviceTrajectory.from_host(t, DEV) for t in trajs]
    b = BatchedLoss(dts, grad=True, graph=True, nn=True)
    b.run(check=True)
    torch.cuda.synchronize()
    for k in (0, 31, 63):
        t = trajs[k]
        frames = sorted({0, t.T // 2, t.T - 1})
        ref = oracle.loss_traj(t, frames=frames)
        parity.check_loss(b.loss_frames[k].cpu().numpy()[frames], ref["loss_frames"][frames])
        parity.check_grad(b.grad_verts[k].cpu().numpy()[frames], ref["grad_verts"][frames])
        for f in frames:
            n0, n1 = t.n_off[f], t.n_off[f + 1]
            m0, m1 = t.m_off[f], t.m_off[f + 1]
            parity.check_nn(b.nn_ab[k][n0:n1].cpu().numpy(), ref["frames"][f]["nn_ab"],
                            b.nn_ba[k][m0:m1].cpu().numpy(), ref["frames"][f]["nn_ba"])
