"""Pipelined loss + gradient over a stream of trajectories (GB300 only): every step's
results equal the plain call's on the same inputs, with several steps in flight."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_pipeline_matches_plain_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_03139_gb300 import _lib
    from paper_2204_03139_gb300.pipeline import LossPipeline

    dev = torch.device("cuda:0")
    trs = [W.lift_trajectory(100 + k, 20, 4, 3000, 3000, name=f"p{k}") for k in range(5)]
    tr0 = trs[0]
    T, V, F, N, M = tr0.T, tr0.V, tr0.F, tr0.n(0), tr0.m(0)
    pipe = LossPipeline(T, V, F, N, M, device=dev, depth=2)
    host = [tuple(LossPipeline.pin(a) for a in (t.verts, t.faces, t.draws_tn3(), t.targets_tm3()))
            for t in trs]
    outs = [(LossPipeline.pinned((T, V, 3)), LossPipeline.pinned(1), LossPipeline.pinned(T))
            for _ in trs]
    events = []
    for k in range(3):  # the same trajectories again: slots are reused while steps are in flight
        for h, o in zip(host, outs):
            events.append(pipe.submit(*h, grad_out=o[0], loss_out=o[1], frames_out=o[2]))
        for e in events:
            e.synchronize()
        events.clear()
        assert pipe.status() == _lib.DC_OK
        for t, o in zip(trs, outs):
            ref = _lib.dc_loss_traj(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
                                      (t.verts, t.faces, t.draws_tn3(), t.targets_tm3())))
            torch.cuda.synchronize()
            np.testing.assert_array_equal(o[2].numpy(), ref["loss_frames"].cpu().numpy())
            np.testing.assert_array_equal(o[1].numpy(), ref["loss_total"].cpu().numpy())
            g = ref["grad_verts"].cpu().numpy()
            assert np.linalg.norm(o[0].numpy() - g) <= 1e-6 * np.linalg.norm(g)


@pytest.mark.parametrize("shape", [("tensor", 0), ("direct", 2)])
def test_batch_pipeline_matches_single_batches(shape):
    """Three batches of one structure (ragged frames, uneven trajectories) with different
    values, through two slots: every result equals the one a fresh batch plan gives for the
    same inputs, so slot reuse while batches are in flight corrupts nothing."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import copy

    from paper_2204_03139_gb300 import _lib
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory
    from paper_2204_03139_gb300.pipeline import BatchPipeline

    dev = torch.device("cuda:0")
    base = W.batched_uneven(n_traj=3, grid=(12, 24), T=(2, 4), m=(500, 2500))
    batches = []
    for k in range(3):  # the same structure, other values: fresh draws, moved targets
        rng = W.rng_for(500 + k)
        bt = []
        for t in base:
            t = copy.copy(t)
            t.draws = np.clip(rng.random(t.draws.shape), 0, np.nextafter(1, 0)).astype(np.float32)
            t.targets = (t.targets + np.float32(0.01 * k)).astype(np.float32)
            t.verts = (t.verts * np.float32(1.0 + 0.02 * k)).astype(np.float32)
            bt.append(t)
        batches.append(bt)
    pipe = BatchPipeline([(t.V, t.F, t.n_off, t.m_off) for t in base], device=dev, depth=2,
                         shape=shape)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    outs, events = [], []
    for bt in batches:
        host = [(pin(t.verts), pin(t.faces), pin(t.draws), pin(t.targets)) for t in bt]
        o = ([torch.empty(t.verts.shape, dtype=torch.float32).pin_memory() for t in bt],
             torch.empty(1, dtype=torch.float32).pin_memory(),
             [torch.empty(t.T, dtype=torch.float32).pin_memory() for t in bt])
        events.append(pipe.submit(host, grads_out=o[0], total_out=o[1], frames_out=o[2]))
        outs.append((host, o))
    for e in events:
        e.synchronize()
    assert pipe.status() == _lib.DC_OK
    for bt, (host, o) in zip(batches, outs):
        ref = BatchedLoss([DeviceTrajectory.from_host(t, dev) for t in bt], grad=True,
                          shape=shape)
        total = ref.run(check=True)
        torch.cuda.synchronize()
        np.testing.assert_allclose(o[1].numpy(), total.cpu().numpy(), rtol=1e-6)
        for k in range(len(bt)):
            np.testing.assert_allclose(o[2][k].numpy(), ref.loss_frames[k].cpu().numpy(),
                                       rtol=1e-6)
            g = ref.grad_verts[k].cpu().numpy()
            assert np.linalg.norm(o[0][k].numpy() - g) <= 1e-6 * np.linalg.norm(g)


def test_fp32_fma_rate_is_near_the_fp32_peak():
    """The measured FMA rate (the cross-check of the roofline's FP32 peak) lies between 30% and
    110% of 2 x 128 lanes x SMs x 2.1 GHz, for scalar and packed FMAs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_03139_gb300 import _lib

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    top = 2 * 128 * sms * 2.1e9
    for packed in (False, True):
        r = _lib.fp32_fma_rate(packed, iters=5000)
        assert 0.3 * top < r < 1.1 * top, (packed, r / top)
