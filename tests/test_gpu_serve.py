"""Continuous-batching server (GB300 only): results alone vs in a mix, admission under an HBM
budget, error propagation."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def _mix(n, seed=7):
    rng = W.rng_for(seed)
    out = []
    for k in range(n):
        g = int(rng.integers(10, 40))
        T = int(rng.integers(2, 6))
        m = int(rng.integers(300, 4000))
        out.append(parity.nudged(
            W.lift_trajectory(int(rng.integers(1 << 30)), g, T, m, m, name=f"mix{k}")))
    return out


def test_result_alone_equals_result_in_mix(dev):
    from paper_2204_03139_gb300.serve import Server

    reqs = _mix(12)
    probe = reqs[5]
    srv = Server(dev, hbm_budget=8 << 30)
    alone = srv.submit(probe).result(timeout=120)
    futs = [srv.submit(r) for r in reqs]
    mixed = [f.result(timeout=120) for f in futs]
    srv.close()
    together = mixed[5]
    # the same kernels: neighbours identical, losses equal up to the order of slice sums
    np.testing.assert_allclose(together.loss_frames, alone.loss_frames, rtol=1e-6)
    assert parity.rel_l2(together.grad_verts, alone.grad_verts) < 1e-6
    assert max(r.batch_requests for r in mixed) > 1  # requests really were batched together
    # and every request of the mix matches the oracle
    for r, res in zip(reqs, mixed):
        ref = oracle.loss_traj(r)
        parity.check_loss(res.loss_frames, ref["loss_frames"])
        parity.check_grad(res.grad_verts, ref["grad_verts"])


def test_admission_under_a_small_budget(dev):
    from paper_2204_03139_gb300.serve import Server, request_bytes

    reqs = _mix(6, seed=9)
    biggest = max(request_bytes(r) for r in reqs)
    srv = Server(dev, hbm_budget=biggest + 1024)  # room for about one request at a time
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=120) for f in futs]
    srv.close()
    assert all(r.batch_requests >= 1 for r in res)
    for r, out in zip(reqs, res):
        ref = oracle.loss_traj(r)
        parity.check_loss(out.loss_frames, ref["loss_frames"])
    # a request larger than the whole budget is refused at once
    srv = Server(dev, hbm_budget=1 << 20)
    f = srv.submit(reqs[0])
    with pytest.raises(Exception) as e:
        f.result(timeout=10)
    assert "budget" in str(e.value)
    srv.close()


def test_device_error_fails_only_its_batch(dev):
    from paper_2204_03139_gb300.serve import Server

    bad = W.lift_trajectory(3, 6, 2, 50, 50, name="bad")
    bad.verts[:] = 0.0  # zero area: DC_EDEGENERATE
    good = _mix(1, seed=3)[0]
    srv = Server(dev, hbm_budget=4 << 30, streams=1)
    fb = srv.submit(bad)
    with pytest.raises(Exception):
        fb.result(timeout=60)
    fg = srv.submit(good)
    out = fg.result(timeout=60)
    srv.close()
    ref = oracle.loss_traj(good)
    parity.check_loss(out.loss_frames, ref["loss_frames"])


@pytest.mark.slow
def test_config5_sizes_alone_equals_in_mix(dev):
    """Requests of the serving mix's two sizes (50x50 / 40 frames / 10 000 points and
    100x100 / 100 frames / 32 768 points): each result in a mix equals the one the request gets
    alone, and a request of each size matches the oracle."""
    from paper_2204_03139_gb300.serve import Server

    small = [parity.nudged(W.lift_trajectory(W.SEED_BASE + 50 + k, 50, 40, 10_000, 10_000,
                                             name=f"small{k}")) for k in range(3)]
    big = parity.nudged(W.trajectory_100x100(seed=W.SEED_BASE + 60))
    srv = Server(dev, hbm_budget=120 << 30)
    alone_small = srv.submit(small[0]).result(timeout=600)
    alone_big = srv.submit(big).result(timeout=600)
    futs = [srv.submit(r) for r in (small[1], big, small[0], small[2])]
    mixed = [f.result(timeout=600) for f in futs]
    srv.close()
    for a, m in ((alone_big, mixed[1]), (alone_small, mixed[2])):
        np.testing.assert_allclose(m.loss_frames, a.loss_frames, rtol=1e-6)
        assert parity.rel_l2(m.grad_verts, a.grad_verts) < 1e-6
    assert max(r.batch_requests for r in mixed) > 1
    for tr, res in ((small[0], alone_small), (big, alone_big)):
        ref = oracle.loss_traj(tr)
        parity.check_loss(res.loss_frames, ref["loss_frames"])
        parity.check_loss([res.loss_total], [ref["loss_total"]], what="total")
        parity.check_grad(res.grad_verts, ref["grad_verts"])
