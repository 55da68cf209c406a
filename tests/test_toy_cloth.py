"""The toy real-to-sim loop: parameters -> vertices -> loss -> vertex gradient -> parameters.

The CPU tests check the toy cloth model and the paper's sigmoid reparameterisation; the GPU
tests check that the parameter gradient through this library equals the one built from the
oracle's FP64 vertex gradient, and that Adam recovers the parameters of a synthetic target.
"""

import numpy as np
import pytest
import torch

import oracle
import parity
import workloads as W


def test_sigmoid_reparameterisation():
    """w = sigma(s) (10 - 0.1) + 0.1: s = 0 is the middle of [0.1, 10] (Sec. IV-B)."""
    from paper_2204_03139_gb300.toy_cloth import params_from_s, s_from_params

    w = params_from_s(torch.tensor([0.0, -40.0, 40.0], dtype=torch.float64))
    np.testing.assert_allclose(w.numpy(), [5.05, 0.1, 10.0], rtol=1e-12)
    s = s_from_params([2.0, 7.5])
    np.testing.assert_allclose(params_from_s(s).numpy(), [2.0, 7.5], rtol=1e-12)


def test_toy_cloth_is_differentiable_and_lifts_the_corner():
    from paper_2204_03139_gb300.toy_cloth import ToyCloth

    cl = ToyCloth(n=6, T=4, device="cpu", dtype=torch.float64)
    w = torch.tensor([2.0, 7.5], dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(cl.verts, (w,), eps=1e-6, atol=1e-6)
    v = cl.verts(w).detach()
    assert v.shape == (4, 36, 3)
    assert torch.all(v[0, :, 2].abs() < 2e-3)          # frame 0: flat on the table
    np.testing.assert_allclose(v[-1, 0].numpy(), [0.2, 0.2, 0.5], atol=3e-3)  # grasped corner
    # heavier cloth hangs more steeply: less of it is off the table in the last frame
    light = cl.verts(torch.tensor([2.0, 1.0], dtype=torch.float64))[-1, :, 2]
    heavy = cl.verts(torch.tensor([2.0, 9.0], dtype=torch.float64))[-1, :, 2]
    assert (light > 0.01).sum() > (heavy > 0.01).sum()


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1])
def test_parameter_gradient_through_the_library_matches_the_oracle(mode):
    """dL/ds through this library's vertex gradient equals dL/ds chained from the oracle's
    FP64 vertex gradient through the same torch model (the model's part is exact in both)."""
    from paper_2204_03139_gb300.autograd import loss_traj
    from paper_2204_03139_gb300.toy_cloth import ToyCloth, params_from_s, sample_targets

    dev = _gpu()
    cl = ToyCloth(n=20, T=5, device=dev)
    Y = sample_targets(cl, [2.0, 7.5], 3000, seed=4)
    s = torch.tensor([0.3, -0.2], dtype=torch.float64, device=dev, requires_grad=True)
    verts = cl.verts(params_from_s(s)).float()
    rng = np.random.default_rng(5)
    n = 2500
    draws = W.uniform_draws(rng, cl.T * n)
    tr = W.Trajectory(verts=verts.detach().cpu().numpy(), faces=cl.faces.cpu().numpy(),
                      draws=draws, targets=Y.cpu().numpy().reshape(-1, 3),
                      n_off=np.arange(cl.T + 1, dtype=np.int64) * n,
                      m_off=np.arange(cl.T + 1, dtype=np.int64) * Y.shape[1])
    tr = parity.nudged(tr)
    d = torch.from_numpy(tr.draws.reshape(cl.T, n, 3)).to(dev)
    total, lf = loss_traj(verts, cl.faces, d, Y, mode=mode)
    (g_lib,) = torch.autograd.grad(total, s)
    ref = oracle.loss_traj(tr, mode=mode)
    parity.check_loss(lf.detach().cpu().numpy(), ref["loss_frames"])
    verts2 = cl.verts(params_from_s(s)).float()
    (g_orc,) = torch.autograd.grad(verts2, s, grad_outputs=torch.from_numpy(
        ref["grad_verts"].astype(np.float32)).to(dev))
    assert parity.rel_l2(g_lib.cpu().numpy(), g_orc.cpu().numpy()) < 1e-4


@pytest.mark.gpu
def test_real_to_sim_recovers_the_parameters():
    """Adam on s from the middle of the range (learning rate 0.2, 50 iterations, Eq. 2 loss,
    fresh samples every iteration) recovers (w_stiff, w_mass) = (2, 7.5) of a synthetic
    target with 2 mm noise; the last-frame-only variant runs on one frame's work."""
    from paper_2204_03139_gb300.toy_cloth import ToyCloth, real_to_sim, sample_targets

    dev = _gpu()
    cl = ToyCloth(n=20, T=6, device=dev)
    Y = sample_targets(cl, [2.0, 7.5], 8192, seed=6)
    r = real_to_sim(cl, Y, 8192, iters=50, lr=0.2, seed=7)
    first = r["history"][0][1]
    w = r["w"]
    assert r["loss"] < 0.6 * first
    assert abs(w[0] - 2.0) < 0.35 * 2.0 and abs(w[1] - 7.5) < 0.15 * 7.5, w
    # frames of weight 0 are skipped; the fit still moves toward the truth
    fw = np.zeros(cl.T, np.float32)
    fw[-1] = 1.0
    r1 = real_to_sim(cl, Y, 8192, iters=30, lr=0.2, seed=8, frame_w=fw)
    assert r1["loss"] < r1["history"][0][1]


@pytest.mark.gpu
def test_loss_module_draws_fresh_samples_and_matches_the_function():
    """DiffCloudLoss(verts) equals loss_traj on the draws it used, and draws new ones per call."""
    from paper_2204_03139_gb300.autograd import DiffCloudLoss, loss_traj
    from paper_2204_03139_gb300.toy_cloth import ToyCloth, sample_targets

    dev = _gpu()
    cl = ToyCloth(n=15, T=3, device=dev)
    Y = sample_targets(cl, [2.0, 7.5], 2000, seed=3)
    mod = DiffCloudLoss(cl.faces, Y, 2000, seed=5)
    v = cl.verts(torch.tensor([3.0, 4.0], dtype=torch.float64, device=dev)).float()
    v.requires_grad_(True)
    t1, _ = mod(v)
    d1 = mod.last_draws.clone()
    (g1,) = torch.autograd.grad(t1, v)
    t_ref, _ = loss_traj(v, cl.faces, d1, Y)
    (g_ref,) = torch.autograd.grad(t_ref, v)
    assert float(t1.detach()) == float(t_ref.detach())
    assert parity.rel_l2(g1.cpu().numpy(), g_ref.cpu().numpy()) < 1e-6
    mod(v)
    assert not torch.equal(mod.last_draws, d1)
