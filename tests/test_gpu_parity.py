"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GB300 only).

Inputs are the seeded workloads; draws that the oracle finds within 1e-6 of a CDF boundary
are moved to their face's CDF midpoint (parity.nudge_draws) wherever the loss and gradient
are compared, since a point that may fall on either face moves the loss by more than the
loss tolerance; test_raw_draws_face_picks_and_neighbours covers the raw draws.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_03139_gb300 import _lib as L

    L.lib()
    return L


def L():
    from paper_2204_03139_gb300 import _lib as L

    return L


def to_dev(tr):
    return (torch.from_numpy(tr.verts).to(DEV), torch.from_numpy(tr.faces).to(DEV),
            torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).to(DEV),
            torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).to(DEV))


def dev_mask(tr):
    m = getattr(tr, "face_mask", None)
    return None if m is None else torch.from_numpy(np.ascontiguousarray(m, np.uint8)).to(DEV)


def run_traj(tr, mode=0, frame_w=None):
    v, f, d, y = to_dev(tr)
    w = None if frame_w is None else torch.tensor(frame_w, dtype=torch.float32, device=DEV)
    r = L().dc_loss_traj(v, f, d, y, mode=mode, frame_w=w, check=True, face_mask=dev_mask(tr))
    torch.cuda.synchronize()
    return {k: (x.cpu().numpy() if isinstance(x, torch.Tensor) else x) for k, x in r.items()}


def compare_traj(tr, g, ref, frames, mode=0, weights=None):
    """Per-frame loss / neighbours / gradient of the frames the oracle ran."""
    for t in frames:
        per = ref["frames"][t]
        parity.check_nn(g["nn_ab"][t], per["nn_ab"],
                        g["nn_ba"][t] if mode == 0 else None, per["nn_ba"] if mode == 0 else None)
    parity.check_loss(g["loss_frames"][frames], ref["loss_frames"][frames])
    parity.check_grad(g["grad_verts"][frames], ref["grad_verts"][frames])
    if len(frames) == tr.T:
        w = np.ones(tr.T) if weights is None else np.asarray(weights)
        parity.check_loss(g["loss_total"], [np.sum(w * ref["loss_frames"])], what="total")


# ---------------------------------------------------------------------------------------------
# the five workloads' sizes
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_single_frame_25x25(mode):
    tr = parity.nudged(W.single_frame())
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, [0], mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_trajectory_50x50_full_size_every_frame(mode):
    """The 40-frame 50x50 trajectory at full size (10 000 x 10 000 per frame), in the launch
    configuration the bench times; every frame against the oracle, and the total."""
    tr = parity.nudged(W.trajectory_50x50())
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, list(range(tr.T)), mode)
    assert np.all(np.isfinite(g["loss_frames"])) and np.all(g["loss_frames"] > 0)


def test_trajectory_50x50_weights_total():
    tr = parity.nudged(W.trajectory_50x50(T=4, n=3000, m=2500))
    w = [0.25, 0.5, 1.0, 2.0]
    g = run_traj(tr, frame_w=w)
    ref = oracle.loss_traj(tr, weights=w)
    compare_traj(tr, g, ref, list(range(tr.T)), weights=w)


@pytest.mark.parametrize("mode", [0, 1])
def test_many_small_frames_one_epilogue_slice_each(mode):
    """700 frames: one epilogue CTA per frame writes the gradient directly (no slice
    reduction); every frame against the oracle."""
    tr = parity.nudged(W.lift_trajectory(41, 8, 700, 96, 80, name="many"))
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, list(range(tr.T)), mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_large_mesh_global_memory_paths(mode):
    """A 175 x 175 grid (30 625 vertices, 60 552 faces): the V x 3 gradient accumulator does
    not fit in shared memory (the scatter goes to global memory) and neither does the area
    CDF (sampling and target staging search it in global memory)."""
    tr = parity.nudged(W.lift_trajectory(43, 175, 2, 3000, 2500, name="big_mesh"))
    assert tr.V * 12 > 227 * 1024 and tr.F * 4 > 227 * 1024
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, list(range(tr.T)), mode)


# ---------------------------------------------------------------------------------------------
# exact ties: the lowest index wins (R6), across sub-chunks, chunks, units and CTAs
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_exact_ties_go_to_the_lowest_index(mode):
    rng = np.random.default_rng(31)
    U = rng.random((500, 3)).astype(np.float32)
    b = np.ascontiguousarray(U[np.arange(5000) % 500])      # copies 500 indices apart
    a = np.ascontiguousarray(U[(np.arange(4000) * 7) % 500] + np.float32(1e-3) *
                             rng.standard_normal((4000, 3)).astype(np.float32))
    a[::5] = U[(np.arange(0, 4000, 5) * 3) % 500]           # some sim points on targets
    a = np.ascontiguousarray(np.concatenate([a, a[:1000]]))  # and repeated sim points
    A = torch.from_numpy(a[None]).to(DEV)
    B = torch.from_numpy(b[None]).to(DEV)
    loss, nab, nba = L().dc_chamfer_fwd(A, B, mode=mode, check=True)
    ref = oracle.nn_pair(a, b)
    np.testing.assert_array_equal(nab[0].cpu().numpy(), ref["nn_ab"])
    assert np.all(nab[0].cpu().numpy() < 500)                # the first copy of each point
    if mode == 0:
        np.testing.assert_array_equal(nba[0].cpu().numpy(), ref["nn_ba"])
    # every target the same point: every sim point's neighbour is target 0, and every
    # target's neighbour is the first sim point at the least distance
    b1 = np.ascontiguousarray(np.repeat(U[:1], 3000, axis=0))
    loss, nab, nba = L().dc_chamfer_fwd(A, torch.from_numpy(b1[None]).to(DEV), mode=mode,
                                        check=True)
    assert np.all(nab[0].cpu().numpy() == 0)
    if mode == 0:
        np.testing.assert_array_equal(nba[0].cpu().numpy(), oracle.nn_pair(a, b1)["nn_ba"])


# ---------------------------------------------------------------------------------------------
# failure detection without a GPU fault
# ---------------------------------------------------------------------------------------------
@pytest.mark.timeout(120)
@pytest.mark.parametrize("shape", [("tensor", 0), ("tcgen05", 0), ("direct", 2)])
def test_bounded_wait_gives_up_with_a_timeout_status_and_the_device_stays_usable(shape):
    """The Chamfer kernels' waits for their target chunks (and, on the tcgen05 engine, for
    the MMAs and the reading warps) are bounded (2 s). A launch whose first chunk is never
    requested must end with DC_ETIMEOUT in the workspace status, and the next call on the same
    context must produce the normal result; for each of the three engines."""
    from paper_2204_03139_gb300 import autotune

    tr = parity.nudged(W.trajectory_50x50(T=2, n=2000, m=2000))
    v, f, d, y = to_dev(tr)
    with autotune.tuned(shape):
        good = L().dc_loss_traj(v, f, d, y, check=True)
        ref_loss = good["loss_frames"].cpu().numpy().copy()
        L().test_inject_stall()
        with pytest.raises(L().DCError) as e:
            L().dc_loss_traj(v, f, d, y, check=True)
        assert e.value.code == L().DC_ETIMEOUT
        again = L().dc_loss_traj(v, f, d, y, check=True)
    np.testing.assert_array_equal(again["loss_frames"].cpu().numpy(), ref_loss)


# ---------------------------------------------------------------------------------------------
# a1: the area CDF against the oracle
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["50x50", "100x100", "masked", "warped"])
def test_area_cdf_within_bound_of_the_oracle(case):
    """max |C_gpu - C_oracle| / A <= 2.5e-7, so that the 1e-6 face-pick window covers every
    float32 disagreement; the GPU's C_f is the float32 rounding of the exact prefix sum of its
    float32 areas, so it stays this close however many faces there are."""
    if case == "100x100":
        tr = W.trajectory_100x100(T=2)
    else:
        tr = W.trajectory_50x50(T=3, n=1000, m=1000)
    mask = W.upper_half_mask(50) if case == "masked" else None
    verts = tr.verts.copy()
    if case == "warped":  # very unequal face areas
        verts[..., 0] = verts[..., 0] ** 3
    v = torch.from_numpy(verts).to(DEV)
    f = torch.from_numpy(tr.faces).to(DEV)
    m = None if mask is None else torch.from_numpy(mask).to(DEV)
    c = L().dc_area_cdf(v, f, face_mask=m, check=True).cpu().numpy().astype(np.float64)
    for t in range(tr.T):
        ref = oracle.area_cdf(oracle.face_areas(verts[t], tr.faces, mask))
        A = ref[-1]
        assert np.max(np.abs(c[t] - ref)) / A <= 2.5e-7
        if mask is not None:
            assert np.all(np.diff(np.concatenate([[0.0], c[t]]))[mask == 0] == 0.0)


# ---------------------------------------------------------------------------------------------
# sampling from a face subset (Sec. IV-F fold scenario)
# ---------------------------------------------------------------------------------------------
def masked(tr, mask):
    import copy

    out = copy.copy(tr)
    out.face_mask = np.ascontiguousarray(mask, np.uint8)
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_face_subset_matches_oracle(mode):
    """The fold scenario's sampling (only the upper half of the cloth): face picks, points,
    neighbours, loss and gradient against the oracle with the same mask; no sample lands on a
    masked face and vertices touched only by masked faces get no gradient."""
    mask = W.upper_half_mask(50)
    tr = parity.nudged(masked(W.trajectory_50x50(T=3, n=4000, m=3000), mask))
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, list(range(tr.T)), mode)
    v, f, d, _ = to_dev(tr)
    pts, fi, _ = L().dc_sample(v, f, d, check=True, face_mask=dev_mask(tr))
    fi = fi.cpu().numpy()
    assert np.all(mask[fi] == 1)
    for t in range(tr.T):
        r = oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t)[:1],
                         mode=1, grads=False, face_mask=mask)
        parity.check_face_picks(fi[t], r["face_idx"], r["margin"])
    kept = np.zeros(tr.V, bool)
    kept[tr.faces[mask == 1].ravel()] = True
    assert np.all(g["grad_verts"][:, ~kept] == 0.0)
    # the backward-only call with the same mask reproduces the gradient
    r = L().dc_loss_traj(v, f, d, to_dev(tr)[3], mode=mode, check=True,
                         face_mask=dev_mask(tr))
    gb = L().dc_loss_traj_bwd(v, f, d, to_dev(tr)[3], r["nn_ab"], r["nn_ba"],
                              torch.ones(tr.T, device=DEV), mode=mode, check=True,
                              face_mask=dev_mask(tr))
    assert parity.rel_l2(gb.cpu().numpy(), g["grad_verts"]) < 1e-6


def test_full_mask_changes_nothing_and_empty_subset_is_degenerate():
    tr = parity.nudged(W.trajectory_50x50(T=2, n=2000, m=2000))
    a = run_traj(tr)
    b = run_traj(masked(tr, np.ones(tr.F, np.uint8)))
    np.testing.assert_array_equal(a["nn_ab"], b["nn_ab"])
    np.testing.assert_array_equal(a["loss_frames"], b["loss_frames"])
    v, f, d, y = to_dev(tr)
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v, f, d, y, check=True,
                         face_mask=torch.zeros(tr.F, dtype=torch.uint8, device=DEV))
    assert e.value.code == L().DC_EDEGENERATE


@pytest.mark.parametrize("w", [[0.0, 0.0, 0.0, 1.0], [0.0, 1.5, 0.0, 0.5], [1.0, 0.0, 2.0, 0.0]])
def test_zero_weight_frames_are_skipped(w):
    """Frames of weight 0 (e.g. last-frame-only, as the paper mostly optimises) do no work:
    their L_t is reported as 0 and their gradient is 0; the other frames are unchanged."""
    tr = parity.nudged(W.trajectory_50x50(T=4, n=3000, m=2500))
    g = run_traj(tr, frame_w=w)
    live = [t for t in range(4) if w[t] != 0.0]
    dead = [t for t in range(4) if w[t] == 0.0]
    ref = oracle.loss_traj(tr, weights=w, frames=live)
    for t in live:
        parity.check_nn(g["nn_ab"][t], ref["frames"][t]["nn_ab"], g["nn_ba"][t],
                        ref["frames"][t]["nn_ba"])
    parity.check_loss(g["loss_frames"][live], ref["loss_frames"][live])
    parity.check_grad(g["grad_verts"][live], ref["grad_verts"][live])
    parity.check_loss(g["loss_total"], [np.nansum(np.asarray(w) * ref["loss_frames"])],
                      what="total")
    assert np.all(g["loss_frames"][dead] == 0.0)
    assert np.all(g["grad_verts"][dead] == 0.0)
    # the backward-only call skips frames whose upstream gradient is 0 the same way
    v, f, d, y = to_dev(tr)
    r = L().dc_loss_traj(v, f, d, y, check=True)
    gb = L().dc_loss_traj_bwd(v, f, d, y, r["nn_ab"], r["nn_ba"],
                              torch.tensor(w, dtype=torch.float32, device=DEV), check=True)
    torch.cuda.synchronize()
    gb = gb.cpu().numpy()
    assert np.all(gb[dead] == 0.0)
    assert parity.rel_l2(gb[live], g["grad_verts"][live]) < 1e-6


@pytest.fixture(scope="module")
def traj100():
    """The 100-frame 100x100 trajectory (32 768 x 32 768 per frame) and its oracle result."""
    tr = parity.nudged(W.trajectory_100x100())
    return tr, oracle.loss_traj(tr)


@pytest.mark.slow
def test_trajectory_100x100_full_size_every_frame(traj100):
    """100x100 grid, T = 100, 32 768 x 32 768 per frame: every frame against the oracle."""
    tr, ref = traj100
    g = run_traj(tr)
    compare_traj(tr, g, ref, list(range(tr.T)))


@pytest.mark.slow
def test_trajectory_100x100_autograd_recompute_matches_oracle_and_fd(traj100):
    """The differentiation configuration at full size: the loss through the autograd Function
    (forward without the gradient, backward recomputing the samples from the stored draws),
    its full 100-frame vertex gradient against the oracle, and 200 random vertex coordinates
    of one frame against FP64 central differences of the oracle at h = 1e-6 m (coordinates
    whose +-h runs change a face pick or a neighbour are skipped)."""
    from paper_2204_03139_gb300.autograd import loss_traj

    tr, ref = traj100
    v, f, d, y = to_dev(tr)
    vv = v.clone().requires_grad_(True)
    total, lf = loss_traj(vv, f, d, y)
    total.backward()
    torch.cuda.synchronize()
    parity.check_loss(lf.detach().cpu().numpy(), ref["loss_frames"])
    parity.check_loss([float(total.detach())], [ref["loss_total"]], what="total")
    gpu_g = vv.grad.cpu().numpy()
    parity.check_grad(gpu_g, ref["grad_verts"])
    fd_check(tr, gpu_g, ref, t=37, n=200, seed=17)


def fd_check(tr, gpu_g, ref, t, n, seed):
    """FP64 central differences of the oracle loss of frame t at h = 1e-6 m on n random
    vertex coordinates against the GPU gradient; coordinates whose +-h runs change a pick or
    a neighbour are skipped (at least three quarters must count)."""
    rng = W.rng_for(seed)
    base = oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t),
                        grads=False)
    scale = np.abs(ref["grad_verts"][t]).max()
    checked = 0
    for _ in range(n):
        vi, k = int(rng.integers(tr.V)), int(rng.integers(3))
        vp, vm = tr.verts[t].copy(), tr.verts[t].copy()
        vp[vi, k] = np.float32(vp[vi, k] + 1e-6)
        vm[vi, k] = np.float32(vm[vi, k] - 1e-6)
        rp = oracle.frame(vp, tr.faces, tr.frame_draws(t), tr.frame_targets(t), grads=False)
        rm = oracle.frame(vm, tr.faces, tr.frame_draws(t), tr.frame_targets(t), grads=False)
        if not all(np.array_equal(rp[q], rm[q]) and np.array_equal(rp[q], base[q])
                   for q in ("face_idx", "nn_ab", "nn_ba")):
            continue
        a_ = float(vp[vi, k]) - float(tr.verts[t][vi, k])
        b_ = float(tr.verts[t][vi, k]) - float(vm[vi, k])
        fd = (b_ * b_ * (rp["loss"] - base["loss"]) + a_ * a_ * (base["loss"] - rm["loss"])) / (
            a_ * b_ * (a_ + b_))
        # the GPU gradient of this coordinate agrees with the FP64 difference quotient
        assert abs(gpu_g[t, vi, k] - fd) <= 1e-4 * scale + 1e-6 * abs(fd), (vi, k, fd)
        checked += 1
    assert checked >= 0.75 * n


# ---------------------------------------------------------------------------------------------
# ragged sizes: tails of every tile level (16-row thread groups, 512-row warps, units of
# 512 / 1024 / 2048 rows, 32-target sub-chunks, 256-target chunks)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(1, 1), (1, 300), (300, 1), (2, 3), (31, 33), (63, 65),
                                 (255, 257), (511, 513), (1023, 1025), (1025, 511),
                                 (2049, 4097), (3000, 64)])
@pytest.mark.parametrize("mode", [0, 1])
def test_ragged_sizes(n, m, mode):
    tr = W.lift_trajectory(7 + n + 3 * m, 9, 2, n, m, name="ragged")
    tr = parity.nudged(tr)
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, [0, 1], mode)


@pytest.mark.parametrize("n", [768, 769, 896, 897, 1280, 1665])
@pytest.mark.parametrize("mode", [0, 1])
def test_tail_warp_tiles(n, mode):
    """A frame's last warp of 512 rows takes 8 rows per lane when 256 or fewer rows are left,
    12 when 384 or fewer, else the full 16: frames whose last warp sits on each side of both
    boundaries (256 / 257, 384 / 385 rows left), and a short warp in a later unit."""
    tr = W.lift_trajectory(11 + n, 9, 2, n, 900, name="tail")
    tr = parity.nudged(tr)
    g = run_traj(tr, mode)
    ref = oracle.loss_traj(tr, mode=mode)
    compare_traj(tr, g, ref, [0, 1], mode)


def test_raw_draws_face_picks_and_neighbours():
    """Without moving any draw: face picks exact outside the 1e-6 window, neighbours exact
    except for points whose face pick fell inside it."""
    tr = W.trajectory_50x50(T=3, n=10000, m=10000)
    v, f, d, y = to_dev(tr)
    pts, fi, bc = L().dc_sample(v, f, d, check=True)
    r = L().dc_loss_traj(v, f, d, y, check=True)
    torch.cuda.synchronize()
    for t in range(tr.T):
        per = oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t))
        diff = parity.check_face_picks(fi[t].cpu().numpy(), per["face_idx"], per["margin"])
        same = np.setdiff1d(np.arange(tr.n(t)), diff)
        np.testing.assert_array_equal(pts[t].cpu().numpy()[same], per["x32"][same])
        parity.check_nn(r["nn_ab"][t].cpu().numpy(), per["nn_ab"],
                        r["nn_ba"][t].cpu().numpy(), per["nn_ba"], moved_rows=diff)


# ---------------------------------------------------------------------------------------------
# the individual entry points
# ---------------------------------------------------------------------------------------------
def test_dc_sample_matches_oracle():
    tr = parity.nudged(W.trajectory_50x50(T=2, n=5000, m=1))
    v, f, d, _ = to_dev(tr)
    pts, fi, bc = L().dc_sample(v, f, d, check=True)
    torch.cuda.synchronize()
    for t in range(2):
        per = oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t))
        np.testing.assert_array_equal(fi[t].cpu().numpy(), per["face_idx"])
        np.testing.assert_array_equal(pts[t].cpu().numpy(), per["x32"])
        np.testing.assert_allclose(bc[t].cpu().numpy(), per["bary"], rtol=0, atol=3e-7)
        np.testing.assert_allclose(pts[t].cpu().numpy(), per["x64"], rtol=0, atol=5e-7)


def test_equal_area_grid_picks_are_floor():
    """On the exactly-equal-area flat 17x17 grid the pick is floor(r_f F) for every draw,
    including draws exactly on a boundary."""
    tr = W.flat_square(17, 20000, seed=5)
    d = tr.draws.copy()
    d[:512, 0] = (np.arange(512) / 512).astype(np.float32)
    _, fi, _ = L().dc_sample(torch.from_numpy(tr.verts).to(DEV), torch.from_numpy(tr.faces).to(DEV),
                             torch.from_numpy(d[None]).to(DEV), check=True)
    np.testing.assert_array_equal(fi[0].cpu().numpy(), np.floor(d[:, 0].astype(np.float64) * 512))


@pytest.mark.parametrize("n,m,mode", [(700, 900, 0), (2048, 333, 1), (5000, 5000, 0)])
def test_chamfer_fwd_bwd_points(n, m, mode):
    a, b = W.random_cloud_pair(n + m, n, m)
    nn = oracle.nn_pair(a, b)
    loss, ga = oracle.chamfer(a, b, mode=mode, gscale=1.5)
    ta, tb = torch.from_numpy(a[None]).to(DEV), torch.from_numpy(b[None]).to(DEV)
    l, nab, nba = L().dc_chamfer_fwd(ta, tb, mode=mode, check=True)
    g = L().dc_chamfer_bwd(ta, tb, nab, nba, torch.tensor([1.5], device=DEV), mode=mode)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(nab[0].cpu().numpy(), nn["nn_ab"])
    if mode == 0:
        np.testing.assert_array_equal(nba[0].cpu().numpy(), nn["nn_ba"])
    parity.check_loss(l.cpu().numpy(), [loss])
    parity.check_grad(g[0].cpu().numpy(), ga)


def test_chamfer_self_zero_and_shift():
    u, v = W.grid_uv(60)
    a = np.stack([u, v, np.zeros_like(u)], 1).astype(np.float32)
    b = a.copy()
    b[:, 2] += np.float32(0.004)
    ta, tb = torch.from_numpy(a[None]).to(DEV), torch.from_numpy(b[None]).to(DEV)
    l0, n0, m0 = L().dc_chamfer_fwd(ta, ta, check=True)
    l1, n1, m1 = L().dc_chamfer_fwd(ta, tb, check=True)
    torch.cuda.synchronize()
    assert float(l0[0]) == 0.0
    np.testing.assert_array_equal(n0[0].cpu().numpy(), np.arange(a.shape[0]))
    np.testing.assert_array_equal(m1[0].cpu().numpy(), np.arange(a.shape[0]))
    assert float(l1[0]) == pytest.approx(2 * float(np.float32(0.004)) ** 2, rel=1e-6)


def test_loss_traj_bwd_recompute_equals_fused():
    tr = parity.nudged(W.trajectory_50x50(T=3, n=4000, m=3500))
    v, f, d, y = to_dev(tr)
    r = L().dc_loss_traj(v, f, d, y, check=True)
    gf = torch.ones(3, device=DEV)
    g2 = L().dc_loss_traj_bwd(v, f, d, y, r["nn_ab"], r["nn_ba"], gf, check=True)
    torch.cuda.synchronize()
    assert parity.rel_l2(g2.cpu().numpy(), r["grad_verts"].cpu().numpy()) < 1e-6


def test_autograd_matches_oracle_and_fd():
    """DCLoss backward (samples recomputed from the draws) against the oracle gradient, and
    the oracle's own FP64 central differences on 200 random vertex coordinates."""
    from paper_2204_03139_gb300.autograd import loss_traj

    tr = parity.nudged(W.lift_trajectory(99, 100, 2, 2048, 2048, name="fd"))
    v, f, d, y = to_dev(tr)
    vv = v.clone().requires_grad_(True)
    total, lf = loss_traj(vv, f, d, y)
    total.backward()
    torch.cuda.synchronize()
    ref = oracle.loss_traj(tr)
    parity.check_loss(lf.detach().cpu().numpy(), ref["loss_frames"])
    gpu_g = vv.grad.cpu().numpy()
    parity.check_grad(gpu_g, ref["grad_verts"])
    fd_check(tr, gpu_g, ref, t=1, n=200, seed=7)


@pytest.mark.parametrize("mode", [0, 1])
def test_autograd_total_and_frame_gradients_combine(mode):
    """An objective of both outputs, J = 2 L_total + sum_t c_t L_t with a frame of weight 0:
    the library forms g_t = 2 w_t + c_t (0 for the weight-0 frame, whose L_t is the constant
    0), and the vertex gradient equals the oracle's with those multipliers."""
    from paper_2204_03139_gb300.autograd import loss_traj

    tr = parity.nudged(W.trajectory_50x50(T=4, n=3000, m=2500))
    v, f, d, y = to_dev(tr)
    w = np.array([1.0, 0.0, 0.5, 2.0])
    c = np.array([0.25, 3.0, -1.0, 0.5])
    vv = v.clone().requires_grad_(True)
    total, lf = loss_traj(vv, f, d, y, mode=mode, frame_w=w)
    J = 2.0 * total + (torch.tensor(c, dtype=torch.float32, device=DEV) * lf).sum()
    J.backward()
    torch.cuda.synchronize()
    gs = np.where(w != 0.0, 2.0 * w + c, 0.0)
    ref = oracle.loss_traj(tr, mode=mode, weights=w, gscale=gs)
    live = [t for t in range(4) if w[t] != 0.0]
    parity.check_loss(lf.detach().cpu().numpy()[live], ref["loss_frames"][live])
    assert float(lf[1]) == 0.0
    g = vv.grad.cpu().numpy()
    parity.check_grad(g[live], ref["grad_verts"][live])
    assert np.all(g[1] == 0.0)


# ---------------------------------------------------------------------------------------------
# device-side errors, determinism
# ---------------------------------------------------------------------------------------------
def test_device_errors_are_reported():
    v = torch.zeros((1, 3, 3), device=DEV)
    f = torch.tensor([[0, 1, 2]], dtype=torch.int32, device=DEV)
    d = torch.full((1, 4, 3), 0.5, device=DEV)
    y = torch.zeros((1, 4, 3), device=DEV)
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v, f, d, y, check=True)
    assert e.value.code == L().DC_EDEGENERATE
    v2 = torch.tensor([[[0, 0, 0], [1, 0, 0], [0, 1, 0]]], dtype=torch.float32, device=DEV)
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v2, torch.tensor([[0, 1, 3]], dtype=torch.int32, device=DEV), d, y,
                         check=True)
    assert e.value.code == L().DC_EINVAL
    y2 = y.clone()
    y2[0, 1, 1] = float("nan")
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v2, f, d, y2, check=True)
    assert e.value.code == L().DC_EINVAL
    # the next good call clears the status
    r = L().dc_loss_traj(v2, f, d, y, check=True)
    assert torch.isfinite(r["loss_frames"]).all()


def test_area_errors_of_any_frame_reach_the_status():
    """The area step of a uniform call runs in the launch that also builds the frame tables,
    and keeps its errors per frame until the sampling launch reports them: a degenerate last
    frame is reported by the forward call, the recomputing backward call and dc_sample; a bad
    face index is reported when the CDF is too large for shared memory, where the sampling
    runs from global memory."""
    T, n = 3, 64
    v = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=torch.float32,
                     device=DEV).repeat(T, 1, 1)
    v[T - 1] = 0.25  # every vertex of the last frame at one point: zero total area
    f = torch.tensor([[0, 1, 2]], dtype=torch.int32, device=DEV)
    d = torch.full((T, n, 3), 0.5, device=DEV)
    y = torch.zeros((T, n, 3), device=DEV)
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v, f, d, y, check=True)
    assert e.value.code == L().DC_EDEGENERATE
    nn_ab = torch.zeros((T, n), dtype=torch.int32, device=DEV)
    nn_ba = torch.zeros((T, n), dtype=torch.int32, device=DEV)
    g = torch.ones(T, device=DEV)
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj_bwd(v, f, d, y, nn_ab, nn_ba, g, check=True)
    assert e.value.code == L().DC_EDEGENERATE
    with pytest.raises(L().DCError) as e:
        L().dc_sample(v, f, d, check=True)
    assert e.value.code == L().DC_EDEGENERATE
    # the same frames with a nonzero area pass
    v[T - 1] = v[0]
    r = L().dc_loss_traj(v, f, d, y, check=True)
    assert torch.isfinite(r["loss_frames"]).all()
    # 70 000 copies of one triangle (a CDF of 280 KB, beyond shared memory), the last one
    # with a vertex index out of range
    F = 70000
    fb = torch.tensor([[0, 1, 2]], dtype=torch.int32, device=DEV).repeat(F, 1)
    fb[F - 1, 2] = 3
    with pytest.raises(L().DCError) as e:
        L().dc_loss_traj(v[:1], fb, d[:1], y[:1], check=True)
    assert e.value.code == L().DC_EINVAL
    fb[F - 1, 2] = 2
    r = L().dc_loss_traj(v[:1], fb, d[:1], y[:1], check=True)
    assert torch.isfinite(r["loss_frames"]).all()


@pytest.mark.parametrize("shape", [(2, 2048, 2048), (3, 5000, 7000)])
def test_every_cta_width_gives_identical_results(shape):
    """The three Chamfer tile shapes (1, 2, 4 warps per CTA) split the same pairs differently;
    minima, neighbours and losses must not change by a single bit."""
    from paper_2204_03139_gb300 import autotune

    T, n, m = shape
    tr = W.trajectory_50x50(T=T, n=n, m=m)
    v, f, d, y = to_dev(tr)
    outs = {}
    for wd in (1, 2, 4):
        with autotune.tuned(wd):
            r = L().dc_loss_traj(v, f, d, y, check=True)
        torch.cuda.synchronize()
        outs[wd] = {k: x.cpu().numpy() for k, x in r.items() if x is not None}
    for wd in (1, 2):
        for k in ("loss_frames", "loss_total", "nn_ab", "nn_ba"):
            np.testing.assert_array_equal(outs[wd][k], outs[4][k])
        assert parity.rel_l2(outs[wd]["grad_verts"], outs[4]["grad_verts"]) < 1e-6
    res = autotune.tune(v, f, d, y, reps=1, save=False)
    assert res["best"] in autotune.SHAPES and all(t > 0 for t in res["ms"].values())


@pytest.mark.parametrize("case", ["traj", "ragged", "ties", "grid", "outliers", "eq2"])
def test_engines_give_identical_results(case):
    """The tensor-core filter (on warp-level MMAs and on tcgen05 MMAs) and the direct engine
    decide every neighbour in the same float32 direct form, so neighbours, per-frame losses
    and totals agree bit for bit; the cases cover uniform trajectories, ragged tails of every
    tile, exact ties in many blocks (every row falls back to a full scan), a regular grid
    (equidistant neighbours), far outliers and Eq. 2."""
    from paper_2204_03139_gb300 import autotune

    mode = 1 if case == "eq2" else 0
    if case == "traj" or case == "eq2":
        tr = W.trajectory_50x50(T=3, n=5000, m=7000)
    elif case == "ragged":
        tr = W.lift_trajectory(3, 20, 2, 1537, 2049 + 255, name="rag")
    elif case == "outliers":
        tr = W.lift_trajectory(4, 30, 2, 3000, 3000, outliers=0.3, name="out")
    else:
        tr = None
    if tr is not None:
        v, f, d, y = to_dev(tr)
        outs = {}
        for sh in (("tensor", 0), ("tcgen05", 0), ("direct", 2)):
            with autotune.tuned(sh):
                r = L().dc_loss_traj(v, f, d, y, mode=mode, check=True)
            torch.cuda.synchronize()
            outs[sh[0]] = {k: x.cpu().numpy() for k, x in r.items() if x is not None}
        for eng in ("tensor", "tcgen05"):
            for k in ("loss_frames", "loss_total", "nn_ab") + (("nn_ba",) if mode == 0 else ()):
                np.testing.assert_array_equal(outs[eng][k], outs["direct"][k])
            assert parity.rel_l2(outs[eng]["grad_verts"], outs["direct"]["grad_verts"]) < 1e-6
        return
    if case == "ties":
        rng = np.random.default_rng(3)
        U = rng.random((400, 3)).astype(np.float32)
        a = np.ascontiguousarray(U[(np.arange(3000) * 7) % 400] + np.float32(1e-3) *
                                 rng.standard_normal((3000, 3)).astype(np.float32))
        b = np.ascontiguousarray(U[np.arange(4000) % 400])  # ten copies of every point
    else:
        u, vv = W.grid_uv(70)
        a = np.stack([u, vv, np.zeros_like(u)], 1).astype(np.float32)
        b = np.ascontiguousarray(a[::-1] + np.float32(0.25) / 69)  # shifted by a quarter step
    A = torch.from_numpy(a[None]).to(DEV)
    B = torch.from_numpy(b[None]).to(DEV)
    ref = oracle.nn_pair(a, b)
    for sh in (("tensor", 0), ("tcgen05", 0), ("direct", 1)):
        with autotune.tuned(sh):
            loss, nab, nba = L().dc_chamfer_fwd(A, B, check=True)
        np.testing.assert_array_equal(nab[0].cpu().numpy(), ref["nn_ab"])
        np.testing.assert_array_equal(nba[0].cpu().numpy(), ref["nn_ba"])


def test_loss_is_deterministic():
    tr = W.trajectory_50x50(T=4, n=6000, m=7000)
    a = run_traj(tr)
    b = run_traj(tr)
    np.testing.assert_array_equal(a["loss_frames"], b["loss_frames"])
    np.testing.assert_array_equal(a["loss_total"], b["loss_total"])
    np.testing.assert_array_equal(a["nn_ab"], b["nn_ab"])
    np.testing.assert_array_equal(a["nn_ba"], b["nn_ba"])
    assert parity.rel_l2(a["grad_verts"], b["grad_verts"]) < 1e-6
