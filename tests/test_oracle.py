"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test below would fail under a plausible mistake in the oracle: a dropped sqrt in the
Eq. 3 reparameterisation, a face pick by count instead of by area, a non-strict CDF
comparison, swapped barycentric weights, a wrong sign or scale in Eq. 1 / Eq. 2, a missing
target-side term in the gradient, or a wrong scatter in Eq. 4.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "two_triangles.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------------------------
# hand-derived worked example (Sec. III-B, Eq. 1-4)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [oracle.BIDIR_MEAN, oracle.UNIDIR_SUM])
def test_golden_two_triangles(mode):
    g = _golden()
    e = g["expected"]
    v = np.array(g["verts"], np.float32)
    f = np.array(g["faces"], np.int32)
    d = np.array(g["draws"], np.float32)
    y = np.array(g["targets"], np.float32)
    np.testing.assert_array_equal(oracle.face_areas(v, f), e["areas"])
    np.testing.assert_array_equal(oracle.area_cdf(oracle.face_areas(v, f)), e["cdf"])
    r = oracle.frame(v, f, d, y, mode=mode)
    np.testing.assert_array_equal(r["face_idx"], e["face_idx"])
    np.testing.assert_array_equal(r["bary"], e["bary"])
    np.testing.assert_array_equal(r["x64"], e["points"])
    np.testing.assert_array_equal(r["x32"], np.array(e["points"], np.float32))
    np.testing.assert_array_equal(r["nn_ab"], e["nn_ab"])
    if mode == oracle.BIDIR_MEAN:
        np.testing.assert_array_equal(r["nn_ba"], e["nn_ba"])
        assert r["loss"] == e["loss_eq1"]
        np.testing.assert_allclose(r["grad_verts"], e["grad_verts_eq1"], rtol=1e-15, atol=1e-15)
    else:
        assert r["loss"] == e["loss_eq2"]
        np.testing.assert_allclose(r["grad_verts"], e["grad_verts_eq2"], rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------------------------------------
# a1/a2: area-weighted face pick (Sec. III-B)
# ---------------------------------------------------------------------------------------------
def test_equal_area_pick_is_floor():
    """A flat 17x17 grid has 512 faces of exactly equal area (spacing 1/16 is exact in
    float32), so the strict inverse-CDF pick is floor(r_f * F) for every draw, including
    draws exactly on a boundary k/F (which go to face k)."""
    tr = W.flat_square(17, 20000, seed=11)
    F = tr.F
    assert F == 512
    d = tr.draws.copy()
    d[:F, 0] = (np.arange(F) / F).astype(np.float32)  # exact boundaries
    r = oracle.frame(tr.verts[0], tr.faces, d, tr.targets[:1], mode=oracle.UNIDIR_SUM)
    expect = np.floor(d[:, 0].astype(np.float64) * F).astype(np.int64)
    np.testing.assert_array_equal(r["face_idx"], expect)


def test_pick_margin_closed_form_equal_area_grid():
    """The margin returned with each pick is the distance of r_f to the nearer interior CDF
    boundary, in units of A. On the exactly-equal-area 17x17 grid the interior boundaries are
    k/F for k = 1 .. F-1, so r = k/F + e has margin |e| (for |e| < 1/(2F)), a draw exactly on
    a boundary has margin 0, and the first and last faces have only one boundary each. The
    parity tests rely on it to decide which draws are ill-posed."""
    tr = W.flat_square(17, 10, seed=11)
    F = tr.F
    cdf = oracle.area_cdf(oracle.face_areas(tr.verts[0], tr.faces))
    rng = np.random.default_rng(5)
    k = rng.integers(1, F, size=600)
    e = rng.uniform(0.0, 0.49 / F, size=600) * np.where(rng.random(600) < 0.5, -1.0, 1.0)
    r = np.concatenate([(k / F + e), np.arange(1, F) / F, [0.0, 0.3 / F, 1.0 - 0.3 / F]])
    r = r.astype(np.float32)
    for ri in r:
        f, m = oracle.pick_face(cdf, float(ri))
        rd = float(ri)
        j = min(max(int(np.rint(rd * F)), 1), F - 1)  # nearest interior boundary j/F
        assert f == int(np.floor(rd * F))
        assert m == abs(rd - j / F), (rd, f, m)
    # draws close to a boundary: the margin is the offset itself
    for kk in (1, 7, 255, 511):
        for off in (2.0 ** -20, 2.0 ** -16, 2.0 ** -12):
            _, m = oracle.pick_face(cdf, float(np.float32(kk / F + off)))
            assert m == off
            _, m = oracle.pick_face(cdf, float(np.float32(kk / F - off)))
            assert m == off


def test_pick_margin_two_triangles():
    """The worked example's CDF is (1, 1.5): one interior boundary at 2/3, so draw A (r = 1/2)
    has margin 1/6 and draw B (r = 3/4) margin 1/12."""
    g = _golden()
    v = np.array(g["verts"], np.float32)
    f = np.array(g["faces"], np.int32)
    cdf = oracle.area_cdf(oracle.face_areas(v, f))
    d = np.array(g["draws"], np.float32)
    r = oracle.frame(v, f, d, np.array(g["targets"], np.float32))
    np.testing.assert_allclose(r["margin"], [1 / 6, 1 / 12], rtol=1e-15)
    assert oracle.pick_face(cdf, 0.5)[1] == pytest.approx(1 / 6, rel=1e-15)


def test_nudge_moves_the_expected_number_of_draws():
    """parity.nudge_draws moves exactly the draws whose margin is below the window, to the
    middle of their face's interval, and their number matches 2 w (F - 1) per draw."""
    import parity

    tr = W.trajectory_50x50(T=3, n=20000, m=10)
    moved_tr, moved = parity.nudge_draws(tr, window=2e-6)
    parity.check_moves(tr, moved, window=2e-6)
    assert moved > 0
    for t in range(tr.T):
        _, mg = parity.frame_margins(moved_tr.verts[t], moved_tr.faces, moved_tr.frame_draws(t))
        assert np.all(mg >= 2e-6)
        changed = np.nonzero(moved_tr.frame_draws(t)[:, 0] != tr.frame_draws(t)[:, 0])[0]
        _, mg0 = parity.frame_margins(tr.verts[t], tr.faces, tr.frame_draws(t))
        np.testing.assert_array_equal(changed, np.nonzero(mg0 < 2e-6)[0])


def test_zero_area_faces_never_picked():
    tr = W.flat_square(9, 5000, seed=12)
    v = tr.verts[0].copy()
    faces = tr.faces.copy()
    # collapse every third face onto a segment (zero area) by repeating a vertex
    faces[::3, 2] = faces[::3, 1]
    r = oracle.frame(v, faces, tr.draws, tr.targets[:1], mode=oracle.UNIDIR_SUM)
    assert not np.any(r["face_idx"] % 3 == 0)


def test_degenerate_and_invalid():
    v = np.zeros((3, 3), np.float32)
    f = np.array([[0, 1, 2]], np.int32)
    d = np.full((4, 3), 0.5, np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.frame(v, f, d, v)
    assert e.value.code == oracle.EDEGENERATE
    with pytest.raises(oracle.OracleError) as e:
        oracle.frame(v, np.array([[0, 1, 3]], np.int32), d, v)
    assert e.value.code == oracle.EINVAL


def test_uniform_density_on_warped_flat_square():
    """Sec. III-B: area weighting makes the density uniform over the surface. The grid is
    warped (u -> u^2) so faces differ in area; picking by face count would crowd the
    samples toward the origin. Chi-square on a 10x10 histogram, mean 1/2 and variance 1/12
    per axis."""
    stats = pytest.importorskip("scipy.stats")
    tr = W.flat_square(12, 200_000, seed=13)
    v = tr.verts[0].copy()
    v[:, 0] = v[:, 0] ** 2
    v[:, 1] = v[:, 1] ** 2
    r = oracle.frame(v, tr.faces, tr.draws, tr.targets[:1], mode=oracle.UNIDIR_SUM)
    x = r["x64"]
    n = x.shape[0]
    h, _, _ = np.histogram2d(x[:, 0], x[:, 1], bins=10, range=[[0, 1], [0, 1]])
    chi2 = float(np.sum((h - n / 100) ** 2 / (n / 100)))
    assert stats.chi2.sf(chi2, 99) > 1e-3
    for k in range(2):
        assert abs(x[:, k].mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
        assert abs(x[:, k].var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)


def test_masked_equal_area_pick_is_floor_over_the_subset():
    """Sampling from a face subset (Sec. IV-F): on the flat 17x17 grid (512 faces of exactly
    equal area) with the upper-half mask (256 faces), the pick is the floor(r_f * K)-th face
    of the subset in face order, for every draw, including draws exactly on a boundary k/K."""
    tr = W.flat_square(17, 20000, seed=14)
    mask = W.upper_half_mask(17)
    sub = np.flatnonzero(mask)
    K = sub.size
    assert K == 256 and np.all(mask[:256] == 0)  # faces are stored row by row from v = 0
    d = tr.draws.copy()
    d[:K, 0] = (np.arange(K) / K).astype(np.float32)  # exact boundaries
    r = oracle.frame(tr.verts[0], tr.faces, d, tr.targets[:1], mode=oracle.UNIDIR_SUM,
                     face_mask=mask)
    expect = sub[np.floor(d[:, 0].astype(np.float64) * K).astype(np.int64)]
    np.testing.assert_array_equal(r["face_idx"], expect)
    # the mask only reweights: an all-ones mask changes nothing
    r1 = oracle.frame(tr.verts[0], tr.faces, d, tr.targets[:1], mode=oracle.UNIDIR_SUM,
                      face_mask=np.ones(tr.F, np.uint8))
    r0 = oracle.frame(tr.verts[0], tr.faces, d, tr.targets[:1], mode=oracle.UNIDIR_SUM)
    np.testing.assert_array_equal(r1["face_idx"], r0["face_idx"])


def test_masked_sampling_uniform_on_the_subset():
    """With the upper-half mask of a 13x13 grid (the line v = 1/2 is a grid line) on a warped
    flat square, every sample lies on a kept face and the density is uniform on the kept
    region [0,1] x [1/2,1] (a mask that only dropped faces from the face count would not
    keep the area weighting). Faces outside the subset are never picked."""
    stats = pytest.importorskip("scipy.stats")
    tr = W.flat_square(13, 200_000, seed=15)
    mask = W.upper_half_mask(13)
    v = tr.verts[0].copy()
    v[:, 0] = v[:, 0] ** 2  # unequal face areas along u (the kept region is unchanged)
    r = oracle.frame(v, tr.faces, tr.draws, tr.targets[:1], mode=oracle.UNIDIR_SUM,
                     face_mask=mask)
    assert np.all(mask[r["face_idx"]] == 1)
    x = r["x64"]
    n = x.shape[0]
    assert np.all(x[:, 1] >= 0.5 - 1e-12)
    h, _, _ = np.histogram2d(x[:, 0], x[:, 1], bins=(10, 5), range=[[0, 1], [0.5, 1]])
    chi2 = float(np.sum((h - n / 50) ** 2 / (n / 50)))
    assert stats.chi2.sf(chi2, 49) > 1e-3
    assert abs(x[:, 0].mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(x[:, 1].mean() - 0.75) < 5 * np.sqrt(1 / 48 / n)


def test_empty_face_subset_is_degenerate():
    tr = W.flat_square(9, 100, seed=16)
    with pytest.raises(oracle.OracleError) as e:
        oracle.frame(tr.verts[0], tr.faces, tr.draws, tr.targets[:1],
                     face_mask=np.zeros(tr.F, np.uint8))
    assert e.value.code == oracle.EDEGENERATE


# ---------------------------------------------------------------------------------------------
# a3: barycentric point (Eq. 3)
# ---------------------------------------------------------------------------------------------
def test_barycentric_moments_single_triangle():
    """A uniform point on a triangle has Dirichlet(1,1,1) barycentric coordinates:
    E[w_k] = 1/3, E[w_k^2] = 1/6, E[w_0 w_1] = 1/12; the weights sum to 1."""
    rng = W.rng_for(21)
    n = 1_000_000
    d = W.uniform_draws(rng, n)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    f = np.array([[0, 1, 2]], np.int32)
    r = oracle.frame(v, f, d, v[:1], mode=oracle.UNIDIR_SUM)
    w = r["bary"]
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    tol = 5 * np.sqrt(1 / 18 / n)
    for k in range(3):
        assert abs(w[:, k].mean() - 1 / 3) < tol
        assert abs((w[:, k] ** 2).mean() - 1 / 6) < tol
    assert abs((w[:, 0] * w[:, 1]).mean() - 1 / 12) < tol
    # the point equals the weighted vertex sum in the stated vertex order
    np.testing.assert_allclose(r["x64"], w @ v.astype(np.float64), rtol=0, atol=1e-15)


def test_point_float32_twin_close_to_double():
    tr = W.trajectory_50x50(T=2, n=3000, m=10)
    r = oracle.frame(tr.verts[1], tr.faces, tr.frame_draws(1), tr.frame_targets(1))
    err = np.abs(r["x32"].astype(np.float64) - r["x64"]).max()
    assert err < 4 * np.finfo(np.float32).eps


# ---------------------------------------------------------------------------------------------
# a4/a5: Chamfer (Eq. 1, Eq. 2)
# ---------------------------------------------------------------------------------------------
def test_chamfer_self_is_zero():
    a, _ = W.random_cloud_pair(31, 500, 1)
    loss, g = oracle.chamfer(a, a)
    assert loss == 0.0
    assert np.all(g == 0.0)
    nn = oracle.nn_pair(a, a)
    np.testing.assert_array_equal(nn["nn_ab"], np.arange(500))
    np.testing.assert_array_equal(nn["nn_ba"], np.arange(500))


def test_chamfer_normal_shift_closed_form():
    """A flat grid cloud against its copy shifted by delta along the normal: every nearest
    neighbour is the point's own copy, each direction contributes delta^2, Eq. 1 = 2 delta^2
    and Eq. 2 = N delta^2."""
    n = 40
    u, v = W.grid_uv(n)
    a = np.stack([u, v, np.zeros_like(u)], 1).astype(np.float32)
    delta = np.float32(0.003)  # below half the 1/39 spacing
    b = a.copy()
    b[:, 2] += delta
    dd = float(delta) ** 2
    loss1, g1 = oracle.chamfer(a, b, oracle.BIDIR_MEAN)
    loss2, _ = oracle.chamfer(a, b, oracle.UNIDIR_SUM)
    assert loss1 == pytest.approx(2 * dd, rel=1e-14)
    assert loss2 == pytest.approx(a.shape[0] * dd, rel=1e-14)
    nn = oracle.nn_pair(a, b)
    np.testing.assert_array_equal(nn["nn_ab"], np.arange(a.shape[0]))
    np.testing.assert_array_equal(nn["nn_ba"], np.arange(a.shape[0]))
    # gradient: every point is pulled toward +z; the total is 4 delta (Eq. 1)
    np.testing.assert_allclose(g1.sum(0), [0, 0, -4 * float(delta)], rtol=1e-12, atol=1e-15)


def test_chamfer_symmetric():
    a, b = W.random_cloud_pair(32, 300, 170)
    la, _ = oracle.chamfer(a, b)
    lb, _ = oracle.chamfer(b, a)
    assert la == pytest.approx(lb, rel=1e-14)


@pytest.mark.parametrize("n,m,seed", [(1, 1, 1), (7, 64, 2), (64, 5, 3), (64, 64, 4),
                                      (33, 17, 5)])
def test_chamfer_brute_force_numpy(n, m, seed):
    """Independent statement: full double distance matrix with numpy, minima per row and
    column, Eq. 1 as means and Eq. 2 as a sum."""
    a, b = W.random_cloud_pair(seed, n, m, scale=0.1)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    D = ((a64[:, None, :] - b64[None, :, :]) ** 2).sum(-1)
    eq1 = D.min(1).mean() + D.min(0).mean()
    eq2 = D.min(1).sum()
    assert oracle.chamfer(a, b, oracle.BIDIR_MEAN)[0] == pytest.approx(eq1, rel=1e-12)
    assert oracle.chamfer(a, b, oracle.UNIDIR_SUM)[0] == pytest.approx(eq2, rel=1e-12)
    nn = oracle.nn_pair(a, b)
    # where the double-precision minimum is well separated, the float32 decision agrees
    srt = np.sort(D, 1)
    sep = srt[:, 1] > srt[:, 0] * (1 + 1e-5) if m > 1 else np.ones(n, bool)
    np.testing.assert_array_equal(nn["nn_ab"][sep], D.argmin(1)[sep])
    srt0 = np.sort(D, 0)
    sep0 = srt0[1] > srt0[0] * (1 + 1e-5) if n > 1 else np.ones(m, bool)
    np.testing.assert_array_equal(nn["nn_ba"][sep0], D.argmin(0)[sep0])
    # the float32 distance is the double distance up to a few float32 roundings
    np.testing.assert_allclose(nn["d_ab"], D.min(1), rtol=1e-6, atol=1e-12)


def test_float32_decision_changes_loss_only_by_rounding():
    tr = W.trajectory_50x50(T=3, n=2000, m=2000)
    r = oracle.frame(tr.verts[2], tr.faces, tr.frame_draws(2), tr.frame_targets(2),
                     exact64=True)
    assert r["loss"] == pytest.approx(r["loss_exact"], rel=1e-6)
    assert r["loss"] >= r["loss_exact"] * (1 - 1e-12)


# ---------------------------------------------------------------------------------------------
# a6/a7: gradients (Eq. 4 and the Chamfer derivative)
# ---------------------------------------------------------------------------------------------
def _small_frame(seed=41, n_grid=6, n=64, m=48):
    tr = W.lift_trajectory(seed, n_grid, 3, n, m, name="fd")
    return tr.verts[2].copy(), tr.faces, tr.frame_draws(2), tr.frame_targets(2)


@pytest.mark.parametrize("mode", [oracle.BIDIR_MEAN, oracle.UNIDIR_SUM])
def test_gradient_central_fd(mode):
    """With face picks and neighbours fixed the loss is a quadratic in the vertices, so the
    three-point difference is exact up to rounding. Coordinates whose +-h evaluations change a
    pick or a neighbour are skipped (and counted)."""
    v, f, d, y = _small_frame()
    base = oracle.frame(v, f, d, y, mode=mode)
    rng = W.rng_for(42)
    checked = skipped = 0
    for _ in range(60):
        vi, k = int(rng.integers(v.shape[0])), int(rng.integers(3))
        h = 1e-3
        vp, vm = v.copy(), v.copy()
        vp[vi, k] = np.float32(v[vi, k] + h)
        vm[vi, k] = np.float32(v[vi, k] - h)
        a, b = float(vp[vi, k]) - float(v[vi, k]), float(v[vi, k]) - float(vm[vi, k])
        rp = oracle.frame(vp, f, d, y, mode=mode)
        rm = oracle.frame(vm, f, d, y, mode=mode)
        same = all(np.array_equal(rp[key], rm[key]) and np.array_equal(rp[key], base[key])
                   for key in ("face_idx", "nn_ab", "nn_ba"))
        if not same:
            skipped += 1
            continue
        # unequal steps a, b (float32 rounding of v +- h): exact for a quadratic
        fd = (b * b * (rp["loss"] - base["loss"]) + a * a * (base["loss"] - rm["loss"])) / (
            a * b * (a + b))
        assert fd == pytest.approx(base["grad_verts"][vi, k], rel=1e-7, abs=1e-12)
        checked += 1
    assert checked >= 30, (checked, skipped)


def test_gradient_invariants():
    v, f, d, y = _small_frame(n=200, m=150)
    r = oracle.frame(v, f, d, y)
    # partition of unity: the barycentric weights sum to 1, so vertex grads sum to point grads
    np.testing.assert_allclose(r["grad_verts"].sum(0), r["grad_points"].sum(0), rtol=1e-12,
                               atol=1e-15)
    # translation invariance: moving both clouds together changes nothing
    np.testing.assert_allclose(r["grad_points"].sum(0) + r["grad_targets"].sum(0), 0.0,
                               atol=1e-14)
    # gscale scales the gradient linearly and leaves the loss alone
    r2 = oracle.frame(v, f, d, y, gscale=-2.5)
    assert r2["loss"] == r["loss"]
    np.testing.assert_allclose(r2["grad_verts"], -2.5 * r["grad_verts"], rtol=1e-14,
                               atol=1e-16)


def test_gradient_shift_closed_form_on_mesh():
    """Sampled cloud of a flat mesh against its own float32 copy lifted by delta: the total
    vertex gradient of Eq. 1 is -4 delta along z (partition of unity)."""
    tr = W.flat_square(9, 400, seed=43)
    r0 = oracle.frame(tr.verts[0], tr.faces, tr.draws, tr.targets[:1], mode=oracle.UNIDIR_SUM)
    delta = np.float32(1e-4)
    y = r0["x32"].copy()
    y[:, 2] += delta
    r = oracle.frame(tr.verts[0], tr.faces, tr.draws, y)
    np.testing.assert_array_equal(r["nn_ab"], np.arange(400))
    # z is exact (the mesh is flat); x, y carry the float32 rounding of the lifted copy:
    # at most (2/N + 2/M) * 6e-8 per point, 2.4e-7 in total
    gs = r["grad_verts"].sum(0)
    assert gs[2] == pytest.approx(-4 * float(delta), rel=1e-9)
    assert np.all(np.abs(gs[:2]) < 2.4e-7)
    assert r["loss"] == pytest.approx(2 * float(delta) ** 2, rel=1e-6)


def test_loss_traj_weights_and_ragged():
    tr = W.batched_uneven(n_traj=1, grid=(8, 10), T=(3, 4), m=(200, 400))[0]
    w = np.linspace(0.5, 1.5, tr.T)
    r = oracle.loss_traj(tr, weights=w)
    per = [oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t))
           for t in range(tr.T)]
    assert r["loss_total"] == pytest.approx(sum(w[t] * per[t]["loss"] for t in range(tr.T)),
                                            rel=1e-14)
    for t in range(tr.T):
        np.testing.assert_allclose(r["grad_verts"][t], w[t] * per[t]["grad_verts"],
                                   rtol=1e-13, atol=1e-16)
