"""Seeded synthetic inputs for the mesh-to-point-cloud loss (cloth grids, draws, target clouds).

This module is shared by the CUDA path, the oracle, the tests and the bench. It holds none of
the loss arithmetic (no areas, no prefix sums, no face picks, no barycentric points, no
distances): it only builds meshes, motions, uniform draws and noisy target clouds.

The paper's recordings (Section IV-D) and simulator scenes (Section IV-F) are not available;
these procedural stand-ins reproduce their shape: a square cloth grid triangulated into
2(n-1)^2 faces, a trajectory of T frames of vertex positions, per-frame target clouds with
sensor-like noise, outliers and partial dropout.

Every array is C-contiguous: vertices and points float32 [.., 3], faces int32 [F, 3], draws
float32 [.., 3] holding (r_f, r_1, r_2) in [0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2204_03139
_ONE_MINUS = np.nextafter(np.float32(1.0), np.float32(0.0))


# ---------------------------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------------------------
@dataclass
class Trajectory:
    """One cloth trajectory: T frames over a shared triangle list.

    Frames may be ragged (config "batched uneven"): frame t has n_pts[t] sim samples (draws)
    and m_pts[t] target points, stored flat with offsets n_off / m_off.
    """

    verts: np.ndarray            # [T, V, 3] float32
    faces: np.ndarray            # [F, 3] int32
    draws: np.ndarray            # [sum N_t, 3] float32
    targets: np.ndarray          # [sum M_t, 3] float32
    n_off: np.ndarray            # [T+1] int64
    m_off: np.ndarray            # [T+1] int64
    face_mask: np.ndarray | None = None  # [F] uint8: sample only faces with a nonzero entry
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def T(self) -> int:
        return int(self.verts.shape[0])

    @property
    def V(self) -> int:
        return int(self.verts.shape[1])

    @property
    def F(self) -> int:
        return int(self.faces.shape[0])

    def n(self, t: int) -> int:
        return int(self.n_off[t + 1] - self.n_off[t])

    def m(self, t: int) -> int:
        return int(self.m_off[t + 1] - self.m_off[t])

    @property
    def uniform(self) -> bool:
        n = np.diff(self.n_off)
        m = np.diff(self.m_off)
        return bool(np.all(n == n[0]) and np.all(m == m[0]))

    def draws_tn3(self) -> np.ndarray:
        """[T, N, 3] view (uniform trajectories only)."""
        assert self.uniform
        return self.draws.reshape(self.T, -1, 3)

    def targets_tm3(self) -> np.ndarray:
        assert self.uniform
        return self.targets.reshape(self.T, -1, 3)

    def frame_draws(self, t: int) -> np.ndarray:
        return self.draws[self.n_off[t]:self.n_off[t + 1]]

    def frame_targets(self, t: int) -> np.ndarray:
        return self.targets[self.m_off[t]:self.m_off[t + 1]]

    def pairs(self) -> int:
        """Unique (sim point, target point) pairs summed over frames."""
        return int(np.sum(np.diff(self.n_off) * np.diff(self.m_off)))


# ---------------------------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------------------------
def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_draws(rng: np.random.Generator, n: int) -> np.ndarray:
    """n triples (r_f, r_1, r_2) of U[0,1) draws as float32.

    A float64 draw just below 1 can round up to 1.0 when cast to float32; those are clamped
    to the largest float32 below 1 so every draw stays in [0, 1).
    """
    r = rng.random((n, 3)).astype(np.float32)
    np.minimum(r, _ONE_MINUS, out=r)
    return np.ascontiguousarray(r)


def grid_faces(n: int) -> np.ndarray:
    """Triangle list of an n x n vertex grid: 2 (n-1)^2 faces, consistently oriented.

    Vertex (ix, iy) has index iy * n + ix; each quad (a, b, c, d) = ((ix,iy), (ix+1,iy),
    (ix,iy+1), (ix+1,iy+1)) is split into (a, b, d) and (a, d, c).
    """
    ix, iy = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    a = (iy * n + ix).ravel()
    b = a + 1
    c = a + n
    d = a + n + 1
    f = np.empty((2 * a.size, 3), dtype=np.int32)
    f[0::2] = np.stack([a, b, d], axis=1)
    f[1::2] = np.stack([a, d, c], axis=1)
    return f


def grid_uv(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Rest coordinates (u, v) in [0, 1]^2 of the n x n grid, in vertex-index order."""
    g = np.linspace(0.0, 1.0, n)
    u, v = np.meshgrid(g, g, indexing="xy")
    return u.ravel(), v.ravel()


def wave_surface(u: np.ndarray, v: np.ndarray, bump: float = 0.0) -> np.ndarray:
    """z = 0.05 sin(2 pi u) cos(2 pi v) on the unit square, optionally plus a Gaussian bump of
    amplitude `bump` (sigma 0.2 m) centred at (0.5, 0.5)."""
    z = 0.05 * np.sin(2 * np.pi * u) * np.cos(2 * np.pi * v)
    if bump:
        r2 = (u - 0.5) ** 2 + (v - 0.5) ** 2
        z = z + bump * np.exp(-r2 / (2 * 0.2 ** 2))
    return np.stack([u, v, z], axis=-1)


def lift_motion(u: np.ndarray, v: np.ndarray, s: float, a: float = 0.35,
                lift: float = 1.0) -> np.ndarray:
    """Procedural lift of a cloth lying on a table, grasped at its (0, 0) corner.

    s in [0, 1] is the trajectory phase. The corner follows the quadratic arc
    c(s) = (0.2 s, 0.2 s, lift (0.6 s - 0.1 s^2)); a point at rest distance rho from the corner
    hangs as a catenary of parameter a below it, h = max(0, c_z - a (cosh(rho / a) - 1)), is
    pulled toward the corner by half its height (at most half its rest distance), and rides
    along with the corner in proportion to how far it is lifted.
    """
    cx, cy = 0.2 * s, 0.2 * s
    cz = lift * (0.6 * s - 0.1 * s * s)
    rho = np.hypot(u, v)
    h = np.maximum(0.0, cz - a * (np.cosh(rho / a) - 1.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        dx = np.where(rho > 0, u / np.where(rho > 0, rho, 1), 0.0)
        dy = np.where(rho > 0, v / np.where(rho > 0, rho, 1), 0.0)
    pull = np.minimum(0.5 * h, 0.5 * rho)
    frac = h / cz if cz > 0 else np.zeros_like(h)
    x = u - pull * dx + frac * cx
    y = v - pull * dy + frac * cy
    return np.stack([x, y, h], axis=-1)


def upper_half_mask(n_grid: int) -> np.ndarray:
    """[F] uint8 mask of the faces of an n x n grid whose rest centroid lies in the upper half
    (v > 1/2): the subset the paper samples from in its fold scenario, where the half of the
    cloth that stays flat on the table is hidden from the cameras (Sec. IV-F)."""
    _, v = grid_uv(n_grid)
    f = grid_faces(n_grid)
    return np.ascontiguousarray((v[f].mean(axis=1) > 0.5).astype(np.uint8))


def add_outliers(rng: np.random.Generator, pts: np.ndarray, frac: float) -> np.ndarray:
    """Replace a fraction of the points by uniform draws in the cloud's bounding box."""
    k = int(round(frac * pts.shape[0]))
    if k == 0:
        return pts
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    idx = rng.choice(pts.shape[0], size=k, replace=False)
    pts = pts.copy()
    pts[idx] = lo + rng.random((k, 3)) * (hi - lo)
    return pts


def planar_dropout(rng: np.random.Generator, pts: np.ndarray, p: float) -> np.ndarray:
    """Drop the points whose projection on a random unit direction lies above the (1-p)
    quantile: a planar region missing from a merged depth-camera cloud."""
    if p <= 0:
        return pts
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    proj = pts @ d
    keep = proj <= np.quantile(proj, 1.0 - p)
    return pts[keep]


def _offsets(counts) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(np.asarray(counts, dtype=np.int64))]).astype(np.int64)


# ---------------------------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------------------------
def single_frame(seed: int = SEED_BASE + 1, n_grid: int = 25, n_samples: int = 2048,
                 m_target: int = 2048) -> Trajectory:
    """Single frame: 25x25 grid on a 1 m square with z = 0.05 sin(2 pi x) cos(2 pi y);
    2048 draws; target = 2048 points of the same surface plus a 3 cm Gaussian bump (sigma
    0.2 m), taken at uniform parameter positions, plus N(0, 2 mm) noise."""
    rng = rng_for(seed)
    u, v = grid_uv(n_grid)
    verts = wave_surface(u, v)[None].astype(np.float32)
    faces = grid_faces(n_grid)
    draws = uniform_draws(rng, n_samples)
    tu, tv = rng.random(m_target), rng.random(m_target)
    tgt = wave_surface(tu, tv, bump=0.03) + rng.normal(0.0, 0.002, (m_target, 3))
    return Trajectory(verts=np.ascontiguousarray(verts), faces=faces, draws=draws,
                      targets=np.ascontiguousarray(tgt.astype(np.float32)),
                      n_off=_offsets([n_samples]), m_off=_offsets([m_target]),
                      name="single_frame_25x25_2048", meta={"seed": seed})


def lift_trajectory(seed: int, n_grid: int, T: int, n_samples, m_target, a: float = 0.35,
                    lift: float = 1.0, jitter: float = 0.001, noise: float = 0.002,
                    outliers: float = 0.03, dropout_max: float = 0.0,
                    name: str = "") -> Trajectory:
    """A lift trajectory and its observed clouds.

    Sim vertices: lift_motion at phase s = t / (T - 1) plus N(0, jitter) per vertex.
    Targets: the same motion with catenary parameter 1.1 a and lift 0.95, evaluated at uniform
    parameter positions, with N(0, noise) per coordinate, a fraction `outliers` replaced by
    uniform points in the frame's bounding box, and (if dropout_max > 0) a planar dropout of
    p ~ U[0, dropout_max]. When m_target is an int every frame has that many target points;
    n_samples may be an int or "match" (N_t = M_t after dropout).
    """
    rng = rng_for(seed)
    u, v = grid_uv(n_grid)
    faces = grid_faces(n_grid)
    verts = np.empty((T, n_grid * n_grid, 3), dtype=np.float32)
    draws, tgts, ns, ms = [], [], [], []
    for t in range(T):
        s = t / (T - 1) if T > 1 else 1.0
        p = lift_motion(u, v, s, a=a, lift=lift) + rng.normal(0.0, jitter, (u.size, 3))
        verts[t] = p.astype(np.float32)
        m0 = int(m_target)
        if dropout_max > 0:
            pdrop = rng.uniform(0.0, dropout_max)
            m_raw = int(np.ceil(m0 / (1.0 - pdrop))) if pdrop < 1 else m0
        else:
            pdrop, m_raw = 0.0, m0
        tu, tv = rng.random(m_raw), rng.random(m_raw)
        clean = lift_motion(tu, tv, s, a=1.1 * a, lift=0.95 * lift)
        tgt = clean + rng.normal(0.0, noise, clean.shape)
        tgt = add_outliers(rng, tgt, outliers)
        if dropout_max > 0:
            tgt = planar_dropout(rng, tgt, pdrop)
            tgt = tgt[:m0] if tgt.shape[0] > m0 else tgt
        m_t = tgt.shape[0]
        n_t = m_t if n_samples == "match" else int(n_samples)
        draws.append(uniform_draws(rng, n_t))
        tgts.append(tgt.astype(np.float32))
        ns.append(n_t)
        ms.append(m_t)
    return Trajectory(verts=verts, faces=faces,
                      draws=np.ascontiguousarray(np.concatenate(draws)),
                      targets=np.ascontiguousarray(np.concatenate(tgts)),
                      n_off=_offsets(ns), m_off=_offsets(ms), name=name,
                      meta={"seed": seed, "n_grid": n_grid, "T": T, "a": a, "lift": lift})


def trajectory_50x50(seed: int = SEED_BASE + 2, T: int = 40, n: int = 10_000,
                     m: int = 10_000) -> Trajectory:
    """Trajectory: 50x50 grid (2500 vertices, 4802 faces), T = 40 frames, 10 000 samples per
    frame against 10 000-point targets (2 mm noise, 3% outliers)."""
    return lift_trajectory(seed, 50, T, n, m, name=f"trajectory_50x50_T{T}_{n}x{m}")


def trajectory_100x100(seed: int = SEED_BASE + 4, T: int = 100, n: int = 32_768,
                       m: int = 32_768) -> Trajectory:
    """Differentiation at scale: 100x100 grid (10 000 vertices, 19 602 faces), T = 100,
    32 768 samples per frame against 32 768-point targets."""
    return lift_trajectory(seed, 100, T, n, m, name=f"trajectory_100x100_T{T}_{n}x{m}")


def batched_uneven(seed: int = SEED_BASE + 3, n_traj: int = 64, grid=(15, 80), T=(20, 100),
                   m=(2_000, 30_000), dropout_max: float = 0.2) -> list[Trajectory]:
    """Batched uneven: n_traj trajectories with grid sizes U{15..80}, T ~ U{20..100}, target
    clouds of U{2000..30000} points per trajectory thinned per frame by a planar dropout of
    p ~ U[0, 0.2], N(0, 3 mm) noise; N_t = M_t."""
    rng = rng_for(seed)
    out = []
    for k in range(n_traj):
        n_grid = int(rng.integers(grid[0], grid[1] + 1))
        t_len = int(rng.integers(T[0], T[1] + 1))
        m_k = int(rng.integers(m[0], m[1] + 1))
        a = float(rng.uniform(0.30, 0.40))
        lift = float(rng.uniform(0.8, 1.2))
        out.append(lift_trajectory(int(rng.integers(1 << 31)), n_grid, t_len, "match", m_k,
                                   a=a, lift=lift, noise=0.003, outliers=0.0,
                                   dropout_max=dropout_max,
                                   name=f"batched_{k}_{n_grid}x{n_grid}_T{t_len}_M{m_k}"))
    return out


def serving_requests(seed: int = SEED_BASE + 5, n_req: int = 64, rate_hz: float = 500.0,
                     big_frac: float = 0.1, small_T: int = 40, big_T: int = 100,
                     small=(50, 10_000), big=(100, 32_768)) -> list[dict]:
    """Serving stream: Poisson arrivals at `rate_hz`; a fraction big_frac of requests at the
    100x100 / 32 768-point size, the rest at the 50x50 / 10 000-point size. Frame counts may
    be reduced (small_T / big_T) to bound memory in tests."""
    rng = rng_for(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_req)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k in range(n_req):
        is_big = bool(rng.random() < big_frac)
        g, npts = big if is_big else small
        t_len = big_T if is_big else small_T
        traj = lift_trajectory(int(rng.integers(1 << 31)), g, t_len, npts, npts,
                               name=f"req{k}_{g}x{g}_T{t_len}_{npts}")
        reqs.append({"id": k, "arrival_s": float(arrivals[k]), "big": is_big, "traj": traj})
    return reqs


def flat_square(n_grid: int, n_samples: int, seed: int) -> Trajectory:
    """Flat unit square z = 0 (one frame); target = the draws' own count of uniform points.
    Used for uniform-density and equal-area closed forms."""
    rng = rng_for(seed)
    u, v = grid_uv(n_grid)
    verts = np.stack([u, v, np.zeros_like(u)], axis=-1)[None].astype(np.float32)
    faces = grid_faces(n_grid)
    draws = uniform_draws(rng, n_samples)
    tgt = np.stack([rng.random(n_samples), rng.random(n_samples),
                    np.zeros(n_samples)], axis=-1).astype(np.float32)
    return Trajectory(verts=np.ascontiguousarray(verts), faces=faces, draws=draws,
                      targets=tgt, n_off=_offsets([n_samples]), m_off=_offsets([n_samples]),
                      name=f"flat_{n_grid}", meta={"seed": seed})


def random_cloud_pair(seed: int, n: int, m: int, scale: float = 1.0):
    """Two uniform random clouds in [0, scale]^3 (float32)."""
    rng = rng_for(seed)
    a = (rng.random((n, 3)) * scale).astype(np.float32)
    b = (rng.random((m, 3)) * scale).astype(np.float32)
    return a, b


WORKLOADS = {
    "single_frame": single_frame,
    "trajectory_50x50": trajectory_50x50,
    "batched_uneven": batched_uneven,
    "trajectory_100x100": trajectory_100x100,
    "serving": serving_requests,
}
