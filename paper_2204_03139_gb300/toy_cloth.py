"""A toy real-to-sim loop: fitting cloth parameters through the point-cloud loss.

The paper fits two scalar multipliers (w_stiff, w_mass) of a differentiable cloth simulator
to observed point clouds (Sec. III-C, Sec. IV-B): the loss between points sampled on the
simulated mesh and the observed cloud is differentiated with respect to the mesh vertices
(this library), and the simulator carries that gradient on to the parameters. The
parameters are optimised through a sigmoid reparameterisation, w = sigma(s) (10 - 0.1) + 0.1,
started at the middle of the range, with Adam (learning rate 0.2, 50 iterations), keeping
the parameters of the lowest loss seen.

The simulator here is NOT the paper's (a differentiable garment simulator, which is out of
scope): it is a small analytic stand-in, differentiable in torch, so that the whole chain --
parameters -> vertices -> sampled points -> loss -> vertex gradient -> parameters -- runs
end to end. A cloth lying on a table is lifted by one corner along a fixed arc. The mass
multiplier sets how steeply the lifted part hangs (a catenary whose parameter shrinks as the
cloth gets heavier); the stiffness multiplier sets how much the hanging part resists being
pulled in toward the grasped corner. The two act on different features of the shape, so both
can be recovered.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib
from .autograd import loss_traj

W_LO, W_HI = 0.1, 10.0  # parameter range of both multipliers (Sec. IV-B)


def params_from_s(s: torch.Tensor) -> torch.Tensor:
    """w = sigmoid(s) (W_HI - W_LO) + W_LO: s = 0 is the middle of the range."""
    return torch.sigmoid(s) * (W_HI - W_LO) + W_LO


def s_from_params(w) -> torch.Tensor:
    w = torch.as_tensor(w, dtype=torch.float64)
    p = (w - W_LO) / (W_HI - W_LO)
    return torch.log(p / (1 - p))


def grid_faces(n: int) -> np.ndarray:
    """Triangles of an n x n vertex grid, 2 (n-1)^2 of them (vertex (i, j) is j * n + i)."""
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    a = (j * n + i).ravel()
    f = np.empty((2 * a.size, 3), np.int32)
    f[0::2] = np.stack([a, a + 1, a + n + 1], 1)
    f[1::2] = np.stack([a, a + n + 1, a + n], 1)
    return f


class ToyCloth:
    """Analytic lifted cloth on an n x n grid over T frames, differentiable in (w_stiff, w_mass).

    Frame t has phase p = t / (T - 1). The grasped corner (rest position (0, 0)) moves to
    c(p) = (0.2 p, 0.2 p, 0.6 p - 0.1 p^2). A vertex at rest distance rho from the corner
    hangs at height h = max(0, c_z - a (cosh(rho / a) - 1)) with catenary parameter
    a = 0.15 + 0.2 sqrt(W0 / w_mass), and is pulled toward the corner by
    min(k h, rho / 2) with k = 0.9 / (1 + 0.3 w_stiff); the lifted part follows the corner in
    proportion to its height. The max and min are smoothed (softplus with a 2 mm scale) so
    that every vertex has a gradient."""

    W0 = 5.05  # the middle of the range

    def __init__(self, n: int = 25, T: int = 10, device="cuda:0", dtype=torch.float32):
        self.n, self.T = n, T
        self.device, self.dtype = torch.device(device), dtype
        g = torch.linspace(0.0, 1.0, n, dtype=torch.float64)
        v, u = torch.meshgrid(g, g, indexing="ij")  # row j = v, column i = u
        self.u = u.reshape(-1).to(self.device, dtype)
        self.v = v.reshape(-1).to(self.device, dtype)
        self.rho = torch.sqrt(self.u ** 2 + self.v ** 2)
        self.faces = torch.from_numpy(grid_faces(n)).to(self.device)
        p = torch.linspace(0.0, 1.0, T, dtype=torch.float64)
        self.cxy = (0.2 * p).to(self.device, dtype)
        self.cz = (0.6 * p - 0.1 * p * p).to(self.device, dtype)

    @property
    def V(self) -> int:
        return self.n * self.n

    @staticmethod
    def _smooth_pos(x, scale=2e-3):
        return scale * torch.nn.functional.softplus(x / scale)

    def verts(self, w: torch.Tensor) -> torch.Tensor:
        """[T, V, 3] vertices for w = (w_stiff, w_mass)."""
        w = w.to(self.dtype)
        w_stiff, w_mass = w[0], w[1]
        a = 0.15 + 0.2 * torch.sqrt(self.W0 / w_mass)
        k = 0.9 / (1.0 + 0.3 * w_stiff)
        rho, u, v = self.rho[None], self.u[None], self.v[None]
        cz = self.cz[:, None]
        # cosh(rho / a) - 1 stays moderate: rho <= sqrt(2), a >= 0.15
        h = self._smooth_pos(cz - a * (torch.cosh(rho / a) - 1.0))
        pull = rho / 2 - self._smooth_pos(rho / 2 - k * h)  # smooth min(k h, rho / 2)
        inv = torch.where(rho > 0, 1.0 / torch.clamp(rho, min=1e-12), torch.zeros_like(rho))
        follow = h / torch.clamp(cz, min=1e-6)
        x = u - pull * u * inv + follow * self.cxy[:, None]
        y = v - pull * v * inv + follow * self.cxy[:, None]
        return torch.stack([x, y, h], dim=-1).contiguous()


def sample_targets(cloth: ToyCloth, w_true, m: int, noise: float = 2e-3, seed: int = 0,
                   face_mask=None) -> torch.Tensor:
    """Observed clouds: m area-weighted samples per frame of the cloth at w_true (this
    library's sampler), plus N(0, noise) per coordinate. [T, m, 3] on the cloth's device."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    with torch.no_grad():
        verts = cloth.verts(torch.as_tensor(w_true, dtype=torch.float64).to(cloth.device))
        verts = verts.float().contiguous()
        draws = torch.rand((cloth.T, m, 3), generator=gen).clamp_(max=1 - 2 ** -24)
        pts, _, _ = _lib.dc_sample(verts, cloth.faces, draws.to(cloth.device), face_idx=False,
                                   bary=False, face_mask=face_mask)
        pts = pts + noise * torch.randn(pts.shape, generator=gen).to(cloth.device)
    return pts.contiguous()


def real_to_sim(cloth: ToyCloth, targets: torch.Tensor, n: int, iters: int = 50,
                lr: float = 0.2, mode: int = _lib.UNIDIR_SUM, frame_w=None, seed: int = 1,
                face_mask=None, s0=None) -> dict:
    """Adam on s (w = params_from_s(s)), starting at the middle of the range, keeping the
    parameters of the lowest loss seen. Each iteration samples n fresh points per frame.
    frame_w [T] (optional) weights the frames; frames of weight 0 cost nothing.
    Returns the best w, its loss and the history of (w, loss)."""
    dev = cloth.device
    s = torch.zeros(2, dtype=torch.float64, device=dev) if s0 is None else s0.clone().to(dev)
    s.requires_grad_(True)
    opt = torch.optim.Adam([s], lr=lr)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    fw = None if frame_w is None else torch.as_tensor(frame_w, dtype=torch.float32, device=dev)
    hist, best = [], (math.inf, None)
    for _ in range(iters):
        w = params_from_s(s)
        verts = cloth.verts(w).float()
        draws = torch.rand((cloth.T, n, 3), generator=gen).clamp_(max=1 - 2 ** -24).to(dev)
        total, _ = loss_traj(verts, cloth.faces, draws, targets, mode=mode, frame_w=fw,
                             face_mask=face_mask)
        opt.zero_grad()
        total.backward()
        lv = float(total.detach())
        wv = w.detach().cpu().numpy()
        hist.append((wv, lv))
        if lv < best[0]:
            best = (lv, wv)
        opt.step()
    return {"w": best[1], "loss": best[0], "history": hist}


def main():
    """python -m paper_2204_03139_gb300.toy_cloth: fit a synthetic target and print the fit."""
    import argparse

    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--w-true", type=float, nargs=2, default=[2.0, 7.5],
                   metavar=("W_STIFF", "W_MASS"))
    p.add_argument("--grid", type=int, default=25)
    p.add_argument("--frames", type=int, default=25)
    p.add_argument("--points", type=int, default=8192)
    p.add_argument("--iters", type=int, default=50)
    p.add_argument("--last-frame-only", action="store_true")
    a = p.parse_args()
    cloth = ToyCloth(n=a.grid, T=a.frames)
    targets = sample_targets(cloth, a.w_true, a.points)
    fw = None
    if a.last_frame_only:
        fw = np.zeros(a.frames, np.float32)
        fw[-1] = 1.0
    r = real_to_sim(cloth, targets, a.points, iters=a.iters, frame_w=fw)
    for k, (w, loss) in enumerate(r["history"]):
        print(f"iter {k:3d}  w_stiff {w[0]:7.3f}  w_mass {w[1]:7.3f}  loss {loss:.6f}")
    print(f"best: w_stiff {r['w'][0]:.3f}  w_mass {r['w'][1]:.3f}  loss {r['loss']:.6f}  "
          f"(true {a.w_true[0]:.3f}, {a.w_true[1]:.3f})")


if __name__ == "__main__":
    main()
