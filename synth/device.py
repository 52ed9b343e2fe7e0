"""Seeded synthetic workloads drawn on a torch device, for the many-mixture configurations
that the NumPy generator (synth/__init__.py) is too slow to draw on the host.

Like the NumPy generator this holds no step of the EM method: it draws mixtures from the
paper's generative model (Sec. 2: y = x1 + x2, x_j ~ CN(0, v_j S_j)) and forms the same
mask-based initial parameters. Same recipe, different random stream (torch's Philox on the
device instead of PCG64), so the values differ from synth.make_mixture for the same seed;
the parity tests copy the drawn inputs of sampled mixtures back to the host for the oracle.

Workloads:
  batch  512 mixtures, M uniform in {2, 4, 6}, N uniform in [200, 6000], F = 513,
         delta = 0.05, sigma = 1.5, 50 EM iterations each;
  serve  requests with M uniform in {2, 4, 8}, N uniform in [60, 1000], F = 513, delta = 0.05,
         sigma = 1.5, 30 EM iterations each, Poisson arrivals at 200 requests/s.
Shapes (and arrival gaps) come from numpy PCG64(config_seed(name)); mixture k's values from a
torch generator seeded with config_seed(name, k).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import config_seed


@dataclasses.dataclass(frozen=True)
class ManyConfig:
    name: str
    count: int
    Ms: tuple
    N_lo: int
    N_hi: int
    F: int
    iters: int
    delta: float
    sigma: float
    rate: float = 0.0  # arrivals per second (serving)


MANY = {
    "batch": ManyConfig("batch", 512, (2, 4, 6), 200, 6000, 513, 50, 0.05, 1.5),
    "serve": ManyConfig("serve", 2000, (2, 4, 8), 60, 1000, 513, 30, 0.05, 1.5, rate=200.0),
}


def shapes(name: str, count: int | None = None):
    """(M, F, N) int lists of the workload's first `count` mixtures, and the arrival gaps (s)."""
    c = MANY[name]
    n = c.count if count is None else count
    rng = np.random.Generator(np.random.PCG64(config_seed(name)))
    M = rng.choice(np.asarray(c.Ms), size=c.count)
    N = rng.integers(c.N_lo, c.N_hi + 1, size=c.count)
    gaps = rng.exponential(1.0 / c.rate, size=c.count) if c.rate > 0 else np.zeros(c.count)
    return [int(m) for m in M[:n]], [c.F] * n, [int(x) for x in N[:n]], gaps[:n]


def mixture(M: int, F: int, N: int, delta: float, sigma: float, seed: int, device):
    """One mixture and its mask-based initial parameters on `device`:
    y complex64 [F][N][M], v0 float64 [2][F][N], S0 complex128 [2][F][M][M]."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))

    def cn(shape):  # CN(0, 1): real and imaginary parts N(0, 1/2)
        g = torch.randn(tuple(shape) + (2,), generator=gen, device=device, dtype=torch.float32)
        return torch.view_as_complex(g * (0.5 ** 0.5))

    eye = torch.eye(M, dtype=torch.complex128, device=device)
    a = cn((2, F, M)).to(torch.complex128)
    R = a[..., :, None] * a[..., None, :].conj() + delta * eye
    # R = C C^H; the factor is tiny ([2][F][M][M]) and taken on the host.
    C = torch.from_numpy(np.linalg.cholesky(R.cpu().numpy())).to(device=device, dtype=torch.complex64)
    v = torch.exp(sigma * torch.randn((2, F, N), generator=gen, device=device, dtype=torch.float32))
    z = cn((2, F, N, M))
    x = v.sqrt()[..., None] * torch.einsum("kfij,kfnj->kfni", C, z)       # [2][F][N][M]
    y = (x[0] + x[1]).contiguous()
    # Mask-based initial values (the recipe of synth.init_params, "mask").
    px = (x.abs() ** 2).sum(-1)                                           # [2][F][N]
    m1 = (px[0] > px[1]).to(torch.float64)
    masks = torch.stack([m1, 1.0 - m1])
    yd = y.to(torch.complex128)
    pw = (yd.abs() ** 2).sum(-1)                                          # [F][N]
    eps = 1e-12 * pw.mean(dim=1, keepdim=True)
    wn = torch.where(pw > 0, M / torch.where(pw > 0, pw, torch.ones_like(pw)), torch.zeros_like(pw))
    S0 = torch.empty((2, F, M, M), dtype=torch.complex128, device=device)
    for j in range(2):
        cnt = masks[j].sum(dim=1)
        w = (masks[j] * wn).to(torch.complex128)
        S = torch.einsum("fn,fni,fnj->fij", w, yd, yd.conj())
        S = S / torch.clamp(cnt, min=1.0)[:, None, None] + 0.01 * eye
        S0[j] = torch.where((cnt > 0)[:, None, None], S, eye.expand(F, M, M))
    tr = torch.diagonal(S0, dim1=-2, dim2=-1).real.sum(-1)                # [2][F]
    v0 = torch.maximum(pw, eps)[None] * (0.1 + 0.8 * masks) / tr[:, :, None]
    return y, v0.contiguous(), S0


def make_packed(name: str, device, count: int | None = None):
    """The workload's mixtures drawn on `device` and packed back to back in the layouts of the
    batch entry points (include/fca.h). Returns dict(M, F, N, y, v0, S0, gaps, iters)."""
    import torch

    c = MANY[name]
    M, F, N, gaps = shapes(name, count)
    fnm = [f * n * m for m, f, n in zip(M, F, N)]
    y = torch.empty(sum(fnm), dtype=torch.complex64, device=device)
    v0 = torch.empty(sum(2 * f * n for f, n in zip(F, N)), dtype=torch.float64, device=device)
    S0 = torch.empty(sum(2 * f * m * m for m, f in zip(M, F)), dtype=torch.complex128, device=device)
    yo = vo = so = 0
    for k, (m, f, n) in enumerate(zip(M, F, N)):
        yk, vk, sk = mixture(m, f, n, c.delta, c.sigma, config_seed(name, k), device)
        y[yo:yo + yk.numel()] = yk.reshape(-1)
        v0[vo:vo + vk.numel()] = vk.reshape(-1)
        S0[so:so + sk.numel()] = sk.reshape(-1)
        yo, vo, so = yo + yk.numel(), vo + vk.numel(), so + sk.numel()
    return {"M": M, "F": F, "N": N, "y": y, "v0": v0, "S0": S0, "gaps": gaps, "iters": c.iters}
