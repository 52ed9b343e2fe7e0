"""Seeded synthetic inputs for two-source FCA (shared by the oracle tests, the GPU
tests and the benchmark).

This module holds no step of the EM method. It draws mixtures from the generative
model the paper assumes (Sec. 2: y = x1 + x2, x_j ~ CN(0, v_j S_j), Eq. (fullrank)),
builds the initial parameters (Algorithm 1 leaves the initial values to the user) and
optionally encodes the mixture as FP16 with a per-frequency scale.

Recipe (all in FP64 NumPy, PCG64 streams, cast to complex64 at the end):
  * per mixture a ``numpy.random.Generator(PCG64(seed))``;
  * for k = 1, 2: a_k(f) ~ CN(0, I_M) for f = 0..F-1, R_k(f) = a_k a_k^H + delta I;
  * v_k(n, f) = exp(sigma g), g ~ N(0, 1), drawn as [F][N] for k = 1 then k = 2;
  * z ~ CN(0, I_M) drawn as [2][F][N][M]; x_k = sqrt(v_k) chol(R_k) z_k; y = x1 + x2.
CN(0, 1) means real and imaginary parts each N(0, 1/2) (the pi^-M density of Eq. (like)).

Initial parameters (Algorithm 1 leaves them to the user; the paper's experiment estimates
the spatial covariances from time-frequency masks). Two recipes:
  * "mask" (default): a stand-in for a mask-based estimate. The ideal binary mask
    m_1(n,f) = [|x_1(n,f)|^2 > |x_2(n,f)|^2], m_2 = 1 - m_1, taken from the generator's source
    images, gives S_j^(0)(f) = mean over {n : m_j = 1} of M y y^H / |y|^2, plus 0.01 I
    (I when the mask is empty), and v_j^(0)(n,f) = max(|y|^2, eps_f) (0.1 + 0.8 m_j) / tr S_j^(0);
  * "random": S_j^(0)(f) = b_j b_j^H + I and v_j^(0)(n, f) = max(|y(n,f)|^2, eps_f) /
    (2 tr S_j^(0)(f)), with b_j(f) ~ CN(0, I_M) from a counter-based generator, so that the
    same values can be drawn independently anywhere (the CUDA library draws them on the device
    for a problem given without initial values): entry m of b_j(f) is draw t = f M + m of
    source j, taken from the Philox4x64-10 block of counter (t, 0, 0, 0) under the key
    (seed, 1000 + j) (numpy.random.Philox), whose words w0, w1 give
    u_k = (floor(w_k / 2^11) + 1/2) 2^-53 and b = sqrt(-ln u0) (cos 2 pi u1 + i sin 2 pi u1).
eps_f = 1e-12 mean_n |y(n,f)|^2, |y|^2 = sum_m (re^2 + im^2).
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 1805_06572


@dataclasses.dataclass(frozen=True)
class MixtureConfig:
    name: str
    M: int
    F: int
    N: int
    iters: int
    delta: float
    sigma: float
    storage: str = "c64"   # "c64" or "f16"


# The workloads: small (M=2), mid (M=4, the benchmark workload), precision (M=8, FP16 y).
CONFIGS = {
    "small": MixtureConfig("small", M=2, F=257, N=300, iters=20, delta=0.1, sigma=1.0),
    "mid": MixtureConfig("mid", M=4, F=513, N=1000, iters=50, delta=0.05, sigma=1.5),
    "precision": MixtureConfig("precision", M=8, F=1025, N=4000, iters=100, delta=0.05,
                               sigma=1.5, storage="f16"),
}
CONFIG_INDEX = {"small": 0, "mid": 1, "precision": 2, "batch": 3, "serve": 4}


def config_seed(config: str, mixture_index: int = 0) -> int:
    return BASE_SEED + 7919 * CONFIG_INDEX[config] + mixture_index


def _cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex normal CN(0, 1) samples: real, imaginary parts N(0, 1/2)."""
    g = rng.standard_normal(tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)


def make_mixture(M: int, F: int, N: int, delta: float, sigma: float, seed: int):
    """Draw one mixture. Returns dict with y (complex64 [F][N][M]), the true R [2][F][M][M]
    (complex128), the true v [2][F][N] (float64) and the source images x [2][F][N][M]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.stack([_cn(rng, (F, M)) for _ in range(2)])                  # [2][F][M]
    R = np.einsum("kfi,kfj->kfij", a, a.conj()) + delta * np.eye(M)     # [2][F][M][M]
    v = np.stack([np.exp(sigma * rng.standard_normal((F, N))) for _ in range(2)])
    z = _cn(rng, (2, F, N, M))
    C = np.linalg.cholesky(R)                                           # R = C C^H
    x = np.sqrt(v)[..., None] * np.einsum("kfij,kfnj->kfni", C, z)
    y = (x[0] + x[1]).astype(np.complex64)
    return {"y": y, "R": R, "v": v, "x": x.astype(np.complex64)}


def init_params(y: np.ndarray, seed: int, x: np.ndarray | None = None, recipe: str | None = None):
    """Initial (v0 [2][F][N] float64, S0 [2][F][M][M] complex128) for mixture y [F][N][M].
    recipe "mask" needs the source images x [2][F][N][M]; the default is "mask" when x is
    given, else "random"."""
    recipe = recipe or ("mask" if x is not None else "random")
    if recipe == "mask":
        return _mask_init(y, x)
    F, N, M = y.shape
    yd = y.astype(np.complex128)
    S0 = np.empty((2, F, M, M), np.complex128)
    for j in range(2):
        b = philox_cn(seed, j, F * M).reshape(F, M)
        S0[j] = np.einsum("fi,fj->fij", b, b.conj()) + np.eye(M)
    pw = np.sum(yd.real ** 2 + yd.imag ** 2, axis=2)                    # [F][N]
    eps = 1e-12 * pw.mean(axis=1, keepdims=True)
    tr = np.real(np.einsum("kfii->kf", S0))                             # [2][F]
    v0 = np.maximum(pw, eps)[None] / (2.0 * tr[:, :, None])
    return v0, S0


def philox_cn(seed: int, j: int, count: int) -> np.ndarray:
    """Draws 0..count-1 of source j of the "random" recipe (module docstring): CN(0, 1) values
    from the Philox4x64-10 blocks of counters 0..count-1 under the key (seed, 1000 + j)."""
    # numpy's Philox advances its 256-bit counter before each block: start from all ones.
    bg = np.random.Philox(counter=np.full(4, 2**64 - 1, dtype=np.uint64),
                          key=np.array([seed % 2**64, 1000 + j], dtype=np.uint64))
    w = bg.random_raw(4 * count).reshape(count, 4)
    u0 = ((w[:, 0] >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u1 = ((w[:, 1] >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    r = np.sqrt(-np.log(u0))
    th = 2 * np.pi * u1
    return r * np.cos(th) + 1j * (r * np.sin(th))


def _mask_init(y: np.ndarray, x: np.ndarray):
    F, N, M = y.shape
    yd = y.astype(np.complex128)
    xd = x.astype(np.complex128)
    px = np.sum(np.abs(xd) ** 2, axis=3)                                 # [2][F][N]
    m1 = (px[0] > px[1]).astype(np.float64)
    masks = np.stack([m1, 1.0 - m1])
    pw = np.sum(np.abs(yd) ** 2, axis=2)                                # [F][N]
    eps = 1e-12 * pw.mean(axis=1, keepdims=True)
    wn = M / np.maximum(pw, np.where(pw > 0, 0.0, 1.0))                 # M / |y|^2 (0 for y = 0)
    wn = np.where(pw > 0, wn, 0.0)
    S0 = np.empty((2, F, M, M), np.complex128)
    for j in range(2):
        cnt = masks[j].sum(axis=1)
        S = np.einsum("fn,fni,fnj->fij", masks[j] * wn, yd, yd.conj())
        S = S / np.maximum(cnt, 1.0)[:, None, None] + 0.01 * np.eye(M)
        S0[j] = np.where((cnt > 0)[:, None, None], S, np.eye(M))
    tr = np.real(np.einsum("kfii->kf", S0))
    v0 = np.maximum(pw, eps)[None] * (0.1 + 0.8 * masks) / tr[:, :, None]
    return v0, S0


def quantize_f16(y: np.ndarray):
    """FP16 storage of y with a per-frequency power scale g_f = (mean_n |y|^2 / M)^(-1/2)
    (FP64 mean of re^2 + im^2 over the bin's N M values, 1 / sqrt in FP64, rounded to float32;
    g_f y formed exactly in FP64 and rounded to float16, nearest even).

    Returns (y16 float16 [F][N][M][2] interleaved re/im of g_f y, g float32 [F]) and the
    dequantised complex128 mixture y16 / g_f that the EM actually sees."""
    F, N, M = y.shape
    yd = y.astype(np.complex128)
    p = np.mean(yd.real ** 2 + yd.imag ** 2, axis=(1, 2))
    g = np.where(p > 0, 1.0 / np.sqrt(np.where(p > 0, p, 1.0)), 1.0).astype(np.float32)
    s = yd * g.astype(np.float64)[:, None, None]
    y16 = np.stack([s.real, s.imag], axis=-1).astype(np.float16)
    deq = (y16[..., 0].astype(np.float64) + 1j * y16[..., 1].astype(np.float64)) \
        / g.astype(np.float64)[:, None, None]
    return y16, g, deq


def make_config(name: str, mixture_index: int = 0, F: int | None = None, recipe: str = "mask"):
    """Mixture + initial params for a named workload (optionally with fewer bins)."""
    c = CONFIGS[name]
    seed = config_seed(name, mixture_index)
    mix = make_mixture(c.M, F or c.F, c.N, c.delta, c.sigma, seed)
    v0, S0 = init_params(mix["y"], seed, x=mix["x"], recipe=recipe)
    return c, mix, v0, S0


def make_time_mixture(M: int, T: int, seed: int, taps: int = 64):
    """Two-source M-channel time-domain mixture (input for the STFT front-end): each source is
    white Gaussian noise under a slowly varying log-normal envelope (power changing from frame
    to frame, as speech does), convolved per microphone with a random exponentially decaying
    FIR of `taps` taps (a short room response). Returns (y [M][T], x [2][M][T]) float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.zeros((2, M, T))
    for k in range(2):
        env = np.exp(0.75 * np.repeat(rng.standard_normal(T // 256 + 1), 256)[:T])
        s = env * rng.standard_normal(T)
        decay = np.exp(-np.arange(taps) / (taps / 4.0))
        for m in range(M):
            h = rng.standard_normal(taps) * decay
            x[k, m] = np.convolve(s, h)[:T]
    return x[0] + x[1], x
