"""STFT / inverse STFT oracle -- TEST INFRASTRUCTURE ONLY (only tests/ may import it).

The plain definitions of the analysis of the paper's experiments (Table 1: square-root Hann
window, frame W, shift H), with centred frames: frame n covers samples [n H - W/2, n H + W/2)
(zeros outside the signal), N = T // H + 1,

    y(n, f) = sum_k w[k] x(n H - W/2 + k) exp(-2 pi i f k / W),   w[k] = sin(pi k / W),

and weighted overlap-add synthesis x(t) = sum_n w u_n(t) / sum_n w^2 with u_n the inverse DFT
of frame n. NumPy's FFT serves as the DFT of one frame; everything else is written out.
Pinned by tests/test_stft_oracle.py (a direct DFT sum on small inputs, perfect
reconstruction, the window's overlap identity).
"""
from __future__ import annotations

import numpy as np


def window(W: int) -> np.ndarray:
    return np.sin(np.pi * np.arange(W) / W)


def frames(T: int, H: int) -> int:
    return T // H + 1


def stft(x: np.ndarray, W: int, H: int) -> np.ndarray:
    """x float [M][T] -> y complex128 [F][N][M]."""
    x = np.asarray(x, dtype=np.float64)
    M, T = x.shape
    N, F = frames(T, H), W // 2 + 1
    w = window(W)
    y = np.zeros((F, N, M), dtype=np.complex128)
    for n in range(N):
        t = n * H - W // 2 + np.arange(W)
        ok = (t >= 0) & (t < T)
        for m in range(M):
            seg = np.zeros(W)
            seg[ok] = x[m, t[ok]]
            y[:, n, m] = np.fft.rfft(w * seg)
    return y


def istft(y: np.ndarray, T: int, W: int, H: int) -> np.ndarray:
    """y complex [F][N][M] -> x float64 [M][T]."""
    y = np.asarray(y, dtype=np.complex128)
    F, N, M = y.shape
    w = window(W)
    num = np.zeros((M, T))
    den = np.zeros(T)
    for n in range(N):
        t = n * H - W // 2 + np.arange(W)
        ok = (t >= 0) & (t < T)
        den[t[ok]] += (w * w)[ok]
        for m in range(M):
            u = np.fft.irfft(y[:, n, m], n=W)
            num[m, t[ok]] += (w * u)[ok]
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
