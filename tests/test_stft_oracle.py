"""Pins of the STFT oracle (CPU): the definition written as a direct DFT sum, perfect
reconstruction, and the window identity that makes it exact."""
import numpy as np
import pytest

import synth
from oracle import stft as ost


def test_window_squares_sum_to_one_at_half_overlap():
    for W in (16, 64, 1024):
        w = ost.window(W)
        assert np.allclose(w[: W // 2] ** 2 + w[W // 2:] ** 2, 1.0, atol=1e-15)


@pytest.mark.parametrize("W,H", [(16, 8), (32, 8), (16, 4)])
def test_stft_is_the_windowed_dft_of_centred_frames(W, H):
    rng = np.random.default_rng(1)
    M, T = 2, 53
    x = rng.standard_normal((M, T))
    y = ost.stft(x, W, H)
    F, N = W // 2 + 1, T // H + 1
    assert y.shape == (F, N, M)
    for n in range(N):
        for m in range(M):
            for f in range(F):
                s = 0.0
                for k in range(W):
                    t = n * H - W // 2 + k
                    if 0 <= t < T:
                        s += np.sin(np.pi * k / W) * x[m, t] * np.exp(-2j * np.pi * f * k / W)
                assert abs(y[f, n, m] - s) < 1e-12


@pytest.mark.parametrize("W,H", [(16, 8), (64, 32), (64, 16), (1024, 512)])
def test_perfect_reconstruction(W, H):
    x, _ = synth.make_time_mixture(3, 4000, 5)
    back = ost.istft(ost.stft(x, W, H), x.shape[1], W, H)
    assert np.max(np.abs(back - x)) < 1e-12 * np.max(np.abs(x))


def test_table1_shapes():
    # 8 s at 16 kHz, 1024-sample frames, shift 512 (Table 1): F = 513 bins.
    y = ost.stft(np.zeros((2, 16000 * 8)), 1024, 512)
    assert y.shape == (513, 16000 * 8 // 512 + 1, 2)


def test_real_signal_gives_real_dc_and_nyquist():
    x, _ = synth.make_time_mixture(2, 3000, 7)
    y = ost.stft(x, 64, 32)
    assert np.max(np.abs(y[0].imag)) < 1e-12 and np.max(np.abs(y[-1].imag)) < 1e-12
