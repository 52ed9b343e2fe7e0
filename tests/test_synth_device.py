"""The many-mixture generator (synth/device.py) on the CPU: shapes, packing, and the
statistics of its recipe (the model of Sec. 2 with the stated distributions)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import device as sdev  # noqa: E402


def test_workload_shapes_follow_the_recipe():
    M, F, N, gaps = sdev.shapes("batch")
    assert len(M) == 512 and set(M) <= {2, 4, 6} and set(F) == {513}
    assert min(N) >= 200 and max(N) <= 6000
    M, F, N, gaps = sdev.shapes("serve", 500)
    assert set(M) <= {2, 4, 8} and min(N) >= 60 and max(N) <= 1000
    assert abs(np.mean(gaps) - 1 / 200.0) < 0.1 / 200.0  # Poisson arrivals at 200/s


def test_packed_layout_and_initial_parameters():
    p = sdev.make_packed("batch", "cpu", count=3)
    M, F, N = p["M"], p["F"], p["N"]
    assert p["y"].numel() == sum(f * n * m for m, f, n in zip(M, F, N))
    assert p["v0"].numel() == sum(2 * f * n for f, n in zip(F, N))
    assert p["S0"].numel() == sum(2 * f * m * m for m, f in zip(M, F))
    assert float(p["v0"].min()) > 0
    so = 0
    for m, f in zip(M, F):
        S = p["S0"][so:so + 2 * f * m * m].reshape(2, f, m, m).numpy()
        so += 2 * f * m * m
        assert np.allclose(S, np.conj(np.swapaxes(S, -1, -2)), atol=1e-12)  # Hermitian
        assert np.linalg.eigvalsh(S).min() > 0                               # positive definite


def test_mixture_power_matches_the_model():
    # E|y_m|^2 = E[v1] (R1)_mm + E[v2] (R2)_mm with R_k = a a^H + delta I, E|a_m|^2 = 1 and
    # E[v] = exp(sigma^2 / 2) for log-normal v: E|y|^2 per channel = 2 e^{sigma^2/2} (1 + delta).
    y, v0, S0 = sdev.mixture(4, 64, 2000, 0.05, 1.5, 9, "cpu")
    p = float((y.abs() ** 2).mean())
    expect = 2 * np.exp(1.5 ** 2 / 2) * 1.05
    assert abs(p / expect - 1) < 0.15
