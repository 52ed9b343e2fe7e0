"""STFT front-end (fca_stft / fca_istft through the C ABI, GPU only) against the STFT oracle,
and the whole time-domain pipeline: STFT -> EM -> posterior means -> inverse STFT."""
import numpy as np
import pytest

import oracle
import synth
from fca_testlib import assert_within, errors
from oracle import stft as ost

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca
    return fca, torch


@pytest.mark.parametrize("W,H,T,M", [(1024, 512, 16000, 4), (64, 32, 3001, 2), (256, 64, 5000, 3),
                                     (16, 8, 40, 1)])
def test_stft_matches_oracle(env, W, H, T, M):
    fca, torch = env
    x, _ = synth.make_time_mixture(M, T, 11)
    y = fca.fca_stft(torch.from_numpy(x.astype(np.float32)).cuda(), W, H).cpu().numpy()
    r = ost.stft(x.astype(np.float32).astype(np.float64), W, H)
    assert y.shape == r.shape
    # error per frame relative to the frame's spectral norm (FP32 FFT of length W/2)
    err = np.linalg.norm(y - r, axis=0) / np.maximum(np.linalg.norm(r, axis=0), 1e-30)
    assert err.max() < 2e-6, err.max()


@pytest.mark.parametrize("W,H", [(1024, 512), (64, 16)])
def test_istft_matches_oracle_and_inverts(env, W, H):
    fca, torch = env
    M, T = 3, 9000
    x, _ = synth.make_time_mixture(M, T, 12)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    y = fca.fca_stft(xd, W, H)
    back = fca.fca_istft(y, T, W, H).cpu().numpy()
    assert np.max(np.abs(back - x.astype(np.float32))) < 1e-5 * np.max(np.abs(x))
    # an arbitrary (non-Hermitian-consistent) spectrum: same result as the oracle
    rng = np.random.default_rng(3)
    z = (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)).astype(np.complex64)
    g = fca.fca_istft(torch.from_numpy(z).cuda(), T, W, H).cpu().numpy()
    r = ost.istft(z.astype(np.complex128), T, W, H)
    assert np.max(np.abs(g - r)) < 2e-6 * np.max(np.abs(r))
    g2 = fca.fca_istft(torch.from_numpy(z).cuda(), T, W, H).cpu().numpy()
    assert np.array_equal(g, g2)  # fixed-order overlap-add


def test_time_domain_pipeline(env):
    """A 2-source, 4-microphone convolutive mixture (1 s at 16 kHz) through Table 1's analysis,
    20 FastFCA iterations and the synthesis: the separated signals sum to the mixture, and
    match the oracle pipeline (oracle STFT, oracle EM, oracle inverse STFT)."""
    fca, torch = env
    M, T, W, H, L = 4, 16000, 1024, 512, 20
    y_t, _ = synth.make_time_mixture(M, T, 21)
    y_t = y_t.astype(np.float32)
    Y = fca.fca_stft(torch.from_numpy(y_t).cuda(), W, H)
    Yh = Y.cpu().numpy()
    v0, S0 = synth.init_params(Yh, 21, recipe="random")
    st = fca.fca_init(Y, torch.from_numpy(v0).cuda(), torch.from_numpy(S0).cuda())
    fca.fca_em_fast(st, L)
    x1 = torch.empty_like(Y)
    x2 = torch.empty_like(Y)
    fca.fca_separate(st, x1, x2)
    assert fca.fca_sync_status(st) == 0
    s1 = fca.fca_istft(x1, T, W, H).cpu().numpy()
    s2 = fca.fca_istft(x2, T, W, H).cpu().numpy()
    assert np.max(np.abs(s1 + s2 - y_t)) < 1e-5 * np.max(np.abs(y_t))
    # oracle pipeline on the same time-domain input
    Yr = ost.stft(y_t.astype(np.float64), W, H)
    r = oracle.em("fast", Yr, v0, S0, L)
    r1 = ost.istft(r["mu1"], T, W, H)
    e = np.linalg.norm(s1 - r1) / np.linalg.norm(r1)
    assert e < 1e-4, e
    # and the frequency-domain outputs at the parity tolerances
    got = {"mu1": x1.cpu().numpy(), "mu2": x2.cpu().numpy(), "v": r["v"], "S": r["S"],
           "ll": r["ll"].sum(axis=1)}
    err = errors(got, r, Yr)
    err.pop("ll")
    assert_within(err, "pipeline")
    fca.fca_free(st)


def test_stft_rejects_bad_shapes(env):
    fca, torch = env
    x = torch.zeros((2, 100), dtype=torch.float32, device="cuda")
    for W, H in ((1000, 500), (8, 4), (64, 33), (64, 0)):
        with pytest.raises(fca.FCAError):
            fca.fca_stft(x, W, H)
