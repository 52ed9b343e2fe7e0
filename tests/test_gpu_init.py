"""Inputs the library builds on the device (through the C ABI): the seeded initial values of a
problem given without v0 and S0, against the host recipe in synth (the same counter-based
draws), and EM runs from them against the oracle run from the host recipe; the FP16 encoding of
a complex64 device mixture, bitwise against synth.quantize_f16."""
import numpy as np
import pytest
import torch

import oracle
import synth
from fca_testlib import assert_within, errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fca():
    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca as mod
    return mod


def _read(fca, st):
    v = torch.empty((2, st.F, st.N), dtype=torch.float32, device="cuda")
    S = torch.empty((2, st.F, st.M, st.M), dtype=torch.complex128)
    fca.fca_get_params(st, v=v, S=S)
    assert fca.fca_sync_status(st) == 0
    return v.cpu().numpy().astype(np.float64), S.numpy()


def _vfloor(yd):
    return np.maximum(1e-12 * np.mean(np.abs(yd) ** 2, axis=(1, 2)), 1e-30)


@pytest.mark.parametrize("M,F,N", [(1, 3, 40), (2, 17, 301), (4, 9, 1000), (8, 5, 77)])
@pytest.mark.parametrize("location", ["device", "host"])
def test_seeded_initial_values_match_the_host_recipe(fca, M, F, N, location):
    seed = 900 + 10 * M + F
    y = synth.make_mixture(M, F, N, 0.1, 1.0, seed)["y"]
    v0, S0 = synth.init_params(y, seed, recipe="random")
    yt = torch.from_numpy(y)
    yt = yt.cuda() if location == "device" else yt.pin_memory()
    st = fca.fca_init(yt, seed=seed)
    v, S = _read(fca, st)
    np.testing.assert_allclose(S, S0, rtol=1e-13, atol=1e-13)
    want = np.maximum(v0.astype(np.float32), _vfloor(y.astype(np.complex128)).astype(np.float32)[None, :, None])
    np.testing.assert_allclose(v, want, rtol=2e-7)
    # a reload with another seed draws other values; the same seed the same ones
    fca.fca_load(st, yt, seed=seed + 1)
    _, S1 = _read(fca, st)
    assert np.abs(S1 - S0).max() > 1e-3
    fca.fca_load(st, yt, seed=seed)
    _, S2 = _read(fca, st)
    np.testing.assert_array_equal(S2, S)


def test_seeded_initial_values_from_an_fp16_mixture(fca):
    M, F, N, seed = 4, 11, 257, 31337
    y = synth.make_mixture(M, F, N, 0.05, 1.5, seed)["y"]
    y16, g, deq = synth.quantize_f16(y)
    v0, S0 = synth.init_params(deq, seed, recipe="random")
    for kw in (dict(y=torch.from_numpy(y16).cuda(), y_scale=torch.from_numpy(g).cuda()),
               dict(y=torch.from_numpy(y).cuda(), encode_f16=True)):
        st = fca.fca_init(kw.pop("y"), seed=seed, **kw)
        v, S = _read(fca, st)
        np.testing.assert_allclose(S, S0, rtol=1e-13, atol=1e-13)
        want = np.maximum(v0.astype(np.float32), _vfloor(deq).astype(np.float32)[None, :, None])
        np.testing.assert_allclose(v, want, rtol=2e-7)


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_em_from_the_seeded_initial_values_matches_the_oracle(fca, form):
    # the small workload's shape (M = 2, N = 300, L = 20) on 64 of its bins
    c = synth.CONFIGS["small"]
    seed = synth.config_seed("small")
    F = 64
    y = synth.make_mixture(c.M, F, c.N, c.delta, c.sigma, seed)["y"]
    v0, S0 = synth.init_params(y, seed, recipe="random")
    r = oracle.em(form, y, v0, S0, c.iters)
    st = fca.fca_init(torch.from_numpy(y).cuda(), seed=seed)
    ll = torch.empty(c.iters, dtype=torch.float64, device="cuda")
    (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, c.iters, ll)
    x1 = torch.empty((F, c.N, c.M), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
    v, S = _read(fca, st)
    got = {"v": v, "S": S, "mu1": x1.cpu().numpy(), "mu2": x2.cpu().numpy(), "ll": ll.cpu().numpy()}
    assert_within(errors(got, r, y), form)


@pytest.mark.parametrize("M,F,N", [(2, 7, 129), (4, 40, 333), (8, 3, 1000)])
def test_fp16_encoding_on_the_device_is_the_host_encoding_bitwise(fca, M, F, N):
    """A state loaded with the complex64 mixture and on-device encoding runs bit for bit as one
    loaded with synth.quantize_f16's FP16 values and scales (deterministic kernels, same
    inputs), so any difference in a single stored value or scale shows in the outputs."""
    seed = 4000 + M
    y = synth.make_mixture(M, F, N, 0.05, 1.5, seed)["y"]
    y[0, :5] *= 1e-3  # a few quiet frames: small FP16 values
    y16, g, _ = synth.quantize_f16(y)
    v0, S0 = synth.init_params(y, seed, recipe="random")
    d = torch.device("cuda")
    v0t, S0t = torch.from_numpy(v0).to(d), torch.from_numpy(S0).to(d)
    outs = []
    for kw in (dict(y=torch.from_numpy(y16).to(d), y_scale=torch.from_numpy(g).to(d)),
               dict(y=torch.from_numpy(y).to(d), encode_f16=True)):
        st = fca.fca_init(kw.pop("y"), v0t, S0t, **kw)
        ll = torch.empty(4, dtype=torch.float64, device=d)
        fca.fca_em_fast(st, 4, ll)
        x1 = torch.empty((F, N, M), dtype=torch.complex64, device=d)
        x2 = torch.empty_like(x1)
        fca.fca_separate(st, x1, x2, fca.FCA_SEP_FINAL_PARAMS)
        v, S = _read(fca, st)
        outs.append((ll.cpu().numpy(), v, S, x1.cpu().numpy(), x2.cpu().numpy()))
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_fp16_encoding_needs_a_device_mixture(fca):
    y = synth.make_mixture(2, 3, 10, 0.1, 1.0, 5)["y"]
    with pytest.raises(ValueError):
        fca.fca_init(torch.from_numpy(y), encode_f16=True)
    with pytest.raises(ValueError):
        fca.fca_init(torch.from_numpy(y).cuda(), v0=torch.zeros(2, 3, 10, dtype=torch.float64).cuda())
