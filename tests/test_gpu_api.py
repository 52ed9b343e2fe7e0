"""C-ABI behaviour on the GPU: form switching, status words, argument errors."""
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


def problem(seed=21, M=3, F=5, N=90):
    mix = synth.make_mixture(M, F, N, 0.1, 1.0, seed)
    v0, S0 = synth.init_params(mix["y"], seed)
    return mix["y"], v0, S0


def to_dev(y, v0, S0):
    d = torch.device("cuda")
    return (torch.from_numpy(y).to(d), torch.from_numpy(v0).to(d), torch.from_numpy(S0).to(d))


def test_switching_forms_midstream_follows_one_trajectory(fca):
    """FastFCA and conventional EM are the same iteration (Sec. 3), so 4 FastFCA iterations
    followed by 4 conventional ones equal 8 oracle iterations of either form."""
    y, v0, S0 = problem()
    F, N, M = y.shape
    st = fca.fca_init(*to_dev(y, v0, S0))
    fca.fca_em_fast(st, 4)
    fca.fca_em_conventional(st, 4)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
    v = torch.empty((2, F, N), dtype=torch.float32, device="cuda")
    S = torch.empty((2, F, M, M), dtype=torch.complex128)
    fca.fca_get_params(st, v=v, S=S)
    assert fca.fca_sync_status(st) == 0
    g = {"v": v.cpu().numpy().astype(np.float64), "S": S.numpy(), "mu1": x1.cpu().numpy(),
         "mu2": x2.cpu().numpy()}
    r = oracle.em("fast", y, v0, S0, 8)
    err = errors(dict(g, ll=np.zeros(0), llf=None), r, y, fs=np.arange(F))
    assert_within(err, "switch")
    # and back again: 3 more FastFCA iterations
    fca.fca_em_fast(st, 3)
    fca.fca_get_params(st, v=v, S=S)
    r = oracle.em("conventional", y, v0, S0, 11)
    g = {"v": v.cpu().numpy().astype(np.float64), "S": S.numpy(), "mu1": r["mu1"], "mu2": r["mu2"]}
    assert_within(errors(dict(g, ll=np.zeros(0), llf=None), r, y, fs=np.arange(F)), "switch back")


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_not_positive_definite_is_reported_and_latched(fca, form):
    y, v0, S0 = problem()
    S0 = S0.copy()
    S0[1, 2] = -np.eye(S0.shape[-1])
    st = fca.fca_init(*to_dev(y, v0, S0))
    (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, 3)
    assert fca.fca_sync_status(st) == 4  # FCA_ERR_NOT_PD
    with pytest.raises(fca.FCAError) as e:
        fca.fca_em_fast(st, 1)
    assert e.value.code == 8  # FCA_ERR_STATE
    y2, v2, S2 = problem()
    fca.fca_load(st, *to_dev(y2, v2, S2))
    fca.fca_em_fast(st, 2)
    assert fca.fca_sync_status(st) == 0


def test_nonfinite_initial_power_is_reported(fca):
    y, v0, S0 = problem()
    v0 = v0.copy()
    v0[0, 1, 3] = np.nan
    st = fca.fca_init(*to_dev(y, v0, S0))
    assert fca.fca_sync_status(st) == 6  # FCA_ERR_NONFINITE


def test_argument_errors_are_synchronous(fca):
    y, v0, S0 = problem()
    F, N, M = y.shape
    st = fca.fca_init(*to_dev(y, v0, S0))
    for call in (lambda: fca.fca_em_fast(st, -1), lambda: fca.fca_em_conventional(st, -2)):
        with pytest.raises(fca.FCAError) as e:
            call()
        assert e.value.code == 1
    x = torch.empty((F, N, M), dtype=torch.complex64, device="cuda")
    with pytest.raises(fca.FCAError):
        fca.fca_separate(st, x, x, 7)
    host = torch.empty((F, N, M), dtype=torch.complex64)
    with pytest.raises(fca.FCAError):
        fca.fca_separate(st, host, x, 0)
    with pytest.raises(fca.FCAError):  # shapes differ from the state's
        y2, v2, S2 = problem(M=2)
        fca.fca_load(st, *to_dev(y2, v2, S2))
    assert fca.fca_sync_status(st) == 0


def test_loglik_bins_sum_to_total(fca):
    y, v0, S0 = problem(F=9)
    st = fca.fca_init(*to_dev(y, v0, S0))
    ll = torch.empty(6, dtype=torch.float64, device="cuda")
    fca.fca_em_fast(st, 6, ll)
    llf = fca.fca_loglik_bins(st).numpy()
    assert llf.shape == (6, 9)
    np.testing.assert_allclose(llf.sum(axis=1), ll.cpu().numpy(), rtol=1e-14)
