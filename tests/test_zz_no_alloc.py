"""fca_em_fast_noalloc: FastFCA for callers that must not allocate device memory.

Such callers -- a real-time audio loop, where cudaMalloc / cudaFree may stall the device, or
a host application that owns all device memory through its own pool -- pass their inputs
and outputs and get the same job as fca_init + fca_em_fast + fca_separate, with the
library's scratch in one fixed device array. Here two calls in a row (different shapes, so
the second runs on scratch the first left behind) are checked through the C ABI against
the allocating entry points at the tolerances of the parity tests. This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import synth
from fca_testlib import TOL_LL, TOL_MAX, TOL_MED

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fca():
    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca as mod
    return mod


def _problem(seed, M, F, N):
    mix = synth.make_mixture(M, F, N, 0.05, 1.5, seed)
    v0, S0 = synth.init_params(mix["y"], seed, x=mix["x"])
    return mix["y"], v0, S0


def _allocating(fca, torch, y, v0, S0, iters):
    st = fca.fca_init(y, v0, S0)
    F, N, M = st.F, st.N, st.M
    ll = torch.empty(iters, dtype=torch.float64, device="cuda")
    fca.fca_em_fast(st, iters, ll)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
    v = torch.empty((2, F, N), dtype=torch.float32, device="cuda")
    fca.fca_get_params(st, v=v)
    assert fca.fca_sync_status(st) == 0
    fca.fca_free(st)
    return v, x1, x2, ll


def test_noalloc_matches_allocating_path_twice_in_a_row(fca):
    import torch
    cases = [(3101, 4, 64, 300, 20), (3102, 2, 33, 517, 12)]
    for seed, M, F, N, iters in cases:
        y, v0, S0 = _problem(seed, M, F, N)
        yd = torch.from_numpy(y).cuda()
        v0d = torch.from_numpy(v0).cuda()
        S0d = torch.from_numpy(S0).cuda()
        v = torch.full((2, F, N), float("nan"), dtype=torch.float32, device="cuda")
        x1 = torch.full((F, N, M), float("nan"), dtype=torch.complex64, device="cuda")
        x2 = torch.full_like(x1, float("nan"))
        ll = torch.full((iters,), float("nan"), dtype=torch.float64, device="cuda")
        code = fca.fca_em_fast_noalloc(yd, v0d, S0d, iters, v, x1, x2, ll)
        assert code == 0, fca.fca_status_string(code)
        rv, rx1, rx2, rll = _allocating(fca, torch, yd, v0d, S0d, iters)
        ev = (torch.abs(v - rv) / rv).cpu().numpy()
        yn = torch.linalg.vector_norm(yd, dim=2).clamp_min(1e-30)
        emu = torch.stack([torch.linalg.vector_norm(x1 - rx1, dim=2) / yn,
                           torch.linalg.vector_norm(x2 - rx2, dim=2) / yn]).cpu().numpy()
        ell = (torch.abs(ll - rll) / torch.abs(rll)).cpu().numpy()
        for name, e in (("v", ev), ("mu", emu)):
            assert np.median(e) <= TOL_MED and e.max() <= TOL_MAX, (name, np.median(e), e.max())
        assert ell.max() <= TOL_LL


def test_noalloc_rejects_problems_beyond_its_scratch(fca):
    import torch
    tiny = torch.zeros(1, dtype=torch.float32, device="cuda")
    # M=8, F=1025, N=4000 needs far more than the fixed scratch; rejected before any work.
    code = fca.lib.fca_em_fast_noalloc(8, 1025, 4000, fca._ptr(tiny), fca._ptr(tiny), fca._ptr(tiny),
                                       100, fca._ptr(tiny), fca._ptr(tiny), fca._ptr(tiny), None, None)
    assert code == 9  # FCA_ERR_SCRATCH
