"""fca_em_fast_noalloc: FastFCA for callers that must not allocate device memory.

Such callers -- a real-time audio loop, where cudaMalloc / cudaFree may stall the device, or
a host application that owns all device memory through its own pool -- pass their inputs
and outputs and get the same job as fca_init + fca_em_fast + fca_separate, with the
library's scratch in one fixed device array. Here two calls in a row (different shapes, so
the second runs on scratch the first left behind) are checked through the C ABI against
the allocating entry points: the same kernels on the same inputs, so the outputs must be
bitwise equal; the first call's outputs are also checked against the FP64 oracle at the
parity tolerances. This file is collected last so that a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

import synth

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

    import oracle
    from fca_testlib import assert_within, errors
    cases = [(3101, 4, 64, 300, 20), (3102, 2, 33, 517, 12)]
    for k, (seed, M, F, N, iters) in enumerate(cases):
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
        for name, a, b in (("v", v, rv), ("x1", x1, rx1), ("x2", x2, rx2), ("ll", ll, rll)):
            assert torch.equal(a, b), f"case {k}: {name} differs from the allocating path"
        if k == 0:
            r = oracle.em("fast", y, v0, S0, iters)
            got = {"v": v.cpu().numpy().astype(np.float64), "mu1": x1.cpu().numpy(),
                   "mu2": x2.cpu().numpy(), "ll": ll.cpu().numpy(), "S": r["S"]}
            assert_within(errors(got, r, y), "noalloc vs oracle")


def test_noalloc_rejects_misaligned_buffers(fca):
    """The buffers are read in place with 16-byte loads; a view one element into a buffer is
    refused on the host (FCA_ERR_ARG) before anything is enqueued."""
    import torch
    M, F, N, iters = 4, 8, 64, 3
    y, v0, S0 = _problem(3103, M, F, N)
    ybig = torch.zeros(F * N * M + 1, dtype=torch.complex64, device="cuda")
    ybig[1:] = torch.from_numpy(y).cuda().reshape(-1)
    yoff = ybig[1:].view(F, N, M)  # 8 bytes past a 256-byte boundary
    v0d = torch.from_numpy(v0).cuda()
    S0d = torch.from_numpy(S0).cuda()
    v = torch.empty((2, F, N), dtype=torch.float32, device="cuda")
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    launches = fca.fca_kernel_launches()
    assert fca.fca_em_fast_noalloc(yoff, v0d, S0d, iters, v, x1, x2) == 1  # FCA_ERR_ARG
    assert fca.fca_kernel_launches() == launches


def test_noalloc_rejects_problems_beyond_its_scratch(fca):
    import torch
    tiny = torch.zeros(1, dtype=torch.float32, device="cuda")
    # M=8, F=1025, N=4000 needs far more than the fixed scratch; rejected before any work.
    code = fca.lib.fca_em_fast_noalloc(8, 1025, 4000, fca._ptr(tiny), fca._ptr(tiny), fca._ptr(tiny),
                                       100, fca._ptr(tiny), fca._ptr(tiny), fca._ptr(tiny), None, None)
    assert code == 9  # FCA_ERR_SCRATCH
