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


def _state_outputs(fca, st, F, N, M):
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
    v = torch.empty((2, F, N), dtype=torch.float32, device="cuda")
    S = torch.empty((2, F, M, M), dtype=torch.complex128)
    fca.fca_get_params(st, v=v, S=S)
    assert fca.fca_sync_status(st) == 0
    return {"v": v.cpu().numpy().astype(np.float64), "S": S.numpy(), "mu1": x1.cpu().numpy(),
            "mu2": x2.cpu().numpy()}


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_resume_in_two_calls_equals_one_call(fca, form):
    """Checkpoint/resume: the state between calls is the EM state (v, and S or P, Lambda,
    log det S2), so 7 + 5 iterations continue the trajectory of 12 (conventional: bitwise, the
    FP64 S and FP32 v are exactly what the kernel keeps; FastFCA: the FP32 basis copy is
    rebuilt from the FP64 basis at a call boundary, so within rounding), and the separation of
    the second call is Algorithm 1's output of iteration 11."""
    y, v0, S0 = problem(seed=31, M=4, F=6, N=200)
    F, N, M = y.shape
    em = fca.fca_em_fast if form == "fast" else fca.fca_em_conventional
    a = fca.fca_init(*to_dev(y, v0, S0))
    em(a, 12)
    ga = _state_outputs(fca, a, F, N, M)
    b = fca.fca_init(*to_dev(y, v0, S0))
    em(b, 7)
    em(b, 5)
    gb = _state_outputs(fca, b, F, N, M)
    if form == "conventional":
        for k in ("v", "S", "mu1", "mu2"):
            assert np.array_equal(ga[k], gb[k]), k
    else:
        rel = np.abs(ga["v"] - gb["v"]) / ga["v"]
        assert np.median(rel) < 1e-5 and rel.max() < 1e-4
    r = oracle.em(form, y, v0, S0, 12)
    assert_within(errors(dict(gb, ll=np.zeros(0), llf=None), r, y, fs=np.arange(F)), "resume")


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_reload_with_fewer_frames(fca, form):
    """A state sized for N = 300 frames takes a mixture of 180 frames: the same results as a
    state made for 180 frames (bitwise)."""
    big = problem(seed=41, M=3, F=5, N=300)
    y, v0, S0 = problem(seed=42, M=3, F=5, N=180)
    em = fca.fca_em_fast if form == "fast" else fca.fca_em_conventional
    st = fca.fca_init(*to_dev(*big))
    fca.fca_load(st, *to_dev(y, v0, S0))
    assert st.N == 300  # the binding keeps the creation shape; the library tracks the load
    em(st, 6)
    x1 = torch.empty((5, 180, 3), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2)
    assert fca.fca_sync_status(st) == 0
    fresh = fca.fca_init(*to_dev(y, v0, S0))
    em(fresh, 6)
    y1 = torch.empty_like(x1)
    y2 = torch.empty_like(x1)
    fca.fca_separate(fresh, y1, y2)
    assert torch.equal(x1, y1) and torch.equal(x2, y2)
    with pytest.raises(fca.FCAError):  # more frames than the state holds
        fca.fca_load(fresh, *to_dev(*big))


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_nan_in_the_mixture_is_reported_and_latched(fca, form):
    y, v0, S0 = problem(seed=51)
    y = y.copy()
    y[2, 10, 1] = np.nan
    em = fca.fca_em_fast if form == "fast" else fca.fca_em_conventional
    st = fca.fca_init(*to_dev(y, v0, S0))
    em(st, 3)
    assert fca.fca_sync_status(st) == 6  # FCA_ERR_NONFINITE
    with pytest.raises(fca.FCAError) as ei:
        em(st, 1)
    assert ei.value.code == 8  # FCA_ERR_STATE until the state is reloaded
    yc, v0c, S0c = problem(seed=51)
    fca.fca_load(st, *to_dev(yc, v0c, S0c))
    em(st, 3)
    assert fca.fca_sync_status(st) == 0


@pytest.mark.parametrize("form,M", [("fast", 4), ("fast", 3), ("conventional", 4)])
def test_results_do_not_depend_on_input_alignment(fca, form, M):
    """The load pass reads device inputs in place (16-byte loads where the addresses allow,
    element by element otherwise, in one summation order either way), and falls back to a
    copy for inputs not aligned to their element. Views offset by one element give bitwise
    the results of aligned inputs."""
    y, v0, S0 = problem(seed=33, M=M, F=6, N=301)  # M = 3: an odd count of values per bin
    F, N, M = y.shape
    d = torch.device("cuda")

    def offset_view(a, dtype):
        t = torch.empty(a.size + 1, dtype=dtype, device=d)
        t[1:] = torch.from_numpy(a.ravel()).to(d)
        return t[1:].view(a.shape)

    def run(yd, vd, Sd):
        st = fca.fca_init(yd, vd, Sd)
        ll = torch.empty(5, dtype=torch.float64, device=d)
        (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, 5, ll)
        x1 = torch.empty((F, N, M), dtype=torch.complex64, device=d)
        x2 = torch.empty_like(x1)
        fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
        v = torch.empty((2, F, N), dtype=torch.float32, device=d)
        fca.fca_get_params(st, v=v)
        assert fca.fca_sync_status(st) == 0
        out = [t.cpu().numpy() for t in (x1, x2, v, ll)]
        fca.fca_free(st)
        return out

    ref = run(*to_dev(y, v0, S0))
    got = run(offset_view(y, torch.complex64), offset_view(v0, torch.float64),
              offset_view(S0, torch.complex128))
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sweep_cap_of_zero_reports_nonconvergence(fca, mode):
    """A Jacobi sweep cap of 0 set from the host: the eigenproblem of S0, solved again with the
    new settings at the next fca_em_fast, stops at once and records FCA_ERR_EIG_NOCONV (5) in
    the status word; the kernels return (nothing waits), the state latches until it is
    reloaded, and the default cap works again afterwards. Every precision mode."""
    y, v0, S0 = problem(seed=61, M=4, F=6, N=120)
    st = fca.fca_init(*to_dev(y, v0, S0))
    fca.fca_set_eigensolver(st, mode, 0)
    fca.fca_em_fast(st, 3)
    assert fca.fca_sync_status(st) == 5  # FCA_ERR_EIG_NOCONV
    with pytest.raises(fca.FCAError) as e:
        fca.fca_em_fast(st, 1)
    assert e.value.code == 8  # FCA_ERR_STATE
    fca.fca_set_eigensolver(st, mode, 30)
    fca.fca_load(st, *to_dev(y, v0, S0))
    fca.fca_em_fast(st, 3)
    assert fca.fca_sync_status(st) == 0


def test_eigensolver_settings_are_checked(fca):
    y, v0, S0 = problem()
    st = fca.fca_init(*to_dev(y, v0, S0))
    for prec, sweeps in ((3, 30), (-1, 30), (0, -1), (2, fca.FCA_MAX_SWEEPS_LIMIT + 1)):
        with pytest.raises(fca.FCAError) as e:
            fca.fca_set_eigensolver(st, prec, sweeps)
        assert e.value.code == 1
    fca.fca_set_eigensolver(st, fca.FCA_GEVD_FP64, 12)
    fca.fca_em_fast(st, 2)
    assert fca.fca_sync_status(st) == 0


def test_modes_agree_with_each_other(fca):
    """The three eigensolver precisions run the same iteration: their results agree to well
    within the parity tolerances on a well-conditioned problem."""
    y, v0, S0 = problem(seed=71, M=4, F=12, N=400)
    F, N, M = y.shape
    outs = []
    for mode in (0, 1, 2):
        st = fca.fca_init(*to_dev(y, v0, S0))
        fca.fca_set_eigensolver(st, mode, 30)
        fca.fca_em_fast(st, 10)
        outs.append(_state_outputs(fca, st, F, N, M))
    for o in outs[:2]:
        rel = np.abs(o["v"] - outs[2]["v"]) / outs[2]["v"]
        assert np.median(rel) < 1e-5 and rel.max() < 1e-3
