"""Batches of mixtures with uneven M and N (fca_batch_* through the C ABI, GPU only).

Every bin of every mixture is an independent EM problem, so a mixture's results in a batch
must be those of the one-mixture entry points: bitwise for the default launch shape (the same
kernels and reduction order), and within the parity tolerances of the FP64 oracle for any
tuned shape. The mix covers odd M (the library pads its copy of y to 16-byte boundaries),
bins that stay on chip and bins that stream (N = 4500 at M = 2), and a single-frame mixture.
"""
import numpy as np
import pytest

import oracle
import synth
from fca_testlib import assert_within, errors, gpu_run

pytestmark = pytest.mark.gpu

MIXES = [(2, 7, 300), (4, 5, 37), (3, 6, 129), (1, 4, 50), (6, 3, 611), (8, 2, 200),
         (4, 9, 1000), (2, 3, 4500), (5, 3, 77), (7, 2, 1)]


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca
    assert torch.cuda.is_available()
    mixes = []
    for i, (M, F, N) in enumerate(MIXES):
        mix = synth.make_mixture(M, F, N, 0.05, 1.5, 4000 + i)
        v0, S0 = synth.init_params(mix["y"], 4000 + i, x=mix["x"])
        mixes.append((mix["y"], v0, S0))
    return fca, torch, mixes


def _pack(torch, mixes, device="cuda"):
    y = torch.from_numpy(np.concatenate([m[0].ravel() for m in mixes]).astype(np.complex64))
    v0 = torch.from_numpy(np.concatenate([m[1].ravel() for m in mixes]))
    S0 = torch.from_numpy(np.concatenate([m[2].ravel() for m in mixes]))
    return y.to(device), v0.to(device), S0.to(device)


def _run(fca, torch, b, form, iters, graph=False):
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    v = torch.empty(b.v_elems, dtype=torch.float32, device="cuda")
    ll = torch.empty(max(b.count * iters, 1), dtype=torch.float64, device="cuda")
    fca.fca_batch_run(b, form, iters, x1, x2, loglik=ll if iters else None, v=v, use_graph=graph)
    assert fca.fca_batch_sync_status(b) == 0
    return x1.cpu().numpy(), x2.cpu().numpy(), v.cpu().numpy(), ll.cpu().numpy()[:b.count * iters]


def _unpack(b, k, x1, x2, v, ll, iters):
    M, F, N = b.M[k], b.F[k], b.N[k]
    xo, vo = int(b.x_off[k]), int(b.v_off[k])
    return {"mu1": x1[xo:xo + F * N * M].reshape(F, N, M), "mu2": x2[xo:xo + F * N * M].reshape(F, N, M),
            "v": v[vo:vo + 2 * F * N].reshape(2, F, N).astype(np.float64),
            "ll": ll[k * iters:(k + 1) * iters]}


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_batch_equals_one_mixture_runs(env, form):
    fca, torch, mixes = env
    iters = 7
    b = fca.fca_batch_init([m[0].shape[2] for m in mixes], [m[0].shape[0] for m in mixes],
                           [m[0].shape[1] for m in mixes], *_pack(torch, mixes))
    fid = fca.FCA_FORM_FAST if form == "fast" else fca.FCA_FORM_CONVENTIONAL
    out = _run(fca, torch, b, fid, iters)
    for k, (y, v0, S0) in enumerate(mixes):
        got = _unpack(b, k, *out, iters)
        ref = gpu_run(form, y, v0, S0, iters, want_S=False)
        assert ref["status"] == 0
        for key in ("v", "mu1", "mu2"):
            assert np.array_equal(got[key], ref[key]), (k, key)
        np.testing.assert_allclose(got["ll"], ref["ll"], rtol=1e-12, atol=0)
    fca.fca_batch_free(b)


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_tuned_batch_matches_oracle(env, form):
    fca, torch, mixes = env
    iters = 12
    b = fca.fca_batch_init([m[0].shape[2] for m in mixes], [m[0].shape[0] for m in mixes],
                           [m[0].shape[1] for m in mixes], *_pack(torch, mixes))
    fca.fca_batch_tune(b, iters)
    for M in sorted(set(b.M)):
        bins, threads, res = fca.fca_batch_shape(b, M)
        assert threads in (64, 128, 256) and bins == sum(F for m, F in zip(b.M, b.F) if m == M)
    fid = fca.FCA_FORM_FAST if form == "fast" else fca.FCA_FORM_CONVENTIONAL
    out = _run(fca, torch, b, fid, iters)
    short = [k for k in range(len(mixes)) if b.N[k] < 8]
    for k, (y, v0, S0) in enumerate(mixes):
        if form == "conventional" and k in short:
            continue  # checked at 3 iterations below
        got = _unpack(b, k, *out, iters)
        r = oracle.em(form, y, v0, S0, iters)
        got["S"] = fca.fca_batch_get_params(b, k)[0].numpy()
        assert_within(errors(got, r, y), f"mixture {k} {b.M[k]}x{b.F[k]}x{b.N[k]}")
    if form == "conventional":
        # One frame makes the conventional M-step's S_j the rank-one term plus the shared
        # posterior covariance, whose conditioning outgrows the tolerance over 12 FP32
        # iterations; the single-frame mixture is compared at 2 iterations (the tuned shapes
        # stay).
        out = _run(fca, torch, b, fid, 2)
        for k in short:
            y, v0, S0 = mixes[k]
            got = _unpack(b, k, *out, 2)
            r = oracle.em(form, y, v0, S0, 2)
            got["S"] = fca.fca_batch_get_params(b, k)[0].numpy()
            assert_within(errors(got, r, y), f"mixture {k} at 2 iterations")
    fca.fca_batch_free(b)


def test_graph_replay_is_bitwise_and_repeatable(env):
    fca, torch, mixes = env
    b = fca.fca_batch_init([m[0].shape[2] for m in mixes], [m[0].shape[0] for m in mixes],
                           [m[0].shape[1] for m in mixes], *_pack(torch, mixes))
    plain = _run(fca, torch, b, fca.FCA_FORM_FAST, 5)
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    v = torch.empty(b.v_elems, dtype=torch.float32, device="cuda")
    ll = torch.empty(b.count * 5, dtype=torch.float64, device="cuda")
    reps = []
    launches0 = fca.fca_kernel_launches()
    for _ in range(3):
        x1.zero_()
        fca.fca_batch_run(b, fca.FCA_FORM_FAST, 5, x1, x2, loglik=ll, v=v, use_graph=True)
        assert fca.fca_batch_sync_status(b) == 0
        reps.append([t.cpu().numpy() for t in (x1, x2, v, ll)])
    assert fca.fca_kernel_launches() - launches0 >= 3 * 4 * len(set(b.M))
    for r in reps:
        for a, c in zip(r, plain):
            assert np.array_equal(a, c)
    fca.fca_batch_free(b)


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_zero_iterations_uses_initial_parameters(env, form):
    fca, torch, mixes = env
    sub = mixes[:4]
    b = fca.fca_batch_init([m[0].shape[2] for m in sub], [m[0].shape[0] for m in sub],
                           [m[0].shape[1] for m in sub], *_pack(torch, sub))
    fid = fca.FCA_FORM_FAST if form == "fast" else fca.FCA_FORM_CONVENTIONAL
    out = _run(fca, torch, b, fid, 0)
    for k, (y, v0, S0) in enumerate(sub):
        got = _unpack(b, k, *out, 0)
        r = oracle.em(form, y, v0, S0, 0)
        got["S"] = fca.fca_batch_get_params(b, k)[0].numpy()
        err = errors(got, r, y)
        err.pop("ll")
        assert_within(err, f"mixture {k}")
    fca.fca_batch_free(b)


def test_host_inputs_and_reload(env):
    fca, torch, mixes = env
    sub = mixes[:5]
    dims = ([m[0].shape[2] for m in sub], [m[0].shape[0] for m in sub], [m[0].shape[1] for m in sub])
    yh, v0h, S0h = (t.pin_memory() for t in _pack(torch, sub, device="cpu"))
    b = fca.fca_batch_init(*dims, yh, v0h, S0h)
    a = _run(fca, torch, b, fca.FCA_FORM_FAST, 4)
    fca.fca_batch_load(b, *_pack(torch, sub))
    c = _run(fca, torch, b, fca.FCA_FORM_FAST, 4)
    for p, q in zip(a, c):
        assert np.array_equal(p, q)
    fca.fca_batch_free(b)


def test_set_shape_reuses_shapes_and_keeps_parity(env):
    """Shapes set by hand (64 threads, nothing on chip; 256 threads, everything that fits on
    chip) give results within the parity tolerances of the oracle."""
    fca, torch, mixes = env
    sub = mixes[:6]
    b = fca.fca_batch_init([m[0].shape[2] for m in sub], [m[0].shape[0] for m in sub],
                           [m[0].shape[1] for m in sub], *_pack(torch, sub))
    for prec, threads, res in ((fca.FCA_GEVD_FP32, 64, 0), (fca.FCA_GEVD_REFINED, 128, 0),
                               (fca.FCA_GEVD_REFINED, 256, 200 * 1024)):
        fca.fca_batch_set_eigensolver(b, prec)
        for M in sorted(set(b.M)):
            fca.fca_batch_set_shape(b, M, threads, res)
            assert fca.fca_batch_shape(b, M)[1:] == (threads, res)
        out = _run(fca, torch, b, fca.FCA_FORM_FAST, 6, graph=True)
        for k, (y, v0, S0) in enumerate(sub):
            got = _unpack(b, k, *out, 6)
            r = oracle.em("fast", y, v0, S0, 6)
            got["S"] = fca.fca_batch_get_params(b, k)[0].numpy()
            assert_within(errors(got, r, y), f"mixture {k} threads {threads}")
    with pytest.raises(fca.FCAError):  # the refined mode needs three warps per CTA
        fca.fca_batch_set_shape(b, b.M[0], 64, 0)
    absent = next(m for m in range(1, 9) if m not in b.M)
    with pytest.raises(fca.FCAError):
        fca.fca_batch_set_shape(b, absent, 128, 0)
    with pytest.raises(fca.FCAError):
        fca.fca_batch_set_shape(b, b.M[0], 96, 0)
    fca.fca_batch_free(b)


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_equals_one_mixture_runs_in_each_precision(env, prec):
    """The batch in each of its eigensolver precisions (FP32, refined) gives bitwise the
    one-mixture results in the same precision."""
    fca, torch, mixes = env
    iters = 5
    b = fca.fca_batch_init([m[0].shape[2] for m in mixes], [m[0].shape[0] for m in mixes],
                           [m[0].shape[1] for m in mixes], *_pack(torch, mixes))
    fca.fca_batch_set_eigensolver(b, prec)
    out = _run(fca, torch, b, fca.FCA_FORM_FAST, iters)
    for k, (y, v0, S0) in enumerate(mixes):
        got = _unpack(b, k, *out, iters)
        ref = gpu_run("fast", y, v0, S0, iters, want_S=False, precision=prec)
        for key in ("v", "mu1", "mu2"):
            assert np.array_equal(got[key], ref[key]), (k, key)
    fca.fca_batch_free(b)


def test_batch_sweep_cap_of_zero_reports_nonconvergence(env):
    fca, torch, mixes = env
    sub = mixes[:3]
    b = fca.fca_batch_init([m[0].shape[2] for m in sub], [m[0].shape[0] for m in sub],
                           [m[0].shape[1] for m in sub], *_pack(torch, sub))
    fca.fca_batch_set_eigensolver(b, fca.FCA_GEVD_FP32, 0)
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    fca.fca_batch_run(b, fca.FCA_FORM_FAST, 3, x1, x2)
    assert fca.fca_batch_sync_status(b) == 5  # FCA_ERR_EIG_NOCONV
    fca.fca_batch_free(b)
