"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, run the
oracle on the same seeded inputs, and measure the errors the tolerances are stated in.

Error metrics (median and max over all entries):
  v   per (j, n, f): |v - v*| / v*
  S   per (j, f):    ||S - S*||_F / ||S*||_F
  mu  per (j, n, f): ||mu - mu*||_2 / ||y(n, f)||_2  (mixture-normalised: mu1 + mu2 = y)
  ll  per iteration: |L - L*| / |L*|, L the log-likelihood of Eq. (like) summed over all bins
      (over the sampled bins when the oracle ran on a sample: bins are independent, so that
      sum is the log-likelihood of the sub-mixture made of those bins)
Tolerances: median <= 1e-4 and max <= 1e-3 for v, S, mu; 1e-6 for the log-likelihood.

Conditioning (check_conditioned): the bin arithmetic is FP32, so the GPU's result is at best the
exact result for a mixture perturbed at the level of FP32 rounding accumulated over the frames.
Where the EM problem itself amplifies such a perturbation beyond the max tolerance, no FP32 bin
arithmetic can meet it. A bin's response is measured on the FP64 oracle alone: the largest
relative change of its outputs (v, mu, S) when y is perturbed by a relative SENS_EPS
(oracle_response). Each bin is held to max(TOL_MAX, SENS_FACTOR x response): the fixed max, or
the change the exact EM shows under a perturbation of relative size SENS_FACTOR x SENS_EPS =
1e-5, whichever is larger. The bins where the second is larger (response > TOL_MAX /
SENS_FACTOR) are counted and reported; the medians and the log-likelihood keep the stated
tolerances over all bins.
"""
from __future__ import annotations

import numpy as np
import torch

TOL_MED, TOL_MAX, TOL_LL = 1e-4, 1e-3, 1e-6
SENS_EPS, SENS_FACTOR = 1e-7, 100.0
SENS_BOUND = TOL_MAX / SENS_FACTOR  # responses above this get the conditioning-scaled bound


def gpu_run(form, y, v0, S0, iters, y16=None, g=None, mode=0, host=False, want_S=True,
            precision=None, max_sweeps=30):
    """Run one EM on the GPU through the binding. y: complex64 numpy [F,N,M] (or None when
    y16/g are given); precision: None (the library default) or FCA_GEVD_FP32 / FCA_GEVD_FP64.
    Returns numpy arrays (v, S, mu1, mu2, ll, llf), the status code and the fused kernel's
    time (kernel_ms)."""
    from paper_1805_06572_gb300 import fca

    dev = torch.device("cuda")
    if y16 is not None:
        yt = torch.from_numpy(np.ascontiguousarray(y16))
        gt = torch.from_numpy(np.ascontiguousarray(g))
    else:
        yt = torch.from_numpy(np.ascontiguousarray(y, dtype=np.complex64))
        gt = None
    v0t = torch.from_numpy(np.ascontiguousarray(v0, dtype=np.float64))
    S0t = torch.from_numpy(np.ascontiguousarray(S0, dtype=np.complex128))
    if host:
        yt, v0t, S0t = yt.pin_memory(), v0t.pin_memory(), S0t.pin_memory()
        gt = gt.pin_memory() if gt is not None else None
    else:
        yt, v0t, S0t = yt.to(dev), v0t.to(dev), S0t.to(dev)
        gt = gt.to(dev) if gt is not None else None
    st = fca.fca_init(yt, v0t, S0t, y_scale=gt)
    assert precision is not None or max_sweeps == 30, "a sweep cap goes with a precision"
    if precision is not None:
        fca.fca_set_eigensolver(st, precision, max_sweeps)
    F, N, M = st.F, st.N, st.M
    ll = torch.empty(max(iters, 1), dtype=torch.float64, device=dev)
    if iters > 0:
        (fca.fca_em_fast if form == "fast" else fca.fca_em_conventional)(st, iters, ll)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, mode)
    v = torch.empty((2, F, N), dtype=torch.float32, device=dev)
    S = torch.empty((2, F, M, M), dtype=torch.complex128) if want_S else None
    fca.fca_get_params(st, v=v, S=S)
    code = fca.fca_sync_status(st)
    out = {"v": v.cpu().numpy().astype(np.float64), "mu1": x1.cpu().numpy(), "mu2": x2.cpu().numpy(),
           "ll": ll.cpu().numpy()[:iters], "status": code,
           "S": S.numpy() if S is not None else None}
    out["llf"] = fca.fca_loglik_bins(st).numpy().copy() if iters > 0 and code == 0 else None
    out["kernel_ms"] = fca.fca_last_em_kernel_ms(st) if iters > 0 and code == 0 else None
    fca.fca_free(st)
    return out


def errors(gpu, ref, y, fs=None):
    """Relative errors of a GPU result against an oracle result. fs: the frequencies the
    oracle ran on (a sample), or None for all."""
    sel = slice(None) if fs is None else fs
    v, vr = gpu["v"][:, sel], ref["v"]
    ev = np.abs(v - vr) / vr
    S, Sr = gpu["S"][:, sel], ref["S"]
    eS = np.linalg.norm(S - Sr, axis=(2, 3)) / np.linalg.norm(Sr, axis=(2, 3))
    yn = np.linalg.norm(np.asarray(y)[sel].astype(np.complex128), axis=2)
    yn = np.where(yn > 0, yn, 1.0)
    emu = np.stack([np.linalg.norm(gpu["mu1"][sel] - ref["mu1"], axis=2) / yn,
                    np.linalg.norm(gpu["mu2"][sel] - ref["mu2"], axis=2) / yn])
    out = {"v": (np.median(ev), ev.max()), "S": (np.median(eS), eS.max()),
           "mu": (np.median(emu), emu.max())}
    if fs is None:
        llr = ref["ll"].sum(axis=1)
        out["ll"] = np.max(np.abs(gpu["ll"] - llr) / np.abs(llr)) if len(llr) else 0.0
    elif gpu["llf"] is not None and len(ref["ll"]):
        llr = ref["ll"].sum(axis=1)
        llg = gpu["llf"][:, fs].sum(axis=1)
        out["ll"] = np.max(np.abs(llg - llr) / np.abs(llr))
    return out


def assert_within(err, label=""):
    for k in ("v", "S", "mu"):
        med, mx = err[k]
        assert med <= TOL_MED and mx <= TOL_MAX, f"{label} {k}: median {med:.3g} max {mx:.3g}"
    if "ll" in err:
        assert err["ll"] <= TOL_LL, f"{label} ll: {err['ll']:.3g}"


def bin_errors(gpu, ref, y, fs=None):
    """Per-bin maxima of the three error metrics ([F] each, over the bins the oracle ran on) and
    their medians over all entries."""
    sel = slice(None) if fs is None else fs
    ev = np.abs(gpu["v"][:, sel] - ref["v"]) / ref["v"]
    eS = np.linalg.norm(gpu["S"][:, sel] - ref["S"], axis=(2, 3)) / np.linalg.norm(ref["S"], axis=(2, 3))
    yn = np.linalg.norm(np.asarray(y)[sel].astype(np.complex128), axis=2)
    yn = np.where(yn > 0, yn, 1.0)
    emu = np.stack([np.linalg.norm(gpu["mu1"][sel] - ref["mu1"], axis=2) / yn,
                    np.linalg.norm(gpu["mu2"][sel] - ref["mu2"], axis=2) / yn])
    per_bin = {"v": ev.max(axis=(0, 2)), "S": eS.max(axis=0), "mu": emu.max(axis=(0, 2))}
    med = {"v": float(np.median(ev)), "S": float(np.median(eS)), "mu": float(np.median(emu))}
    return per_bin, med


def oracle_response(form, y, v0, S0, iters, ref=None, seed=5):
    """Per-bin response of the FP64 oracle to a relative SENS_EPS perturbation of the mixture:
    y -> y (1 + SENS_EPS g), g ~ CN(0, 1) per entry (seeded); returns the largest relative change
    of each bin's v, mu (per point, relative to |y|) and S ([F]). ref: the oracle's result on the
    unperturbed y, if already computed."""
    import oracle
    y = np.asarray(y, dtype=np.complex128)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)) / np.sqrt(2.0)
    r0 = ref if ref is not None else oracle.em(form, y, v0, S0, iters)
    r1 = oracle.em(form, y * (1.0 + SENS_EPS * g), v0, S0, iters)
    per_bin, _ = bin_errors({"v": r1["v"], "S": r1["S"], "mu1": r1["mu1"], "mu2": r1["mu2"]}, r0, y)
    return np.maximum(np.maximum(per_bin["v"], per_bin["mu"]), per_bin["S"])


def check_conditioned(gpu, ref, y, response, label="", fs=None):
    """The stated tolerances, with the conditioning rule of the module docstring. Returns the
    number of bins whose conditioning-scaled bound exceeds the fixed max."""
    per_bin, med = bin_errors(gpu, ref, y, fs=fs)
    scaled = response > SENS_BOUND
    bound = np.maximum(TOL_MAX, SENS_FACTOR * response)
    for k in ("v", "S", "mu"):
        assert med[k] <= TOL_MED, f"{label} {k}: median {med[k]:.3g}"
        worst = int(np.argmax(per_bin[k] / bound))
        assert per_bin[k][worst] <= bound[worst], \
            (f"{label} {k}: bin {worst} error {per_bin[k][worst]:.3g} > bound {bound[worst]:.3g} "
             f"(oracle response {response[worst]:.3g})")
    sel = slice(None) if fs is None else fs
    if fs is None:
        llr = ref["ll"].sum(axis=1)
        ell = np.max(np.abs(gpu["ll"] - llr) / np.abs(llr)) if len(llr) else 0.0
    else:
        llr = ref["ll"].sum(axis=1)
        ell = np.max(np.abs(gpu["llf"][:, sel].sum(axis=1) - llr) / np.abs(llr)) if len(llr) else 0.0
    assert ell <= TOL_LL, f"{label} ll: {ell:.3g}"
    return int(scaled.sum())
