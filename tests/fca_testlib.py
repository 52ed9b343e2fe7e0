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
"""
from __future__ import annotations

import numpy as np
import torch

TOL_MED, TOL_MAX, TOL_LL = 1e-4, 1e-3, 1e-6


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
