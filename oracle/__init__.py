"""FP64 CPU oracle for two-source FCA EM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It is a plain complex128 C++ implementation of both forms of the EM
(conventional, Sec. 2; FastFCA, Sec. 3 and Algorithm 1) plus the Appendix's constructive
generalised eigendecomposition. It shares no code with the CUDA library.

Every function here is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``
(closed forms, library routines, invariants and brute force on tiny inputs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fca_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

STATUS = {0: "ok", 1: "bad argument", 2: "not positive definite",
          3: "eigensolver did not converge", 4: "singular matrix", 5: "non-finite value"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (OpenMP over frequencies if available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I, D = ctypes.c_int, ctypes.c_double
        lib.oracle_openmp_threads.restype = I
        lib.oracle_inverse.argtypes = [I, P, P, P]
        lib.oracle_herm_eig.argtypes = [I, P, P, P]
        lib.oracle_gevd.argtypes = [I, P, P, P, P]
        lib.oracle_estep_conventional.argtypes = [I, P, D, D, P, P, P, P, P, P, P]
        lib.oracle_estep_fast.argtypes = [I, P, D, D, P, P, P, P, P, P]
        lib.oracle_em.argtypes = [I, I, I, I, I, P, P, P, I, P, P, P, P, P, P, P, I]
        for f in ("oracle_inverse", "oracle_herm_eig", "oracle_gevd", "oracle_estep_conventional",
                  "oracle_estep_fast", "oracle_em"):
            getattr(lib, f).restype = I
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle status {rc}: {STATUS.get(rc, '?')}")


def threads() -> int:
    return _load().oracle_openmp_threads()


def inverse(A):
    A = _c128(A)
    M = A.shape[0]
    out = np.empty_like(A)
    ld = np.zeros(1)
    _check(_load().oracle_inverse(M, _p(A), _p(out), _p(ld)))
    return out, float(ld[0])


def herm_eig(A):
    A = _c128(A)
    M = A.shape[0]
    V = np.empty_like(A)
    w = np.empty(M)
    _check(_load().oracle_herm_eig(M, _p(A), _p(V), _p(w)))
    return V, w


def gevd(Phi, Psi):
    """P, lam with Phi P = Psi P diag(lam), P^H Psi P = I (Eq. (GEVD), Appendix Theorem)."""
    Phi, Psi = _c128(Phi), _c128(Psi)
    M = Phi.shape[0]
    P = np.empty_like(Phi)
    lam = np.empty(M)
    _check(_load().oracle_gevd(M, _p(Phi), _p(Psi), _p(P), _p(lam)))
    return P, lam


def estep_conventional(y, v1, v2, S1, S2):
    """One time-frequency point of Eqs. (MMSE), (postquadexp) and its Eq. (like) term."""
    y, S1, S2 = _c128(y), _c128(S1), _c128(S2)
    M = y.shape[0]
    mu1, mu2 = np.empty(M, np.complex128), np.empty(M, np.complex128)
    Phi1, Phi2 = np.empty((M, M), np.complex128), np.empty((M, M), np.complex128)
    ll = np.zeros(1)
    _check(_load().oracle_estep_conventional(M, _p(y), float(v1), float(v2), _p(S1), _p(S2),
                                             _p(mu1), _p(mu2), _p(Phi1), _p(Phi2), _p(ll)))
    return mu1, mu2, Phi1, Phi2, float(ll[0])


def estep_fast(y, v1, v2, P, lam):
    """One time-frequency point of Eqs. (MMSEtilde), (updatePhitildeeff)."""
    y, P, lam = _c128(y), _c128(P), _f64(lam)
    M = y.shape[0]
    m1, m2 = np.empty(M, np.complex128), np.empty(M, np.complex128)
    P1, P2 = np.empty((M, M), np.complex128), np.empty((M, M), np.complex128)
    _check(_load().oracle_estep_fast(M, _p(y), float(v1), float(v2), _p(P), _p(lam),
                                     _p(m1), _p(m2), _p(P1), _p(P2)))
    return m1, m2, P1, P2


def em(form: str, y, v0, S0, iters: int, sep_mode: int = 0, want_mu: bool = True,
       nthreads: int = 0):
    """Run L = iters EM iterations, form "conventional" or "fast".

    y [F][N][M] complex, v0 [2][F][N], S0 [2][F][M][M]. Returns a dict with v [2][F][N],
    S [2][F][M][M], ll [L][F] (log-likelihood at the parameters of each iteration), mu1, mu2
    [F][N][M] (posterior means; sep_mode 0 = Algorithm 1's output, 1 = final parameters) and,
    for the fast form, P [F][M][M], lam [F][M]."""
    fid = {"conventional": 0, "fast": 1}[form]
    y, v0, S0 = _c128(y), _f64(v0), _c128(S0)
    F, N, M = y.shape
    out = {"v": np.empty((2, F, N)), "S": np.empty((2, F, M, M), np.complex128),
           "ll": np.empty((iters, F))}
    mu1 = np.empty((F, N, M), np.complex128) if want_mu else None
    mu2 = np.empty((F, N, M), np.complex128) if want_mu else None
    P = np.empty((F, M, M), np.complex128) if fid == 1 else None
    lam = np.empty((F, M)) if fid == 1 else None
    rc = _load().oracle_em(fid, M, F, N, iters, _p(y), _p(v0), _p(S0), sep_mode, _p(out["v"]),
                           _p(out["S"]), _p(out["ll"]), _p(mu1), _p(mu2), _p(P), _p(lam),
                           nthreads)
    _check(rc)
    out.update(mu1=mu1, mu2=mu2)
    if fid == 1:
        out.update(P=P, lam=lam)
    return out
