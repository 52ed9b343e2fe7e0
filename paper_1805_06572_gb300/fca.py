"""Thin ctypes binding of libfca.so (include/fca.h), same names as the C ABI.

Argument marshalling only: every step of the EM runs in the library's CUDA kernels. Tensors
are torch tensors (device tensors, or host tensors -- pinned for asynchronous copies); the
binding passes their data pointers and the CUDA stream handle. If the compiled library is
missing this module raises at import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfca.so")

FCA_OK = 0
FCA_STORE_C64, FCA_STORE_F16_SCALED = 0, 1
FCA_MEM_DEVICE, FCA_MEM_HOST = 0, 1
FCA_SEP_ALG1, FCA_SEP_FINAL_PARAMS = 0, 1
FCA_FORM_FAST, FCA_FORM_CONVENTIONAL = 0, 1
FCA_GEVD_FP32, FCA_GEVD_FP64, FCA_GEVD_REFINED = 0, 1, 2
FCA_GEVD_DEFAULT = FCA_GEVD_REFINED
FCA_CONV_AUTO, FCA_CONV_THREAD, FCA_CONV_GROUP = 0, 1, 2
FCA_MAX_SWEEPS_LIMIT = 1000
STATUS_NAMES = {0: "FCA_OK", 1: "FCA_ERR_ARG", 2: "FCA_ERR_CUDA", 3: "FCA_ERR_NOMEM",
                4: "FCA_ERR_NOT_PD", 5: "FCA_ERR_EIG_NOCONV", 6: "FCA_ERR_NONFINITE",
                7: "FCA_ERR_TIMEOUT", 8: "FCA_ERR_STATE", 9: "FCA_ERR_SCRATCH"}
FCA_NOALLOC_SCRATCH_BYTES = 8 << 20

# Every entry point declared in include/fca.h.
EXPORTS = ("fca_init", "fca_load", "fca_em_conventional", "fca_em_fast", "fca_em_fast_recover",
           "fca_separate", "fca_get_params", "fca_loglik_bins", "fca_last_em_kernel_ms",
           "fca_kernel_launches", "fca_set_eigensolver", "fca_measure_peaks",
           "fca_sync_status", "fca_free", "fca_status_string", "fca_version",
           "fca_em_fast_noalloc", "fca_batch_init", "fca_batch_load", "fca_batch_run",
           "fca_batch_tune", "fca_batch_shape", "fca_batch_set_shape", "fca_batch_set_eigensolver",
           "fca_batch_get_params", "fca_batch_sync_status",
           "fca_batch_free",
           "fca_server_create", "fca_server_request_bytes", "fca_server_submit",
           "fca_server_wait", "fca_server_stats", "fca_server_destroy", "fca_stft_frames",
           "fca_stft", "fca_istft", "fca_set_conv_layout")


class fca_problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("F", ctypes.c_int32), ("N", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("location", ctypes.c_int32),
                ("y", ctypes.c_void_p), ("y_scale", ctypes.c_void_p),
                ("v0", ctypes.c_void_p), ("S0", ctypes.c_void_p), ("seed", ctypes.c_uint64)]


class fca_batch_problem(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("M", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("N", ctypes.c_void_p), ("location", ctypes.c_int32), ("y", ctypes.c_void_p),
                ("v0", ctypes.c_void_p), ("S0", ctypes.c_void_p)]


class fca_server_config(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32)]


class fca_request(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("F", ctypes.c_int32), ("N", ctypes.c_int32),
                ("form", ctypes.c_int32), ("iters", ctypes.c_int32), ("y", ctypes.c_void_p),
                ("v0", ctypes.c_void_p), ("S0", ctypes.c_void_p), ("x1", ctypes.c_void_p),
                ("x2", ctypes.c_void_p), ("loglik", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class fca_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class fca_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint64), ("max_in_flight", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_uint64), ("bytes_peak", ctypes.c_uint64),
                ("bytes_budget", ctypes.c_uint64)]


class FCAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({fca_status_string(code)})")


def _load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libfca.so not built at {path}: run paper_1805_06572_gb300/build.py "
                          "(the FCA kernels have no CPU fallback)")
    lib = ctypes.CDLL(path)
    V, I = ctypes.c_void_p, ctypes.c_int32
    lib.fca_init.argtypes = [ctypes.POINTER(fca_problem), V, ctypes.POINTER(V)]
    lib.fca_load.argtypes = [V, ctypes.POINTER(fca_problem), V]
    lib.fca_em_conventional.argtypes = [V, I, V, V]
    lib.fca_em_fast.argtypes = [V, I, V, V]
    lib.fca_set_conv_layout.argtypes = [V, I]
    lib.fca_em_fast_recover.argtypes = [V, I, V, V]
    lib.fca_separate.argtypes = [V, V, V, I, V]
    lib.fca_get_params.argtypes = [V, V, V, V]
    lib.fca_loglik_bins.argtypes = [V, V, ctypes.POINTER(I), V]
    lib.fca_last_em_kernel_ms.argtypes = [V, ctypes.POINTER(ctypes.c_float)]
    lib.fca_kernel_launches.argtypes = []
    lib.fca_kernel_launches.restype = ctypes.c_uint64
    lib.fca_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.fca_measure_peaks.restype = ctypes.c_int
    lib.fca_set_eigensolver.argtypes = [V, I, I]
    lib.fca_set_eigensolver.restype = ctypes.c_int
    lib.fca_sync_status.argtypes = [V, V]
    lib.fca_free.argtypes = [V]
    lib.fca_free.restype = None
    lib.fca_status_string.argtypes = [ctypes.c_int]
    lib.fca_status_string.restype = ctypes.c_char_p
    lib.fca_em_fast_noalloc.argtypes = [I, I, I, V, V, V, I, V, V, V, V, V]
    lib.fca_em_fast_noalloc.restype = ctypes.c_int
    lib.fca_batch_init.argtypes = [ctypes.POINTER(fca_batch_problem), V, ctypes.POINTER(V)]
    lib.fca_batch_load.argtypes = [V, ctypes.POINTER(fca_batch_problem), V]
    lib.fca_batch_run.argtypes = [V, I, I, V, V, V, V, I, V]
    lib.fca_batch_tune.argtypes = [V, I, V]
    lib.fca_batch_shape.argtypes = [V, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.fca_batch_set_shape.argtypes = [V, I, I, I]
    lib.fca_batch_set_shape.restype = ctypes.c_int
    lib.fca_batch_get_params.argtypes = [V, I, V, V, V]
    lib.fca_batch_get_params.restype = ctypes.c_int
    lib.fca_batch_set_eigensolver.argtypes = [V, I, I]
    lib.fca_batch_set_eigensolver.restype = ctypes.c_int
    lib.fca_batch_sync_status.argtypes = [V, V]
    lib.fca_batch_free.argtypes = [V]
    lib.fca_batch_free.restype = None
    for name in ("fca_batch_init", "fca_batch_load", "fca_batch_run", "fca_batch_tune",
                 "fca_batch_shape", "fca_batch_sync_status"):
        getattr(lib, name).restype = ctypes.c_int
    lib.fca_server_create.argtypes = [ctypes.POINTER(fca_server_config), ctypes.POINTER(V)]
    lib.fca_server_request_bytes.argtypes = [I, I, I, I]
    lib.fca_server_request_bytes.restype = ctypes.c_size_t
    lib.fca_server_submit.argtypes = [V, ctypes.POINTER(fca_request), ctypes.POINTER(ctypes.c_uint64)]
    lib.fca_server_wait.argtypes = [V, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(fca_request_info)]
    lib.fca_server_stats.argtypes = [V, ctypes.POINTER(fca_server_counters)]
    lib.fca_server_destroy.argtypes = [V]
    lib.fca_server_destroy.restype = None
    for name in ("fca_server_create", "fca_server_submit", "fca_server_wait", "fca_server_stats"):
        getattr(lib, name).restype = ctypes.c_int
    lib.fca_stft_frames.argtypes = [ctypes.c_int64, I, I]
    lib.fca_stft_frames.restype = ctypes.c_int64
    lib.fca_stft.argtypes = [I, ctypes.c_int64, V, I, I, V, V]
    lib.fca_stft.restype = ctypes.c_int
    lib.fca_istft.argtypes = [I, I, V, I, I, V, V, ctypes.c_int64, V]
    lib.fca_istft.restype = ctypes.c_int
    lib.fca_version.argtypes = []
    lib.fca_version.restype = ctypes.c_char_p
    for name in ("fca_init", "fca_load", "fca_em_conventional", "fca_em_fast", "fca_em_fast_recover",
                 "fca_separate", "fca_get_params", "fca_loglik_bins", "fca_last_em_kernel_ms",
                 "fca_sync_status"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def fca_status_string(code: int) -> str:
    return lib.fca_status_string(int(code)).decode()


def fca_version() -> str:
    return lib.fca_version().decode()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(rc: int, where: str):
    if rc != FCA_OK:
        raise FCAError(rc, where)


def _problem(y, v0, S0, y_scale, seed=0, encode_f16=False):
    if y.dtype == torch.complex64:
        F, N, M = y.shape
        storage = FCA_STORE_F16_SCALED if encode_f16 else FCA_STORE_C64
        if encode_f16 and (y_scale is not None or not y.is_cuda):
            raise ValueError("encode_f16 takes a complex64 mixture on the device and no y_scale")
    elif y.dtype == torch.float16:
        F, N, M, two = y.shape
        assert two == 2
        storage = FCA_STORE_F16_SCALED
        if y_scale is None:
            raise ValueError("a float16 mixture needs its y_scale")
    else:
        raise TypeError("y must be complex64 [F,N,M] or float16 [F,N,M,2]")
    if (v0 is None) != (S0 is None):
        raise ValueError("give both v0 and S0, or neither (seeded initial values)")
    for t in (y, v0, S0, y_scale):
        if t is None:
            continue
        if not t.is_contiguous():
            raise ValueError("inputs must be contiguous")
        if t.is_cuda != y.is_cuda:
            raise ValueError("y, y_scale, v0 and S0 must all be on the device or all on the host")
    if v0 is not None and (v0.dtype != torch.float64 or S0.dtype != torch.complex128):
        raise TypeError("v0 must be float64 [2,F,N], S0 complex128 [2,F,M,M]")
    p = fca_problem(M=M, F=F, N=N, storage=storage,
                    location=FCA_MEM_DEVICE if y.is_cuda else FCA_MEM_HOST,
                    y=y.data_ptr(), y_scale=None if y_scale is None else y_scale.data_ptr(),
                    v0=None if v0 is None else v0.data_ptr(),
                    S0=None if S0 is None else S0.data_ptr(), seed=int(seed) & (2**64 - 1))
    return p


class State:
    """Owning handle of an fca_state (freed by fca_free or garbage collection)."""

    def __init__(self, handle: int, M: int, F: int, N: int, storage: int):
        self.handle, self.M, self.F, self.N, self.storage = handle, M, F, N, storage

    def __del__(self):
        if getattr(self, "handle", None):
            lib.fca_free(ctypes.c_void_p(self.handle))
            self.handle = None


def fca_init(y, v0=None, S0=None, y_scale=None, stream=None, seed=0, encode_f16=False) -> State:
    """v0 = S0 = None: the library's seeded initial values from `seed` (fca_problem in fca.h).
    encode_f16: store the complex64 device mixture y as FP16 with a per-frequency scale, encoded
    by the library."""
    p = _problem(y, v0, S0, y_scale, seed, encode_f16)
    out = ctypes.c_void_p()
    _check(lib.fca_init(ctypes.byref(p), ctypes.c_void_p(_stream(stream)), ctypes.byref(out)), "fca_init")
    return State(out.value, p.M, p.F, p.N, p.storage)


def fca_load(state: State, y, v0=None, S0=None, y_scale=None, stream=None, seed=0, encode_f16=False):
    p = _problem(y, v0, S0, y_scale, seed, encode_f16)
    _check(lib.fca_load(ctypes.c_void_p(state.handle), ctypes.byref(p), ctypes.c_void_p(_stream(stream))),
           "fca_load")


def fca_set_conv_layout(state: State, layout: int):
    """FCA_CONV_AUTO, FCA_CONV_THREAD or FCA_CONV_GROUP for the state's conventional EM."""
    _check(lib.fca_set_conv_layout(ctypes.c_void_p(state.handle), int(layout)), "fca_set_conv_layout")


def fca_em_fast(state: State, iters: int, loglik=None, stream=None):
    _check(lib.fca_em_fast(ctypes.c_void_p(state.handle), int(iters), _ptr(loglik),
                           ctypes.c_void_p(_stream(stream))), "fca_em_fast")


def fca_em_fast_recover(state: State, iters: int, loglik=None, stream=None):
    _check(lib.fca_em_fast_recover(ctypes.c_void_p(state.handle), int(iters), _ptr(loglik),
                                   ctypes.c_void_p(_stream(stream))), "fca_em_fast_recover")


def fca_em_conventional(state: State, iters: int, loglik=None, stream=None):
    _check(lib.fca_em_conventional(ctypes.c_void_p(state.handle), int(iters), _ptr(loglik),
                                   ctypes.c_void_p(_stream(stream))), "fca_em_conventional")


def fca_separate(state: State, x1, x2, mode: int = FCA_SEP_ALG1, stream=None):
    _check(lib.fca_separate(ctypes.c_void_p(state.handle), _ptr(x1), _ptr(x2), int(mode),
                            ctypes.c_void_p(_stream(stream))), "fca_separate")


def fca_get_params(state: State, v=None, S=None, stream=None):
    """v: device float32 [2,F,N] or None; S: host complex128 [2,F,M,M] or None."""
    _check(lib.fca_get_params(ctypes.c_void_p(state.handle), _ptr(v), _ptr(S),
                              ctypes.c_void_p(_stream(stream))), "fca_get_params")


def fca_loglik_bins(state: State, stream=None):
    """Per-frequency log-likelihood [L, F] (float64, host) of the last EM call."""
    n = ctypes.c_int32(0)
    _check(lib.fca_loglik_bins(ctypes.c_void_p(state.handle), None, ctypes.byref(n),
                               ctypes.c_void_p(_stream(stream))), "fca_loglik_bins")
    out = torch.empty((n.value, state.F), dtype=torch.float64).pin_memory()
    _check(lib.fca_loglik_bins(ctypes.c_void_p(state.handle), _ptr(out), None,
                               ctypes.c_void_p(_stream(stream))), "fca_loglik_bins")
    return out


def fca_last_em_kernel_ms(state: State) -> float:
    ms = ctypes.c_float(0.0)
    _check(lib.fca_last_em_kernel_ms(ctypes.c_void_p(state.handle), ctypes.byref(ms)),
           "fca_last_em_kernel_ms")
    return float(ms.value)


def fca_kernel_launches() -> int:
    return int(lib.fca_kernel_launches())


def fca_set_eigensolver(state: State, precision: int = FCA_GEVD_FP32, max_sweeps: int = 30):
    """Precision of FastFCA's per-bin eigensolver and Gram merge (FCA_GEVD_FP32, _FP64 or
    _REFINED) and its Jacobi sweep cap."""
    _check(lib.fca_set_eigensolver(ctypes.c_void_p(state.handle), int(precision), int(max_sweeps)),
           "fca_set_eigensolver")


def fca_measure_peaks():
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.fca_measure_peaks(ctypes.byref(a), ctypes.byref(b)), "fca_measure_peaks")
    return a.value, b.value


def fca_sync_status(state: State, stream=None) -> int:
    return int(lib.fca_sync_status(ctypes.c_void_p(state.handle), ctypes.c_void_p(_stream(stream))))


def fca_free(state: State):
    if state.handle:
        lib.fca_free(ctypes.c_void_p(state.handle))
        state.handle = None


def _expect(t, name, dtype, shape, dev):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be {dtype} {list(shape)}, got {t.dtype} {list(t.shape)}")
    if not t.is_contiguous() or t.device != dev:
        raise ValueError(f"{name} must be contiguous and on {dev}")


def fca_em_fast_noalloc(y, v0, S0, iters: int, v, x1, x2, loglik=None, stream=None) -> int:
    """FastFCA on caller-owned device tensors with the library's fixed scratch array (no
    device allocation). Synchronises the stream; returns the status code. Shapes, dtypes,
    contiguity and device are checked here (the library can only check pointers)."""
    if y.dim() != 3:
        raise ValueError("y must be complex64 [F,N,M]")
    F, N, M = y.shape
    dev = torch.device("cuda", torch.cuda.current_device())
    _expect(y, "y", torch.complex64, (F, N, M), dev)
    _expect(v0, "v0", torch.float64, (2, F, N), dev)
    _expect(S0, "S0", torch.complex128, (2, F, M, M), dev)
    _expect(v, "v", torch.float32, (2, F, N), dev)
    _expect(x1, "x1", torch.complex64, (F, N, M), dev)
    _expect(x2, "x2", torch.complex64, (F, N, M), dev)
    if loglik is not None:
        if loglik.dtype != torch.float64 or loglik.numel() < iters or not loglik.is_contiguous() \
                or loglik.device != dev:
            raise ValueError(f"loglik must be contiguous float64 on {dev} with >= {iters} elements")
    return int(lib.fca_em_fast_noalloc(M, F, N, _ptr(y), _ptr(v0), _ptr(S0), int(iters), _ptr(v),
                                       _ptr(x1), _ptr(x2), _ptr(loglik),
                                       ctypes.c_void_p(_stream(stream))))


def run(y, v0, S0, iters: int, form: str = "fast", y_scale=None, mode: int = FCA_SEP_ALG1,
        want_ll: bool = True, stream=None):
    """One-shot convenience over the C ABI: load, `iters` EM iterations, posterior means.

    Inputs may be device tensors or (pinned) host tensors. Returns device tensors
    (x1, x2, loglik, v) and the state."""
    dev = torch.device("cuda", torch.cuda.current_device())
    st = fca_init(y, v0, S0, y_scale=y_scale, stream=stream)
    ll = torch.empty(iters, dtype=torch.float64, device=dev) if want_ll and iters > 0 else None
    (fca_em_fast if form == "fast" else fca_em_conventional)(st, iters, ll, stream=stream)
    x1 = torch.empty((st.F, st.N, st.M), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    fca_separate(st, x1, x2, mode, stream=stream)
    v = torch.empty((2, st.F, st.N), dtype=torch.float32, device=dev)
    fca_get_params(st, v=v, stream=stream)
    return x1, x2, ll, v, st


# ------------------------------------------------------------------------------ batches
def batch_offsets(M, F, N):
    """Element offsets of each mixture in the packed layouts of include/fca.h:
    (y/x offsets in complex elements, v offsets, S offsets in complex elements) and the totals."""
    import numpy as np
    M, F, N = (np.asarray(a, dtype=np.int64) for a in (M, F, N))
    fnm, fn2, fmm2 = F * N * M, 2 * F * N, 2 * F * M * M
    off = lambda a: np.concatenate([[0], np.cumsum(a)[:-1]])  # noqa: E731
    return (off(fnm), off(fn2), off(fmm2)), (int(fnm.sum()), int(fn2.sum()), int(fmm2.sum()))


class Batch:
    """Owning handle of an fca_batch."""

    def __init__(self, handle: int, M, F, N):
        self.handle = handle
        self.M, self.F, self.N = list(M), list(F), list(N)
        (self.x_off, self.v_off, self.S_off), (self.x_elems, self.v_elems, self.S_elems) = \
            batch_offsets(M, F, N)

    @property
    def count(self):
        return len(self.M)

    def __del__(self):
        if getattr(self, "handle", None):
            lib.fca_batch_free(ctypes.c_void_p(self.handle))
            self.handle = None


def _batch_problem(M, F, N, y, v0, S0):
    import numpy as np
    Ma, Fa, Na = (np.ascontiguousarray(a, dtype=np.int32) for a in (M, F, N))
    for t, dt in ((y, torch.complex64), (v0, torch.float64), (S0, torch.complex128)):
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError("batch inputs: y complex64, v0 float64, S0 complex128, contiguous")
        if t.is_cuda != y.is_cuda:
            raise ValueError("y, v0 and S0 must all be on the device or all on the host")
    p = fca_batch_problem(count=len(Ma), M=Ma.ctypes.data, F=Fa.ctypes.data, N=Na.ctypes.data,
                          location=FCA_MEM_DEVICE if y.is_cuda else FCA_MEM_HOST,
                          y=y.data_ptr(), v0=v0.data_ptr(), S0=S0.data_ptr())
    return p, (Ma, Fa, Na)


def fca_batch_init(M, F, N, y, v0, S0, stream=None) -> Batch:
    """y, v0, S0: flat packed tensors (complex64, float64, complex128)."""
    p, keep = _batch_problem(M, F, N, y, v0, S0)
    out = ctypes.c_void_p()
    _check(lib.fca_batch_init(ctypes.byref(p), ctypes.c_void_p(_stream(stream)), ctypes.byref(out)),
           "fca_batch_init")
    del keep
    return Batch(out.value, M, F, N)


def fca_batch_load(batch: Batch, y, v0, S0, stream=None):
    p, keep = _batch_problem(batch.M, batch.F, batch.N, y, v0, S0)
    _check(lib.fca_batch_load(ctypes.c_void_p(batch.handle), ctypes.byref(p),
                              ctypes.c_void_p(_stream(stream))), "fca_batch_load")
    del keep


def fca_batch_run(batch: Batch, form: int, iters: int, x1, x2, loglik=None, v=None,
                  use_graph: bool = False, stream=None):
    _check(lib.fca_batch_run(ctypes.c_void_p(batch.handle), int(form), int(iters), _ptr(loglik),
                             _ptr(x1), _ptr(x2), _ptr(v), 1 if use_graph else 0,
                             ctypes.c_void_p(_stream(stream))), "fca_batch_run")


def fca_batch_tune(batch: Batch, iters: int, stream=None):
    _check(lib.fca_batch_tune(ctypes.c_void_p(batch.handle), int(iters),
                              ctypes.c_void_p(_stream(stream))), "fca_batch_tune")


def fca_batch_shape(batch: Batch, M: int):
    """(bins, threads per CTA, dynamic shared memory bytes) of the channel-count group M."""
    b, t, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.fca_batch_shape(ctypes.c_void_p(batch.handle), int(M), ctypes.byref(b),
                               ctypes.byref(t), ctypes.byref(r)), "fca_batch_shape")
    return b.value, t.value, r.value


def fca_batch_set_shape(batch: Batch, M: int, threads: int, res_bytes: int):
    _check(lib.fca_batch_set_shape(ctypes.c_void_p(batch.handle), int(M), int(threads),
                                   int(res_bytes)), "fca_batch_set_shape")


def fca_batch_get_params(batch: Batch, k: int, want_S: bool = True, want_llf: bool = False,
                         iters: int = 0, stream=None):
    """Mixture k's S (host complex128 [2,F,M,M]) and per-bin log-likelihood (host float64
    [iters, F]) after the last batch run; None for the ones not asked for."""
    M, F = batch.M[k], batch.F[k]
    S = torch.empty((2, F, M, M), dtype=torch.complex128) if want_S else None
    llf = torch.empty((iters, F), dtype=torch.float64) if want_llf else None
    _check(lib.fca_batch_get_params(ctypes.c_void_p(batch.handle), int(k), _ptr(S), _ptr(llf),
                                    ctypes.c_void_p(_stream(stream))), "fca_batch_get_params")
    return S, llf


def fca_batch_set_eigensolver(batch: Batch, precision: int = FCA_GEVD_DEFAULT, max_sweeps: int = 30):
    _check(lib.fca_batch_set_eigensolver(ctypes.c_void_p(batch.handle), int(precision), int(max_sweeps)),
           "fca_batch_set_eigensolver")


def fca_batch_sync_status(batch: Batch, stream=None) -> int:
    return int(lib.fca_batch_sync_status(ctypes.c_void_p(batch.handle),
                                         ctypes.c_void_p(_stream(stream))))


def fca_batch_free(batch: Batch):
    if batch.handle:
        lib.fca_batch_free(ctypes.c_void_p(batch.handle))
        batch.handle = None


# ------------------------------------------------------------------------------ serving
class Server:
    """Owning handle of an fca_server; keeps every submitted request's tensors alive until the
    request has been waited for."""

    def __init__(self, handle: int):
        self.handle = handle
        self.live = {}

    def __del__(self):
        if getattr(self, "handle", None):
            lib.fca_server_destroy(ctypes.c_void_p(self.handle))
            self.handle = None


def fca_server_create(device_bytes: int, max_inflight: int = 8) -> Server:
    cfg = fca_server_config(device_bytes=int(device_bytes), max_inflight=int(max_inflight))
    out = ctypes.c_void_p()
    _check(lib.fca_server_create(ctypes.byref(cfg), ctypes.byref(out)), "fca_server_create")
    return Server(out.value)


def fca_server_request_bytes(M: int, F: int, N: int, iters: int) -> int:
    return int(lib.fca_server_request_bytes(int(M), int(F), int(N), int(iters)))


def fca_server_submit(srv: Server, y, v0, S0, x1, x2, iters: int, form: int = FCA_FORM_FAST,
                      loglik=None, v=None) -> int:
    """y complex64 [F,N,M], v0 float64 [2,F,N], S0 complex128 [2,F,M,M]; outputs x1, x2
    complex64 [F,N,M], loglik float64 [iters] (or None) and v float32 [2,F,N] (or None). Host
    tensors should be pinned."""
    F, N, M = y.shape
    r = fca_request(M=M, F=F, N=N, form=int(form), iters=int(iters), y=y.data_ptr(),
                    v0=v0.data_ptr(), S0=S0.data_ptr(), x1=x1.data_ptr(), x2=x2.data_ptr(),
                    loglik=None if loglik is None else loglik.data_ptr(),
                    v=None if v is None else v.data_ptr())
    t = ctypes.c_uint64()
    _check(lib.fca_server_submit(ctypes.c_void_p(srv.handle), ctypes.byref(r), ctypes.byref(t)),
           "fca_server_submit")
    srv.live[t.value] = (y, v0, S0, x1, x2, loglik, v)
    return t.value


def fca_server_wait(srv: Server, ticket: int, timeout_ms: int = -1):
    """Returns (status code, {"t_submit", "t_admit", "t_done"}) (status FCA_ERR_TIMEOUT = 7 if
    the limit passed; the ticket then stays valid)."""
    info = fca_request_info()
    rc = int(lib.fca_server_wait(ctypes.c_void_p(srv.handle), ctypes.c_uint64(ticket),
                                 ctypes.c_int64(timeout_ms), ctypes.byref(info)))
    if rc != 7:
        srv.live.pop(ticket, None)
    return rc, {"t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done}


def fca_server_stats(srv: Server) -> dict:
    c = fca_server_counters()
    _check(lib.fca_server_stats(ctypes.c_void_p(srv.handle), ctypes.byref(c)), "fca_server_stats")
    return {k: getattr(c, k) for k, _ in fca_server_counters._fields_}


def fca_server_destroy(srv: Server):
    if srv.handle:
        lib.fca_server_destroy(ctypes.c_void_p(srv.handle))
        srv.handle = None
        srv.live.clear()


# ------------------------------------------------------------------------------------ STFT
def fca_stft_frames(T: int, W: int = 1024, H: int = 512) -> int:
    return int(lib.fca_stft_frames(int(T), int(W), int(H)))


def fca_stft(x, W: int = 1024, H: int = 512, stream=None):
    """x: device float32 [M, T] -> device complex64 [F, N, M] (F = W/2 + 1)."""
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.dim() != 2:
        raise TypeError("x must be a contiguous device float32 tensor [M, T]")
    M, T = x.shape
    N = fca_stft_frames(T, W, H)
    y = torch.empty((W // 2 + 1, max(N, 1), M), dtype=torch.complex64, device=x.device)
    _check(lib.fca_stft(M, T, _ptr(x), W, H, _ptr(y), ctypes.c_void_p(_stream(stream))), "fca_stft")
    return y


def fca_istft(y, T: int, W: int = 1024, H: int = 512, stream=None):
    """y: device complex64 [F, N, M] -> device float32 [M, T]."""
    F, N, M = y.shape
    frames = torch.empty(N * M * W, dtype=torch.float32, device=y.device)
    x = torch.empty((M, T), dtype=torch.float32, device=y.device)
    _check(lib.fca_istft(M, N, _ptr(y), W, H, _ptr(frames), _ptr(x), int(T),
                         ctypes.c_void_p(_stream(stream))), "fca_istft")
    return x
