"""The C-ABI library loads and exports every entry point include/fca.h declares; host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "fca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fca_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1805_06572_gb300 as pkg
    path = pkg.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_same_symbols():
    from paper_1805_06572_gb300 import fca
    assert sorted(fca.EXPORTS) == declared_entry_points()


def test_status_strings_and_version(lib):
    lib.fca_status_string.restype = ctypes.c_char_p
    lib.fca_version.restype = ctypes.c_char_p
    assert lib.fca_status_string(0) == b"ok"
    assert b"positive definite" in lib.fca_status_string(4)
    assert b"sm_103a" in lib.fca_version()


def test_invalid_problems_are_rejected_on_the_host(lib):
    from paper_1805_06572_gb300.fca import fca_problem
    lib.fca_init.argtypes = [ctypes.POINTER(fca_problem), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    dummy = ctypes.c_void_p(16)
    for kw in (dict(M=0), dict(M=9), dict(F=0), dict(N=0), dict(storage=2), dict(location=3),
               dict(y=None), dict(S0=None), dict(v0=None), dict(storage=1, y_scale=None),
               dict(M=8, F=1 << 14, N=1 << 14)):
        args = dict(M=2, F=3, N=4, storage=0, location=1, y=dummy.value, y_scale=dummy.value,
                    v0=dummy.value, S0=dummy.value)
        args.update(kw)
        p = fca_problem(**args)
        out = ctypes.c_void_p(123)
        assert lib.fca_init(ctypes.byref(p), None, ctypes.byref(out)) == 1, kw
        assert out.value is None
    lib.fca_em_fast.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.fca_em_fast(None, 3, None, None) == 1
    lib.fca_free.argtypes = [ctypes.c_void_p]
    lib.fca_free(None)


def test_invalid_batches_are_rejected_on_the_host(lib):
    import numpy as np
    from paper_1805_06572_gb300.fca import fca_batch_problem
    lib.fca_batch_init.argtypes = [ctypes.POINTER(fca_batch_problem), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]
    dummy = 16
    for Ms, Fs, Ns, kw in (([2], [3], [4], dict(count=0)), ([9], [3], [4], {}), ([0], [3], [4], {}),
                           ([2, 2], [3, 0], [4, 4], {}), ([2], [3], [0], {}),
                           ([2], [3], [4], dict(location=5)), ([2], [3], [4], dict(y=None)),
                           ([2], [3], [4], dict(S0=None)), ([8], [1 << 14], [1 << 14], {})):
        M, F, N = (np.asarray(a, dtype=np.int32) for a in (Ms, Fs, Ns))
        args = dict(count=len(M), M=M.ctypes.data, F=F.ctypes.data, N=N.ctypes.data, location=0,
                    y=dummy, v0=dummy, S0=dummy)
        args.update(kw)
        p = fca_batch_problem(**args)
        out = ctypes.c_void_p(123)
        assert lib.fca_batch_init(ctypes.byref(p), None, ctypes.byref(out)) == 1, (Ms, Fs, Ns, kw)
        assert out.value is None
    lib.fca_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.c_void_p]
    assert lib.fca_batch_run(None, 0, 3, None, None, None, None, 0, None) == 1
    lib.fca_batch_free.argtypes = [ctypes.c_void_p]
    lib.fca_batch_free(None)


def test_server_arguments_are_checked_on_the_host(lib):
    from paper_1805_06572_gb300 import fca
    out = ctypes.c_void_p(123)
    for kw in (dict(device_bytes=0, max_inflight=4), dict(device_bytes=1 << 20, max_inflight=0),
               dict(device_bytes=1 << 20, max_inflight=65)):
        cfg = fca.fca_server_config(**kw)
        assert fca.lib.fca_server_create(ctypes.byref(cfg), ctypes.byref(out)) == 1, kw
        assert out.value is None
    for shape in ((0, 3, 4, 1), (9, 3, 4, 1), (2, 0, 4, 1), (2, 3, 0, 1), (2, 3, 4, -1)):
        assert fca.fca_server_request_bytes(*shape) == 0
    assert fca.fca_server_request_bytes(8, 513, 1000, 30) > 8 * 513 * 1000 * 8 * 3
    t = ctypes.c_uint64()
    assert fca.lib.fca_server_submit(None, None, ctypes.byref(t)) == 1
    fca.lib.fca_server_destroy(None)
