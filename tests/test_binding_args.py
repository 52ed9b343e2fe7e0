"""Argument marshalling of the Python binding for fca_init / fca_load (host side, no GPU): the
problem struct it builds for caller-given and seeded initial values, and the inputs it refuses
before calling the library."""
import ctypes

import pytest
import torch


@pytest.fixture(scope="module")
def fca():
    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca as mod
    return mod


def _y(F=3, N=4, M=2):
    return torch.zeros((F, N, M), dtype=torch.complex64)


def test_seeded_problem_has_null_initial_values(fca):
    p = fca._problem(_y(), None, None, None, seed=2**64 + 5)
    assert p.v0 is None and p.S0 is None and p.seed == 5  # seed taken modulo 2^64
    assert (p.M, p.F, p.N, p.storage, p.location) == (2, 3, 4, fca.FCA_STORE_C64, fca.FCA_MEM_HOST)


def test_given_initial_values(fca):
    v0 = torch.ones((2, 3, 4), dtype=torch.float64)
    S0 = torch.zeros((2, 3, 2, 2), dtype=torch.complex128)
    p = fca._problem(_y(), v0, S0, None)
    assert p.v0 == v0.data_ptr() and p.S0 == S0.data_ptr() and p.seed == 0


def test_refused_before_the_library(fca):
    v0 = torch.ones((2, 3, 4), dtype=torch.float64)
    S0 = torch.zeros((2, 3, 2, 2), dtype=torch.complex128)
    with pytest.raises(ValueError):      # one of v0, S0 without the other
        fca._problem(_y(), v0, None, None)
    with pytest.raises(ValueError):
        fca._problem(_y(), None, S0, None)
    with pytest.raises(ValueError):      # on-device encoding needs a device mixture
        fca._problem(_y(), None, None, None, encode_f16=True)
    y16 = torch.zeros((3, 4, 2, 2), dtype=torch.float16)
    with pytest.raises(ValueError):      # an FP16 mixture needs its scales
        fca._problem(y16, v0, S0, None)
    with pytest.raises(TypeError):       # wrong precision of the initial values
        fca._problem(_y(), v0.float(), S0, None)
    with pytest.raises(TypeError):
        fca._problem(torch.zeros((3, 4, 2)), v0, S0, None)


def test_struct_layout_matches_the_header(fca):
    """fca_problem: five int32 (M, F, N, storage, location), four pointers (y, y_scale, v0,
    S0) from the next 8-byte boundary, then the uint64 seed."""
    names = [n for n, _ in fca.fca_problem._fields_]
    assert names[-1] == "seed" and fca.fca_problem.seed.offset == 24 + 4 * 8
    assert ctypes.sizeof(fca.fca_problem) == fca.fca_problem.seed.offset + 8
