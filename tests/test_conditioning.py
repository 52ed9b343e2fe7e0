"""How strongly the EM problem itself amplifies rounding-level perturbations of the mixture (FP64
oracle only; no GPU). This is the evidence behind the conditioning rule of the GPU parity tests
(fca_testlib.check_conditioned): from the random initialisation, at M = 8, N = 4000 and 100
iterations, the exact EM map amplifies a 1e-7 relative perturbation of y by more than 100x
(so a 1e-5 perturbation, FP32 rounding accumulated over a bin's frames, moves the outputs by more
than the 1e-3 max tolerance) on most bins, and by more than 1000x on some; from the mask-based
initialisation, and at the small workload, on none.

Bins are independent EM problems, so a sample of bins (every 16th) measures the same per-bin
responses as the full workload would.
"""
import numpy as np
import pytest

import synth
from fca_testlib import SENS_BOUND, SENS_EPS, oracle_response


def _response(name, recipe, step=1):
    c, mix, v0, S0 = synth.make_config(name, recipe=recipe)
    y = mix["y"].astype(np.complex128)
    if c.storage == "f16":
        _, _, y = synth.quantize_f16(mix["y"])
    fs = np.arange(0, c.F, step)
    return oracle_response("fast", y[fs], v0[:, fs], S0[:, fs], c.iters)


@pytest.fixture(scope="module")
def responses():
    return {("precision", "random"): _response("precision", "random", 16),
            ("precision", "mask"): _response("precision", "mask", 16),
            ("mid", "random"): _response("mid", "random"),
            ("small", "random"): _response("small", "random")}


def test_precision_workload_from_the_random_start_is_ill_conditioned(responses):
    r = responses[("precision", "random")]
    scaled = int((r > SENS_BOUND).sum())
    print(f"precision/random: {scaled} of {len(r)} sampled bins respond above {SENS_BOUND:g} "
          f"to a {SENS_EPS:g} perturbation (max {r.max():.3g})")
    assert scaled >= len(r) // 2 and r.max() > 1e-4


def test_mask_start_and_smaller_workloads_are_well_conditioned(responses):
    for key in (("precision", "mask"), ("small", "random")):
        r = responses[key]
        print(key, f"max response {r.max():.3g}")
        assert r.max() <= SENS_BOUND, key
    r = responses[("mid", "random")]
    print("mid/random", f"{(r > SENS_BOUND).sum()} of {len(r)} bins above {SENS_BOUND:g}, max {r.max():.3g}")
    # At M = 4 from the random start a minority of bins is above the bound, none by more than
    # a factor of 30 (the largest response of this draw is about 1e-4).
    assert (r > SENS_BOUND).sum() <= 0.25 * len(r) and r.max() < 30 * SENS_BOUND


def test_response_is_linear_in_the_perturbation():
    """The response is a derivative, not noise: halving the perturbation halves it."""
    c, mix, v0, S0 = synth.make_config("mid", recipe="random")
    fs = np.arange(0, c.F, 64)
    y = mix["y"].astype(np.complex128)[fs]
    import fca_testlib
    a = oracle_response("fast", y, v0[:, fs], S0[:, fs], c.iters)
    old = fca_testlib.SENS_EPS
    try:
        fca_testlib.SENS_EPS = old / 2
        b = fca_testlib.oracle_response("fast", y, v0[:, fs], S0[:, fs], c.iters)
    finally:
        fca_testlib.SENS_EPS = old
    ratio = a / b
    assert np.all(np.abs(ratio - 2.0) < 0.1), ratio
