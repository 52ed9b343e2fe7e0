"""The basis update of Eq. (recoverS) (back-transform S, then a full generalised
eigendecomposition each iteration) against the efficient update of Eq. (updatePeff) and the
FP64 oracle, through the C ABI (GPU only). Sec. 3 proves the two updates equal, so both
trajectories must match the oracle at the parity tolerances."""
import numpy as np
import pytest
import torch

import oracle
import synth
from fca_testlib import assert_within, errors

pytestmark = pytest.mark.gpu


def _run(fca, y, v0, S0, iters, recover):
    dev = torch.device("cuda")
    st = fca.fca_init(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                        for a in (y.astype(np.complex64), v0, S0)))
    F, N, M = y.shape
    ll = torch.empty(iters, dtype=torch.float64, device=dev)
    (fca.fca_em_fast_recover if recover else fca.fca_em_fast)(st, iters, ll)
    x1 = torch.empty((F, N, M), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(x1)
    fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
    v = torch.empty((2, F, N), dtype=torch.float32, device=dev)
    S = torch.empty((2, F, M, M), dtype=torch.complex128)
    fca.fca_get_params(st, v=v, S=S)
    assert fca.fca_sync_status(st) == 0
    out = {"v": v.cpu().numpy().astype(np.float64), "mu1": x1.cpu().numpy(),
           "mu2": x2.cpu().numpy(), "ll": ll.cpu().numpy(), "S": S.numpy()}
    out["llf"] = fca.fca_loglik_bins(st).numpy().copy()
    fca.fca_free(st)
    return out


@pytest.fixture(scope="module")
def fca():
    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca as mod
    return mod


@pytest.mark.parametrize("name", ["small", "mid"])
def test_recover_update_matches_oracle_and_efficient_update(fca, name):
    c, mix, v0, S0 = synth.make_config(name, F=64 if name == "mid" else None)
    g = _run(fca, mix["y"], v0, S0, c.iters, recover=True)
    r = oracle.em("fast", mix["y"], v0, S0, c.iters)
    assert_within(errors(g, r, mix["y"]), f"{name} recoverS")
    e = _run(fca, mix["y"], v0, S0, c.iters, recover=False)
    rel = np.abs(g["v"] - e["v"]) / e["v"]
    assert np.median(rel) < 1e-4 and rel.max() < 1e-3
    assert g["llf"].shape == (c.iters, mix["y"].shape[0])
    assert np.all(np.diff(g["ll"]) >= -1e-6 * np.abs(g["ll"][1:]))


def test_recover_update_every_channel_count(fca):
    for M in range(1, 9):
        mix = synth.make_mixture(M, 6, 150, 0.1, 1.0, 3000 + M)
        v0, S0 = synth.init_params(mix["y"], 3000 + M, x=mix["x"])
        g = _run(fca, mix["y"], v0, S0, 8, recover=True)
        r = oracle.em("fast", mix["y"], v0, S0, 8)
        assert_within(errors(g, r, mix["y"]), f"M={M}")
