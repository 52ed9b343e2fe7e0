"""Both layouts of the conventional EM kernel (one thread per point, lane groups) against the
oracle at every M, with ragged frame counts (a partial last pass of the lane groups)."""
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


@pytest.mark.parametrize("M", range(1, 9))
def test_conventional_layouts_match_the_oracle(fca, M):
    F, N, L, seed = 5, 37 + 11 * M, 6, 700 + M
    mix = synth.make_mixture(M, F, N, 0.1, 1.0, seed)
    v0, S0 = synth.init_params(mix["y"], seed, x=mix["x"])
    r = oracle.em("conventional", mix["y"], v0, S0, L)
    d = torch.device("cuda")
    outs = {}
    for layout in (fca.FCA_CONV_THREAD, fca.FCA_CONV_GROUP, fca.FCA_CONV_AUTO):
        st = fca.fca_init(torch.from_numpy(mix["y"]).to(d), torch.from_numpy(v0).to(d),
                          torch.from_numpy(S0).to(d))
        fca.fca_set_conv_layout(st, layout)
        ll = torch.empty(L, dtype=torch.float64, device=d)
        fca.fca_em_conventional(st, L, ll)
        x1 = torch.empty((F, N, M), dtype=torch.complex64, device=d)
        x2 = torch.empty_like(x1)
        fca.fca_separate(st, x1, x2, fca.FCA_SEP_ALG1)
        v = torch.empty((2, F, N), dtype=torch.float32, device=d)
        S = torch.empty((2, F, M, M), dtype=torch.complex128)
        fca.fca_get_params(st, v=v, S=S)
        assert fca.fca_sync_status(st) == 0
        g = {"v": v.cpu().numpy().astype(np.float64), "S": S.numpy(), "mu1": x1.cpu().numpy(),
             "mu2": x2.cpu().numpy(), "ll": ll.cpu().numpy()}
        assert_within(errors(g, r, mix["y"]), f"M={M} layout={layout}")
        outs[layout] = g
    np.testing.assert_array_equal(outs[fca.FCA_CONV_AUTO]["v"], outs[fca.FCA_CONV_THREAD]["v"])


def test_unknown_layout_is_rejected(fca):
    mix = synth.make_mixture(2, 3, 10, 0.1, 1.0, 3)
    v0, S0 = synth.init_params(mix["y"], 3, x=mix["x"])
    d = torch.device("cuda")
    st = fca.fca_init(torch.from_numpy(mix["y"]).to(d), torch.from_numpy(v0).to(d), torch.from_numpy(S0).to(d))
    with pytest.raises(fca.FCAError):
        fca.fca_set_conv_layout(st, 3)
