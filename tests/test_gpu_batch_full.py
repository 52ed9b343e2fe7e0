"""The many-mixture workload at full size, in the launch configuration the benchmark times
(512 mixtures, M in {2,4,6}, N in [200, 6000], F = 513, L = 50; tuned shapes; one CUDA graph
launch), checked against the FP64 oracle on sampled bins of sampled mixtures: v, the
posterior means, S and the per-bin log-likelihood (read back per mixture). Bins are
independent EM problems, so the oracle on a bin's own inputs is that bin's exact reference.
"""
import numpy as np
import pytest

import oracle
from fca_testlib import assert_within, errors

pytestmark = pytest.mark.gpu

SAMPLE_MIX = (0, 97, 211, 305, 406, 511)
SAMPLE_F = (0, 131, 256, 512)


@pytest.fixture(scope="module")
def full():
    import torch

    import paper_1805_06572_gb300 as pkg
    from synth import device as sdev
    pkg.build()
    from paper_1805_06572_gb300 import fca
    dev = torch.device("cuda")
    p = sdev.make_packed("batch", dev)
    b = fca.fca_batch_init(p["M"], p["F"], p["N"], p["y"], p["v0"], p["S0"])
    fca.fca_batch_tune(b, p["iters"])
    yield fca, torch, p, b
    fca.fca_batch_free(b)


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_full_batch_sampled_bins_match_oracle(full, form):
    fca, torch, p, b = full
    L = p["iters"]
    x1 = torch.empty(b.x_elems, dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    v = torch.empty(b.v_elems, dtype=torch.float32, device="cuda")
    fid = fca.FCA_FORM_FAST if form == "fast" else fca.FCA_FORM_CONVENTIONAL
    ll = torch.empty(b.count * L, dtype=torch.float64, device="cuda")
    fca.fca_batch_run(b, fid, L, x1, x2, loglik=ll, v=v, use_graph=True)
    assert fca.fca_batch_sync_status(b) == 0
    ll = ll.cpu().numpy().reshape(b.count, L)
    fs = np.asarray(SAMPLE_F)
    for k in SAMPLE_MIX:
        M, F, N = b.M[k], b.F[k], b.N[k]
        xo, vo, so = int(b.x_off[k]), int(b.v_off[k]), int(b.S_off[k])
        y = p["y"][xo:xo + F * N * M].view(F, N, M)[fs].cpu().numpy()
        v0 = p["v0"][vo:vo + 2 * F * N].view(2, F, N)[:, fs].cpu().numpy()
        S0 = p["S0"][so:so + 2 * F * M * M].view(2, F, M, M)[:, fs].cpu().numpy()
        r = oracle.em(form, y, v0, S0, L)
        S, llf = fca.fca_batch_get_params(b, k, want_llf=True, iters=L)
        llf = llf.numpy()
        # The per-bin log-likelihoods add up to the batch's per-mixture total.
        np.testing.assert_allclose(llf.sum(axis=1), ll[k], rtol=1e-12)
        got = {"mu1": x1[xo:xo + F * N * M].view(F, N, M)[fs].cpu().numpy(),
               "mu2": x2[xo:xo + F * N * M].view(F, N, M)[fs].cpu().numpy(),
               "v": v[vo:vo + 2 * F * N].view(2, F, N)[:, fs].cpu().numpy().astype(np.float64),
               "S": S.numpy()[:, fs], "llf": llf[:, fs]}
        err = errors(got, r, y, fs=np.arange(len(fs)))
        assert_within(err, f"{form} mixture {k} (M={M}, N={N})")
