"""Serving (fca_server_* through the C ABI, GPU only): requests admitted by device memory as
they arrive, run concurrently on their own streams, each with the results it gets alone.

Each request's kernels are the one-mixture kernels, whose arithmetic for a bin does not depend
on what else runs on the GPU, so the results in a mix must equal the results alone bitwise;
one request is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from fca_testlib import assert_within, errors

pytestmark = pytest.mark.gpu

F = 65
REQS = [(2, 300, 8), (4, 60, 8), (8, 120, 6), (2, 1000, 8), (4, 700, 10), (8, 64, 8),
        (2, 333, 5), (4, 1000, 7), (8, 500, 4), (2, 61, 9), (4, 250, 8), (8, 999, 3)]


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1805_06572_gb300 as pkg
    pkg.build()
    from paper_1805_06572_gb300 import fca
    reqs = []
    for i, (M, N, L) in enumerate(REQS):
        mix = synth.make_mixture(M, F, N, 0.05, 1.5, 7000 + i)
        v0, S0 = synth.init_params(mix["y"], 7000 + i, x=mix["x"])
        reqs.append((mix["y"], v0, S0, L))
    return fca, torch, reqs


def _buffers(torch, y, v0, S0, L):
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    Fy, N, M = y.shape
    return (pin(y.astype(np.complex64)), pin(v0), pin(S0),
            torch.empty((Fy, N, M), dtype=torch.complex64).pin_memory(),
            torch.empty((Fy, N, M), dtype=torch.complex64).pin_memory(),
            torch.empty(max(L, 1), dtype=torch.float64).pin_memory(),
            torch.empty((2, Fy, N), dtype=torch.float32).pin_memory())


def _submit(fca, srv, buf, L, form):
    y, v0, S0, x1, x2, ll, v = buf
    return fca.fca_server_submit(srv, y, v0, S0, x1, x2, L, form=form, loglik=ll if L else None,
                                 v=v)


@pytest.mark.parametrize("form", ["fast", "conventional"])
def test_results_in_the_mix_equal_results_alone(env, form):
    fca, torch, reqs = env
    fid = fca.FCA_FORM_FAST if form == "fast" else fca.FCA_FORM_CONVENTIONAL
    srv = fca.fca_server_create(2 << 30, max_inflight=8)
    alone = []
    for y, v0, S0, L in reqs:
        buf = _buffers(torch, y, v0, S0, L)
        rc, _ = fca.fca_server_wait(srv, _submit(fca, srv, buf, L, fid))
        assert rc == 0
        alone.append([t.numpy().copy() for t in buf[3:]])
    assert fca.fca_server_stats(srv)["max_in_flight"] == 1
    bufs = [_buffers(torch, y, v0, S0, L) for y, v0, S0, L in reqs]
    tickets = [_submit(fca, srv, b, L, fid) for b, (_, _, _, L) in zip(bufs, reqs)]
    infos = [fca.fca_server_wait(srv, t) for t in tickets]
    assert all(rc == 0 for rc, _ in infos)
    st = fca.fca_server_stats(srv)
    assert st["max_in_flight"] > 1, st  # the burst overlapped on the GPU
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0 and st["bytes_in_use"] == 0
    for a, b, (_, _, _, L) in zip(alone, bufs, reqs):
        for p, q in zip(a[:2], b[3:5]):
            assert np.array_equal(p, q.numpy())
        assert np.array_equal(a[2][:L], b[5].numpy()[:L])
        assert np.array_equal(a[3], b[6].numpy())
    # One request of the mix against the oracle (S is not an output of a request).
    y, v0, S0, L = reqs[4]
    r = oracle.em(form, y, v0, S0, L)
    got = {"mu1": bufs[4][3].numpy(), "mu2": bufs[4][4].numpy(), "ll": bufs[4][5].numpy()[:L],
           "v": bufs[4][6].numpy().astype(np.float64), "S": r["S"]}
    assert_within(errors(got, r, y), form)
    fca.fca_server_destroy(srv)


def test_admission_is_bounded_by_device_memory(env):
    fca, torch, reqs = env
    big = max(fca.fca_server_request_bytes(y.shape[2], F, y.shape[1], L) for y, _, _, L in reqs)
    srv = fca.fca_server_create(2 * big + 4096, max_inflight=8)
    bufs = [_buffers(torch, y, v0, S0, L) for y, v0, S0, L in reqs]
    tickets = [_submit(fca, srv, b, L, fca.FCA_FORM_FAST) for b, (_, _, _, L) in zip(bufs, reqs)]
    infos = [fca.fca_server_wait(srv, t) for t in tickets]
    assert all(rc == 0 for rc, _ in infos)
    st = fca.fca_server_stats(srv)
    assert 1 <= st["max_in_flight"] <= 8 and st["bytes_peak"] <= st["bytes_budget"]
    # A request is admitted ahead of an earlier one only while that one waits for memory, and
    # at most 8 requests go ahead of any one request.
    admits = [inf["t_admit"] for _, inf in infos]
    for i in range(len(admits)):
        ahead = sum(1 for j in range(i + 1, len(admits)) if admits[j] < admits[i])
        assert ahead <= 8, (i, ahead)
    fca.fca_server_destroy(srv)
    # A request larger than the whole arena is refused at submission.
    srv = fca.fca_server_create(big // 2, max_inflight=2)
    y, v0, S0, L = reqs[7]
    with pytest.raises(fca.FCAError) as ei:
        _submit(fca, srv, _buffers(torch, y, v0, S0, L), L, fca.FCA_FORM_FAST)
    assert ei.value.code == 3
    fca.fca_server_destroy(srv)


def test_small_requests_pass_a_large_one_waiting_for_memory(env):
    """A long first request holds part of the arena; the large request behind it cannot fit
    until the first finishes, and the small requests behind the large one are admitted ahead of
    it (within the arena left over) instead of waiting with it; all complete, with the results
    they get alone."""
    fca, torch, _ = env
    mk = lambda M, N, L, seed: (lambda m: (m["y"],) + synth.init_params(m["y"], seed, x=m["x"]) + (L,))(
        synth.make_mixture(M, F, N, 0.05, 1.5, seed))  # noqa: E731
    first = mk(8, 1000, 2000, 8101)  # long: 2000 iterations
    large = mk(8, 1000, 4, 8102)
    small = [mk(2, 100, 4, 8103 + k) for k in range(3)]
    b_first = fca.fca_server_request_bytes(8, F, 1000, 2000)
    b_large = fca.fca_server_request_bytes(8, F, 1000, 4)
    b_small = fca.fca_server_request_bytes(2, F, 100, 4)
    arena = b_first + max(b_large // 2, 3 * b_small + 3 * 4096)  # large cannot fit beside first
    assert arena < b_first + b_large and arena >= b_first + 3 * b_small
    srv = fca.fca_server_create(arena, max_inflight=8)
    reqs = [first, large] + small
    bufs = [_buffers(torch, y, v0, S0, L) for y, v0, S0, L in reqs]
    tickets = [_submit(fca, srv, b, L, fca.FCA_FORM_FAST) for b, (_, _, _, L) in zip(bufs, reqs)]
    infos = [fca.fca_server_wait(srv, t, timeout_ms=60000) for t in tickets]
    assert all(rc == 0 for rc, _ in infos)
    t_admit = [inf["t_admit"] for _, inf in infos]
    t_done = [inf["t_done"] for _, inf in infos]
    assert t_admit[1] >= t_done[0] - 1e-3           # the large one waited for the first one
    assert all(t_admit[k] < t_admit[1] for k in (2, 3, 4))  # the small ones went ahead of it
    fca.fca_server_destroy(srv)
    # each result equals the request run alone
    for (y, v0, S0, L), b in zip(reqs, bufs):
        alone = _buffers(torch, y, v0, S0, L)
        srv = fca.fca_server_create(fca.fca_server_request_bytes(y.shape[2], F, y.shape[1], L), max_inflight=1)
        rc, _ = fca.fca_server_wait(srv, _submit(fca, srv, alone, L, fca.FCA_FORM_FAST))
        assert rc == 0
        fca.fca_server_destroy(srv)
        for a, c in zip(b[3:], alone[3:]):
            np.testing.assert_array_equal(a.numpy(), c.numpy())


def test_a_failing_request_does_not_disturb_the_others(env):
    fca, torch, reqs = env
    srv = fca.fca_server_create(2 << 30, max_inflight=4)
    bufs = [_buffers(torch, y, v0, S0, L) for y, v0, S0, L in reqs[:6]]
    bufs[2][1][0, 0, 0] = float("nan")  # non-finite initial v: the device reports it
    tickets = [_submit(fca, srv, b, L, fca.FCA_FORM_FAST) for b, (_, _, _, L) in zip(bufs, reqs)]
    rcs = [fca.fca_server_wait(srv, t)[0] for t in tickets]
    assert rcs[2] == 6 and all(rc == 0 for i, rc in enumerate(rcs) if i != 2)
    st = fca.fca_server_stats(srv)
    assert st["failed"] == 1 and st["completed"] == 5
    fca.fca_server_destroy(srv)


def test_wait_with_a_time_limit(env):
    fca, torch, reqs = env
    srv = fca.fca_server_create(2 << 30, max_inflight=2)
    mix = synth.make_mixture(8, 513, 1000, 0.05, 1.5, 7100)
    v0, S0 = synth.init_params(mix["y"], 7100, x=mix["x"])
    buf = _buffers(torch, mix["y"], v0, S0, 30)
    t = _submit(fca, srv, buf, 30, fca.FCA_FORM_FAST)
    rc, _ = fca.fca_server_wait(srv, t, timeout_ms=0)
    assert rc in (0, 7)
    if rc == 7:
        rc, _ = fca.fca_server_wait(srv, t, timeout_ms=60000)
    assert rc == 0
    fca.fca_server_destroy(srv)
