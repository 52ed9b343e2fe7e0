"""The multi-process path on CPU with gloo (world size 2): frequency shards need no exchange
during EM; the log-likelihood sum and the benchmark's max-over-ranks timing are the only
reductions."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1805_06572_gb300.shard import (allreduce_max, allreduce_sum, frequency_shard,
                                              weak_scaling_value)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    c, mix, v0, S0 = synth.make_config("small", F=21)
    lo, hi = frequency_shard(21, rank, world)
    r = oracle.em("fast", mix["y"][lo:hi], v0[:, lo:hi], S0[:, lo:hi], 6, want_mu=False,
                  nthreads=1)
    ll = allreduce_sum(r["ll"].sum(axis=1), dist)
    slow = allreduce_max(0.5 + rank, dist)
    val = weak_scaling_value(100.0, world, slow)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, r["v"]))
    if rank == 0:
        np.savez(os.path.join(out_dir, "out.npz"), ll=ll.numpy(), slow=slow, val=val,
                 v=np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])], axis=1))
    dist.barrier()
    dist.destroy_process_group()


def test_frequency_shards_are_balanced_and_cover():
    from paper_1805_06572_gb300.shard import frequency_shard, mixture_shard
    for F in (1, 2, 5, 257, 513):
        for world in (1, 2, 3, 8):
            ranges = [frequency_shard(F, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == F
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [h - l for l, h in ranges]
            assert max(sizes) - min(sizes) <= 1
    assert sorted(sum((mixture_shard(10, r, 3) for r in range(3)), [])) == list(range(10))


def test_two_rank_gloo_shards_equal_the_single_run(tmp_path):
    import oracle
    import synth
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    got = np.load(tmp_path / "out.npz")
    c, mix, v0, S0 = synth.make_config("small", F=21)
    full = oracle.em("fast", mix["y"], v0, S0, 6, want_mu=False, nthreads=1)
    np.testing.assert_allclose(got["ll"], full["ll"].sum(axis=1), rtol=1e-13)
    np.testing.assert_array_equal(got["v"], full["v"])
    assert float(got["slow"]) == 1.5
    assert float(got["val"]) == pytest.approx(2 * 100.0 / 1.5)
