"""The multi-GPU form is replicas: each rank aligns its own shard, no
alignment data crosses ranks, and only bookkeeping collectives run (a
barrier and the maximum of the ranks' elapsed times).  Checked here with two
gloo ranks on the CPU."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2204_02085_gb300 import sharding


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        r, w, local = sharding.dist_env()
        begin, end = sharding.shard_range(n, r, w)
        sharding.barrier()
        t_max = sharding.max_over_ranks(float(10 + 5 * r))
        seed = sharding.shard_seed(1, r)
        q.put((r, begin, end, t_max, seed, local))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = 1001
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, e0, t0, s0, l0), (r1, b1, e1, t1, s1, l1) = res
    assert (b0, e0, b1, e1) == (0, 501, 501, 1001)  # disjoint, covering, balanced
    assert t0 == t1 == 15.0  # max over ranks
    assert s0 == 1 and s1 != s0  # rank 0 keeps the workload's seed
    assert (l0, l1) == (0, 1)


@pytest.mark.parametrize("n,world", [(0, 3), (7, 3), (10, 4), (5, 8)])
def test_shard_range_covers(n, world):
    seen = []
    for r in range(world):
        b, e = sharding.shard_range(n, r, world)
        assert 0 <= b <= e <= n
        seen.extend(range(b, e))
    assert seen == list(range(n))
    sizes = [sharding.shard_range(n, r, world)[1] - sharding.shard_range(n, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_identity():
    assert sharding.max_over_ranks(3.5) == 3.5
    sharding.barrier()


def _work_worker(rank, world, port, q):
    """Rank `rank` aligns its work-balanced share of a mixed-length sample
    with the oracle (CPU) and sends it to rank 0, which reassembles."""
    import torch.distributed as dist

    import oracle
    from paper_2204_02085_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        batch = synth.mixed_reads(300, 100, 2000, 0.10, 0.05, seed=3)
        w = sharding.work_estimate(batch.pattern_lengths, batch.text_lengths)
        b, e = sharding.shard_by_work(w, rank, world)
        sc, st, words, off = oracle.wfa_batch(sharding.sub_batch(batch, b, e), (4, 6, 2), nthreads=2)
        gathered = [None] * world if rank == 0 else None
        dist.gather_object((b, sc, st, words, off), gathered, dst=0)
        if rank == 0:
            q.put(("parts", gathered, [sharding.shard_by_work(w, r, world) for r in range(world)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_work_balanced_reassembly(oracle_mod):
    from paper_2204_02085_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_work_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tag, parts, ranges = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batch = synth.mixed_reads(300, 100, 2000, 0.10, 0.05, seed=3)
    w = sharding.work_estimate(batch.pattern_lengths, batch.text_lengths)
    # the shares' estimated work differs by at most one pair's
    loads = [float(w[b:e].sum()) for b, e in ranges]
    assert abs(loads[0] - loads[1]) <= float(w.max())
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == batch.n
    got = sharding.reassemble(parts, batch.n)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=4)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_shard_by_work_balances(world):
    rng = np.random.default_rng(world)
    w = rng.integers(1, 1000, size=997).astype(np.float64) ** 2
    bounds = [sharding.shard_by_work(w, r, world) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == len(w)
    for (b0, e0), (b1, e1) in zip(bounds, bounds[1:]):
        assert e0 == b1
    loads = [w[b:e].sum() for b, e in bounds]
    assert max(loads) - min(loads) <= 2 * w.max()
    # each share's end is the first pair reaching its fraction of the total
    total = w.sum()
    for r, (b, e) in enumerate(bounds[:-1]):
        assert w[:e].sum() >= (r + 1) * total / world > w[:e - 1].sum()
