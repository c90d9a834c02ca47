"""Host-side bookkeeping for running the aligner on several GPUs.

Read pairs are independent (the paper aligns each pair on its own, with no
communication between processing units, Sec. I), so the multi-GPU form is
replicas: each rank aligns its own shard and no alignment data crosses
ranks.  The only collectives are bookkeeping ones: a barrier around the
timed region and the maximum of the ranks' elapsed times.

One caller batch over several GPUs: contiguous shares of equal estimated
work (a pair's wavefront cells grow with the square of its length at a given
edit rate), each aligned on its own device, and the shards' outputs placed
into one result (scores and status at the shard's pairs, CIGAR words after
the earlier shards' words, offsets moved by that count).
"""

from __future__ import annotations

import os

import numpy as np


def dist_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n units for rank; shares differ by at
    most one unit and cover [0, n) exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def work_estimate(pattern_lengths, text_lengths) -> np.ndarray:
    """Estimated work of each pair: (max(n, m) + 1)^2 (at a fixed edit rate
    the score grows with the length and the wavefront cells with the square
    of the score)."""
    L = np.maximum(np.asarray(pattern_lengths, dtype=np.float64), np.asarray(text_lengths, dtype=np.float64))
    return (L + 1.0) ** 2


def shard_by_work(weights, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of rank such that the shares' summed
    weights differ by at most one pair's weight: share r ends at the first
    pair whose running total reaches (r + 1) / world of the whole."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    w = np.asarray(weights, dtype=np.float64)
    n = len(w)
    if n == 0:
        return 0, 0
    prefix = np.cumsum(w)
    total = float(prefix[-1])

    def cut(r):  # pairs before share r
        if r <= 0:
            return 0
        if r >= world:
            return n
        # the smallest i with prefix[i-1] >= r * total / world
        return int(np.searchsorted(prefix, r * total / world, side="left")) + 1

    return min(cut(rank), n), min(max(cut(rank + 1), cut(rank)), n)


def sub_batch(batch, begin: int, end: int):
    """Pairs [begin, end) of a batch (offsets into the same sequence bytes)."""
    from . import synth

    return synth.Batch(batch.patterns, np.ascontiguousarray(batch.pattern_offsets[begin:end]),
                       np.ascontiguousarray(batch.pattern_lengths[begin:end]), batch.texts,
                       np.ascontiguousarray(batch.text_offsets[begin:end]),
                       np.ascontiguousarray(batch.text_lengths[begin:end]))


def reassemble(parts, n: int):
    """One result from shards [(begin, scores, status, words, offsets)] that
    cover [0, n) (each with its own offsets from 0): scores and status at the
    shard's pairs, words after the earlier shards' words."""
    parts = sorted(parts, key=lambda p: p[0])
    scores = np.empty(n, dtype=np.int32)
    status = np.empty(n, dtype=np.int8)
    offsets = np.zeros(n + 1, dtype=np.int64)
    words = []
    base, at = 0, 0
    for begin, sc, st, w, off in parts:
        k = len(sc)
        if begin != at:
            raise ValueError("shards do not cover the batch in order")
        scores[begin:begin + k] = sc
        status[begin:begin + k] = st
        offsets[begin + 1:begin + k + 1] = np.asarray(off[1:k + 1], dtype=np.int64) + base
        words.append(np.asarray(w[:int(off[k])], dtype=np.uint32))
        base += int(off[k])
        at = begin + k
    if at != n:
        raise ValueError("shards do not cover the batch")
    return scores, status, (np.concatenate(words) if words else np.zeros(0, np.uint32)), offsets


def align_multi_gpu(batch, pen, devices, scratch_bytes: int = 0):
    """Align one batch over several GPUs (one host thread and context per
    entry of `devices`; an entry may repeat): work-balanced contiguous
    shares, each aligned on its device with host buffers, reassembled.  No
    data crosses devices.  Returns (scores, status, cigar words, offsets)."""
    import threading

    from . import Aligner

    n = len(batch.pattern_lengths)
    w = work_estimate(batch.pattern_lengths, batch.text_lengths)
    world = len(devices)
    parts, errors = [None] * world, []

    def run(r):
        try:
            b, e = shard_by_work(w, r, world)
            with Aligner(devices[r], scratch_bytes) as al:
                sc, st, words, off = al.align(sub_batch(batch, b, e), pen)
            parts[r] = (b, sc, st, words, off)
        except Exception as exc:  # reported after every thread has stopped
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return reassemble(parts, n)


def shard_seed(seed: int, rank: int) -> int:
    """Seed of rank's own shard of a weak-scaling workload (rank 0 keeps the
    workload's seed)."""
    return seed if rank == 0 else seed + 7919 * rank


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a per-rank float across the process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def barrier(group=None) -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
