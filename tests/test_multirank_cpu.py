"""Multi-rank logic on CPU with the gloo backend (world size 2), no GPU.

Sharding covers every unit exactly once; the max-over-ranks step time is the
max; and splitting the 4^k cut index across ranks then sum-reducing the
partial marginals reproduces the full contraction (checked with the oracle's
FP64 contraction on a small cut circuit).
"""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2303_10788_gb300.sharding import shard_range


def test_shard_range_partitions():
    for n in (0, 1, 7, 168, 20736):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2303_10788_gb300.sharding import shard_range, max_over_ranks, sum_over_ranks
    from workloads import small_star
    from oracle.pipeline import evaluate_workload
    from oracle.cutting import recombine
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = max_over_ranks(1.0 + rank, dist)
    w = small_star()
    r = evaluate_workload(w, mode="exact")
    k = len(r.cuts)
    lo, hi = shard_range(4 ** k, rank, world)
    frags = r.fragments
    full = recombine(frags, r.tensors, k, len(w.marginal))
    # this rank's share of the naive sum over cut terms P in [lo, hi)
    o = np.arange(1 << len(w.marginal))
    p = np.zeros(1 << len(w.marginal))
    for P in range(lo, hi):
        prod = np.ones(1 << len(w.marginal))
        for f, T_ in zip(frags, r.tensors):
            of = np.zeros_like(o)
            for j, (mi, _) in enumerate(f.marg):
                of |= ((o >> mi) & 1) << j
            pf = 0
            for j, c in enumerate(f.slots):
                pf |= ((P >> (2 * c)) & 3) << (2 * j)
            prod = prod * T_[of, pf]
        p += prod
    total = sum_over_ranks(p / 2.0 ** k, dist).numpy()
    if rank == 0:
        out.put((t, float(np.abs(total - full).max())))
    dist.destroy_process_group()


def test_two_rank_reductions_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    t, err = q.get(timeout=5)
    assert t == 2.0
    assert err < 1e-12
