"""The multi-process path on CPU: world size 2, gloo, 127.0.0.1.

A batch of independent trees is split by tree across the ranks (no data-path collective);
each rank runs its shard (here with the CPU oracle, so no GPU is needed), the slowest rank's
time is the job's time, and rank 0 gathers the per-tree results.  The gathered batch must
equal a single-process run, with every tree computed exactly once.
"""
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

from paper_1710_01362_gb300 import shard
from paper_1710_01362_gb300 import workloads as W

N_TREES, N_STEPS = 5, 3   # 5 trees over 2 ranks: an uneven split (3 + 2)


def _problems():
    return [W.sf_small(seed=s, n_env=2, L=3, d=3, D=3, n_modes=6, n_steps=N_STEPS) for s in range(30, 30 + N_TREES)]


def _run_tree(p):
    from oracle.ttns import TTNS
    st = TTNS(p)
    pops = []
    for _ in range(N_STEPS):
        st.step(p.dt)
        pops.append(np.real(np.diag(st.rho_el())).copy())
    return np.array(pops)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ps = _problems()
        lo, hi = shard.shard_range(len(ps), rank, world)
        shard.barrier()
        t0 = time.perf_counter()
        mine = {k: _run_tree(ps[k]) for k in range(lo, hi)}
        secs = time.perf_counter() - t0
        tmax = shard.max_over_ranks(secs)
        parts = shard.gather_to_rank0(mine)
        q.put((rank, lo, hi, secs, tmax, parts))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_partitions_every_item_once():
    for n in range(0, 11):
        for world in range(1, 5):
            blocks = [shard.shard_range(n, r, world) for r in range(world)]
            covered = [k for lo, hi in blocks for k in range(lo, hi)]
            assert covered == list(range(n))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.merge_shards([{0: 1}, {0: 2}], 1)
    with pytest.raises(ValueError):
        shard.merge_shards([{0: 1}], 2)
    assert shard.aggregate_rate(10, 2, 4.0) == 5.0


def test_two_ranks_gloo_batch_equals_single_process():
    torch = pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    (r0, lo0, hi0, s0, tmax0, parts0), (r1, lo1, hi1, s1, tmax1, parts1) = results
    assert (lo0, hi0, lo1, hi1) == (0, 3, 3, 5)
    assert tmax0 == tmax1 == pytest.approx(max(s0, s1))
    assert parts1 is None and len(parts0) == 2
    gathered = shard.merge_shards(parts0, N_TREES)
    single = [_run_tree(p) for p in _problems()]
    for a, b in zip(gathered, single):
        assert np.array_equal(a, b)


def _plan_worker(rank, world, port, q):
    # each rank compiles (host only, ttns_plan in libttns.so) exactly the trees of its shard of
    # the batched workload, as bench.py's batched run builds them on its GPU; rank 0 gathers
    # the per-tree bond tables
    import torch.distributed as dist
    from paper_1710_01362_gb300 import build, ttns
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        build.build()
        seeds = list(range(1000, 1000 + 40))
        lo, hi = shard.shard_range(len(seeds), rank, world)
        mine = {k: ttns.plan([W.batched_spin_boson(seeds[k])])["bonds"] for k in range(lo, hi)}
        info = ttns.plan([W.batched_spin_boson(seeds[k]) for k in range(lo, hi)])
        parts = shard.gather_to_rank0(mine)
        q.put((rank, lo, hi, info["n_nodes"], parts))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_plan_the_batched_shards_through_the_library():
    pytest.importorskip("torch")
    from paper_1710_01362_gb300 import ttns
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_plan_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lo0, hi0, n0, parts0), (r1, lo1, hi1, n1, _) = results
    assert (lo0, hi0, lo1, hi1) == (0, 20, 20, 40)
    gathered = shard.merge_shards(parts0, 40)   # every tree planned by exactly one rank
    whole = ttns.plan([W.batched_spin_boson(s) for s in range(1000, 1040)])
    assert n0 + n1 == whole["n_nodes"]
    for k, bonds in enumerate(gathered):
        assert bonds == ttns.plan([W.batched_spin_boson(1000 + k)])["bonds"]
