"""Multi-rank host logic on CPU (gloo, world size 2): sharding of independent
systems, per-rank work with no data-path collective, max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest

from paper_1211_2292_gb300 import inputs, shard


def test_shard_partitions_and_balances():
    sizes = inputs.batch_sizes(512, seed=3)
    for ws in (1, 2, 3, 4, 8):
        owned = [shard.shard_systems(sizes, ws, r) for r in range(ws)]
        allk = np.sort(np.concatenate(owned))
        assert np.array_equal(allk, np.arange(512))
        loads = [int((sizes[o].astype(np.int64) ** 2).sum()) for o in owned]
        # LPT bound: max load <= mean + largest single job
        assert max(loads) <= sum(loads) / ws + int(sizes.max()) ** 2
    with pytest.raises(ValueError):
        shard.shard_systems(sizes, 2, 2)


def test_gather_rows():
    off = [0, 3, 3, 10, 12]
    idx, local = shard.gather_rows(off, [2, 0, 1])
    assert list(idx) == [3, 4, 5, 6, 7, 8, 9, 0, 1, 2]
    assert list(local) == [0, 7, 10, 10]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bodies, off = inputs.plummer_batch(sizes=[40, 300, 64, 7, 150, 90, 1, 33], seed=5)
        mine = shard.shard_systems(np.diff(off), ws, rank)
        res = {}
        for k in mine:  # no collective on the data path
            s, e = off[k], off[k + 1]
            res[int(k)] = oracle.accel(bodies.pos[s:e], bodies.mass[s:e], 1.0, 0.01)
        t = shard.max_over_ranks(1.0 + rank, dist)
        gathered = [None] * ws  # test-only collection of the results
        dist.all_gather_object(gathered, res)
        q.put((rank, t, gathered if rank == 0 else None))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_time_with_gloo():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = {r: t for r, t, _ in out}
    assert times == {0: 2.0, 1: 2.0}
    gathered = [g for r, _, g in out if r == 0][0]
    merged = {}
    for part in gathered:
        assert not set(part) & set(merged)
        merged.update(part)
    bodies, off = inputs.plummer_batch(sizes=[40, 300, 64, 7, 150, 90, 1, 33], seed=5)
    assert sorted(merged) == list(range(8))
    for k, a in merged.items():
        s, e = off[k], off[k + 1]
        assert np.array_equal(a, oracle.accel(bodies.pos[s:e], bodies.mass[s:e], 1.0, 0.01))
