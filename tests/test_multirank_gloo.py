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


# ---------------------------------------------------------------------------
# Parallel tree code host logic (paper Sec. IV-B) over gloo: ORB partition,
# body exchange and LET exchange between two processes on the CPU.
class CpuOps:
    """A CPU stand-in for one process's library steps of the ORB (numpy,
    written from the documented semantics of nb_orb_box, nb_orb_hist,
    nb_orb_cut, nb_orb_pack and nb_orb_order), so that the package's host
    orchestration runs across gloo processes without a GPU."""

    @staticmethod
    def _key_hi(pos, axis):
        b = (np.asarray(pos)[:, axis] + 0.0).view(np.uint64)
        return np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))

    def orb_box(self, pos, group, ngroups):
        x, g = pos.numpy(), group.numpy()
        out = np.tile(np.array([np.inf] * 3 + [-np.inf] * 3), (ngroups, 1))
        for q in range(ngroups):
            if np.any(g == q):
                out[q, :3] = x[g == q].min(0)
                out[q, 3:] = x[g == q].max(0)
        return out

    def _rows(self, pos, ids, group, active, axis):
        x, g, i = pos.numpy(), group.numpy(), ids.numpy().astype(np.uint64)
        for r, a in enumerate(active):
            sel = np.flatnonzero(g == a)
            yield r, sel, self._key_hi(x[sel], axis[r]), i[sel] & np.uint64(0xffffffff)

    def orb_hist(self, pos, ids, group, active, axis, prefix, rnd):
        out = np.zeros((len(active), 256), dtype=np.int64)
        bits = 8 * rnd
        for r, _, hi, lo in self._rows(pos, ids, group, active, axis):
            ph, pl = np.uint64(prefix[r][0]), np.uint64(prefix[r][1])
            if bits == 0:
                ok = np.ones(hi.size, bool)
            elif bits <= 64:
                s = np.uint64(64 - bits)
                ok = (hi >> s) == (ph >> s)
            else:
                s = np.uint64(32 - (bits - 64))
                ok = (hi == ph) & ((lo >> s) == (pl >> s))
            if rnd < 8:
                d = (hi >> np.uint64(56 - 8 * rnd)) & np.uint64(255)
            else:
                d = (lo >> np.uint64(24 - 8 * (rnd - 8))) & np.uint64(255)
            out[r] = np.bincount(d[ok].astype(np.int64), minlength=256)
        return out

    def orb_cut(self, pos, ids, group, active, axis, split, upper):
        g = group.numpy()
        for r, sel, hi, lo in list(self._rows(pos, ids, group, active, axis)):
            sh, sl = np.uint64(split[r][0]), np.uint64(split[r][1])
            below = (hi < sh) | ((hi == sh) & (lo < sl))
            g[sel[~below]] = upper[r]

    def orb_pack(self, rank, P, pos, vel, mass, ids):
        import torch
        o = np.argsort(rank.numpy(), kind="stable")
        counts = np.bincount(rank.numpy(), minlength=P).astype(np.int64)
        return (*(torch.as_tensor(t.numpy()[o]) for t in (pos, vel, mass, ids)), counts)

    def orb_order(self, pos, vel, mass, ids):
        import torch
        o = np.argsort(ids.numpy(), kind="stable")
        return tuple(torch.as_tensor(t.numpy()[o]) for t in (pos, vel, mass, ids))


def _crit2(pos, theta):
    ext = float((pos.max(0) - pos.min(0)).max())
    ext = ext if ext > 0 else 1.0
    return [np.float32(np.float32(ext / 2 ** L) / np.float32(theta)) ** 2 for L in range(11)]


def _let_worker(rank, ws, port, q):
    import pickle
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1211_2292_gb300 import let
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        comm = let.TorchComm(device="cpu")
        b = inputs.two_plummer(1500, seed=95)
        N = b.n
        lo, hi = rank * N // ws, (rank + 1) * N // ws
        pos, vel, mass = (torch.as_tensor(a[lo:hi].copy()) for a in (b.pos, b.vel, b.mass))
        ids = torch.arange(lo, hi, dtype=torch.int64)
        ops = CpuOps()
        part = let.orb_partition(ops, comm, pos, ids)
        pos, vel, mass, ids = let.exchange(ops, comm, part, pos, vel, mass, ids)
        # the LET of this process's tree for the other process's bodies, sent
        # as bytes: only the sent nodes (kind, level, cube, children)
        theta, leaf_cap = 0.6, 16
        x = pos.numpy()
        xf = x.astype(np.float32)
        boxes = comm.allgather(np.concatenate([xf.min(0), xf.max(0)]))
        sends = []
        for d in range(ws):
            if d == rank:
                sends.append(torch.empty(0, dtype=torch.uint8))
                continue
            t = oracle.bh_let(x, mass.numpy(), theta, leaf_cap, boxes[d][:3], boxes[d][3:])
            sent = np.flatnonzero(t["kind"] != 0)
            payload = {"crit2": _crit2(x, theta),
                       "nodes": {int(u): (int(t["kind"][u]), int(t["level"][u]), t["lo"][u],
                                          t["hi"][u], [int(k) for k in t["child"][u] if k >= 0])
                                 for u in sent}}
            sends.append(torch.frombuffer(bytearray(pickle.dumps(payload)), dtype=torch.uint8))
        recvs = comm.alltoallv(sends)
        # brute force on the receiving side: each local body walks the remote
        # tree alone, seeing only what was received
        missing = 0
        for s in range(ws):
            if s == rank:
                continue
            let_s = pickle.loads(recvs[s].numpy().tobytes())
            nodes, crit2 = let_s["nodes"], let_s["crit2"]
            for p in xf:
                stack = [0]
                while stack:
                    u = stack.pop()
                    if u not in nodes:
                        missing += 1
                        continue
                    kind, level, clo, chi, kids = nodes[u]
                    dd = np.maximum(np.maximum(clo - p, p - chi), np.float32(0))
                    d2 = np.float32(0)
                    for c in range(3):
                        d2 = np.float32(d2 + np.float32(dd[c] * dd[c]))
                    if d2 >= crit2[level]:
                        continue  # accepted: the node itself suffices
                    if kids:
                        missing += kind != 2
                        stack.extend(kids)
                    else:
                        missing += kind != 3
        q.put((rank, part.numpy(), ids.numpy(), missing))
    finally:
        dist.destroy_process_group()


def test_two_processes_orb_exchange_and_let_with_gloo():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_let_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = inputs.two_plummer(1500, seed=95)
    ref = oracle.orb(b.pos, 2)
    # the distributed ORB is the oracle's, and it is equal-count
    assert np.array_equal(np.concatenate([o[1] for o in out]), ref)
    assert abs(int((ref == 0).sum()) - int((ref == 1).sum())) <= 1
    for rank, _, ids, missing in out:
        # the exchange delivered exactly this domain's bodies, in id order
        assert np.array_equal(ids, np.flatnonzero(ref == rank))
        # every node a local body opens or accepts in the remote tree arrived
        assert missing == 0


@pytest.mark.parametrize("P", [1, 3, 4, 7])
def test_thread_emulated_processes_partition_like_the_oracle(P):
    # the same host logic with P processes emulated by threads (as the GPU
    # tests run it on one device), with the CPU stand-in for the kernels
    import torch
    import oracle
    from paper_1211_2292_gb300 import let
    b = inputs.two_plummer(800, seed=96)
    N = b.n

    def fn(comm):
        r = comm.rank
        lo, hi = r * N // P, (r + 1) * N // P
        pos, vel, mass = (torch.as_tensor(a[lo:hi].copy()) for a in (b.pos, b.vel, b.mass))
        ids = torch.arange(lo, hi, dtype=torch.int64)
        ops = CpuOps()
        part = let.orb_partition(ops, comm, pos, ids)
        _, _, _, mine = let.exchange(ops, comm, part, pos, vel, mass, ids)
        return part.numpy(), mine.numpy()

    res = let.run_threads(P, fn)
    ref = oracle.orb(b.pos, P)
    assert np.array_equal(np.concatenate([r[0] for r in res]), ref)
    for r, (_, mine) in enumerate(res):
        assert np.array_equal(mine, np.flatnonzero(ref == r))
