"""Parallel tree code across processes (paper Sec. IV-B): orthogonal
recursive bisection (ORB) of space into one equal-count domain per process,
the exchange that moves every body to its domain's process, and locally
essential trees (LET): each process builds a tree over its own bodies,
sends every other process the part of it that process's bodies need, and
then computes its bodies' forces as in the sequential tree code.

This module is host orchestration only.  Every computation on bodies runs in
the library's kernels behind an ``ops`` object (an :class:`~.nbody.NBody`
context: ``orb_box``, ``orb_hist``, ``orb_cut``, ``orb_pack``, ``orb_order``,
``let_build``, ``let_export``, ``let_forces``); this module orders those
calls and moves their results between processes through a communicator:

* :class:`TorchComm` -- ``torch.distributed`` (NCCL for CUDA tensors across
  GPUs, gloo on the CPU);
* :class:`ThreadComm` -- P processes emulated by P threads of one process
  (each with its own context), for running the same code on one GPU.

The collectives are host-side: no kernel ever waits for another process.
"""
from __future__ import annotations

import threading

import numpy as np

ROUNDS = 12  # 8-bit digits of the 96-bit key (coordinate image, body id)


# --------------------------------------------------------------- communicators
class Comm:
    """What the orchestration needs from a communicator."""

    rank: int
    size: int

    def allreduce(self, a: np.ndarray, op: str) -> np.ndarray:  # op: sum, min, max
        raise NotImplementedError

    def allgather(self, a: np.ndarray) -> list:
        raise NotImplementedError

    def alltoallv(self, sends: list) -> list:
        """sends[d]: a 1-D tensor for process d (all of one dtype); returns
        recvs[s]: what process s sent here."""
        raise NotImplementedError


class TorchComm(Comm):
    """torch.distributed: host arrays travel as tensors on `device` (CUDA for
    NCCL, CPU for gloo); alltoallv exchanges the sizes, then the data."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist, self.group, self.device = dist, group, device
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allreduce(self, a, op):
        import torch
        t = torch.as_tensor(np.ascontiguousarray(a)).to(self.device)
        ops = {"sum": self.dist.ReduceOp.SUM, "min": self.dist.ReduceOp.MIN,
               "max": self.dist.ReduceOp.MAX}
        self.dist.all_reduce(t, op=ops[op], group=self.group)
        return t.cpu().numpy()

    def allgather(self, a):
        import torch
        t = torch.as_tensor(np.ascontiguousarray(a)).to(self.device)
        out = [torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t, group=self.group)
        return [o.cpu().numpy() for o in out]

    def alltoallv(self, sends):
        import torch
        dev = sends[0].device
        n_send = torch.tensor([int(s.numel()) for s in sends], dtype=torch.int64, device=self.device)
        n_recv = torch.empty_like(n_send)
        self.dist.all_to_all_single(n_recv, n_send, group=self.group)
        n_recv = [int(v) for v in n_recv.cpu()]
        inp = torch.cat([s.reshape(-1) for s in sends]).to(self.device)
        out = torch.empty(sum(n_recv), dtype=inp.dtype, device=self.device)
        self.dist.all_to_all_single(out, inp, output_split_sizes=n_recv,
                                    input_split_sizes=[int(s.numel()) for s in sends],
                                    group=self.group)
        return [t.to(dev) for t in torch.split(out, n_recv)]


class ThreadWorld:
    """Shared state of P emulated processes (one thread each)."""

    def __init__(self, size: int):
        self.size = size
        self.barrier = threading.Barrier(size)
        self.slots = [None] * size


class ThreadComm(Comm):
    def __init__(self, world: ThreadWorld, rank: int):
        self.world, self.rank, self.size = world, rank, world.size

    def _exchange(self, value):
        w = self.world
        w.slots[self.rank] = value
        w.barrier.wait()
        out = list(w.slots)
        w.barrier.wait()  # everyone has read before the next exchange writes
        return out

    def allreduce(self, a, op):
        vals = self._exchange(np.array(a, copy=True))
        f = {"sum": np.add, "min": np.minimum, "max": np.maximum}[op]
        out = vals[0]
        for v in vals[1:]:
            out = f(out, v)
        return out

    def allgather(self, a):
        return [np.array(v, copy=True) for v in self._exchange(np.array(a, copy=True))]

    def alltoallv(self, sends):
        table = self._exchange([s.clone() for s in sends])
        return [table[s][self.rank] for s in range(self.size)]


def run_threads(size: int, fn):
    """Run fn(comm) in `size` threads with a ThreadComm each; returns the
    results in rank order (an exception in any thread is re-raised)."""
    world = ThreadWorld(size)
    out, err = [None] * size, [None] * size

    def body(r):
        try:
            out[r] = fn(ThreadComm(world, r))
        except BaseException as e:  # noqa: BLE001 - re-raised below
            err[r] = e
            world.barrier.abort()

    ts = [threading.Thread(target=body, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for e in err:
        if e is not None and not isinstance(e, threading.BrokenBarrierError):
            raise e
    for e in err:
        if e is not None:
            raise e
    return out


# ------------------------------------------------------------------------ ORB
def _set_digit(key, rnd, d):
    """Place digit d of round rnd in a 96-bit key held as [high 64, low 32]."""
    if rnd < 8:
        key[0] |= np.uint64(d) << np.uint64(56 - 8 * rnd)
    else:
        key[1] |= np.uint64(d) << np.uint64(24 - 8 * (rnd - 8))


def orb_partition(ops, comm: Comm, pos, ids):
    """Each local body's processor under the ORB of all processes' bodies
    (int32 CUDA tensor).  Every part shared by p > 1 processors is cut across
    the longest side of its global bounding box, the lower part taking
    floor(p/2) processors and floor(count floor(p/2) / p) bodies; the cut key
    is found by a radix select whose digit histograms are summed over the
    processes."""
    import torch
    P = comm.size
    group = torch.zeros(ids.shape[0], dtype=torch.int32, device=ids.device)
    parts = [(0, P)]
    while any(p > 1 for _, p in parts):
        active = [(r0, p) for r0, p in parts if p > 1]
        box = ops.orb_box(pos, group, P)
        lo = comm.allreduce(box[:, :3], "min")
        hi = comm.allreduce(box[:, 3:], "max")
        axis = []
        for r0, _ in active:
            ext = hi[r0] - lo[r0]
            a = 0
            for c in (1, 2):  # the longest side, the lowest axis on ties
                if ext[c] > ext[a]:
                    a = c
            axis.append(a)
        key = np.zeros((len(active), 2), dtype=np.uint64)
        need = np.zeros(len(active), dtype=np.int64)
        heads = [r0 for r0, _ in active]
        for rnd in range(ROUNDS):
            h = comm.allreduce(ops.orb_hist(pos, ids, group, heads, axis, key, rnd), "sum")
            for r, (_, p) in enumerate(active):
                if rnd == 0:
                    need[r] = int(h[r].sum()) * (p // 2) // p  # bodies below the cut
                cum = np.cumsum(h[r])
                if cum[-1] == 0:
                    continue  # the part holds no body
                d = int(np.searchsorted(cum, need[r], side="right"))
                need[r] -= int(cum[d - 1]) if d > 0 else 0
                _set_digit(key[r], rnd, d)
        ops.orb_cut(pos, ids, group, heads, axis, key, [r0 + p // 2 for r0, p in active])
        parts = [c for r0, p in parts
                 for c in (((r0, p),) if p == 1 else ((r0, p // 2), (r0 + p // 2, p - p // 2)))]
    return group


def exchange(ops, comm: Comm, rank, pos, vel, mass, ids):
    """Move every body to its processor (rank, from orb_partition); returns
    this process's (pos, vel, mass, ids), ordered by id."""
    P = comm.size
    p2, v2, m2, i2, counts = ops.orb_pack(rank, P, pos, vel, mass, ids)
    off = np.concatenate([[0], np.cumsum(counts)])
    rows = [slice(int(off[d]), int(off[d + 1])) for d in range(P)]
    rp = comm.alltoallv([p2[s].reshape(-1) for s in rows])
    rv = comm.alltoallv([v2[s].reshape(-1) for s in rows])
    rm = comm.alltoallv([m2[s] for s in rows])
    ri = comm.alltoallv([i2[s] for s in rows])
    import torch
    cat = lambda ts, shape: torch.cat(ts).reshape(shape).contiguous()  # noqa: E731
    n = sum(int(t.numel()) for t in rm)
    return ops.orb_order(cat(rp, (n, 3)), cat(rv, (n, 3)), cat(rm, (n,)), cat(ri, (n,)))


# ------------------------------------------------------------------------ LET
def let_forces(ops, comm: Comm, pos, mass, G, eps, theta, leaf_cap, group, counts=False,
               return_lets=False):
    """Accelerations of this process's bodies (in their order) from its own
    tree and the LETs the other processes send it: each process builds its
    tree, the float32 boxes of all processes' bodies are gathered, each
    process exports one LET per other non-empty process, the LETs are
    exchanged, and each walks its own tree, then the received ones in
    processor order.  With return_lets, (result, received LETs) so that the
    walks can be repeated on the same trees."""
    import torch
    P, me = comm.size, comm.rank
    n = int(mass.shape[0])
    if n > 0:
        box = ops.let_build(pos, mass, leaf_cap)
    else:
        box = np.array([np.inf] * 3 + [-np.inf] * 3, dtype=np.float32)
    boxes = comm.allgather(box)
    dev = mass.device
    sends = []
    for d in range(P):
        empty = not np.all(boxes[d][:3] <= boxes[d][3:])
        if d == me or n == 0 or empty:
            sends.append(torch.empty(0, dtype=torch.uint8, device=dev))
        else:
            sends.append(ops.let_export(theta, boxes[d]))
    recvs = comm.alltoallv(sends)
    lets = [recvs[s] for s in range(P) if s != me and recvs[s].numel() > 0]
    if n == 0:
        z = torch.empty((0, 3), dtype=torch.float64, device=dev)
        out = (z, torch.empty((0, 2), dtype=torch.int32, device=dev)) if counts else z
    else:
        out = ops.let_forces(G, eps, theta, group, lets, counts=counts)
    return (out, lets) if return_lets else out
