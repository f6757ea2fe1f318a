"""Parallel tree code (paper Sec. IV-B) on the GPU: ORB decomposition, body
exchange and locally essential trees, with P processes emulated by P threads
of this process on one GPU (each with its own library context; the
collectives are host-side, no kernel waits for another).

Against the oracle's parallel tree code: the ORB assigns every body the
oracle's processor and the exchange delivers each process exactly its
domain's bodies in id order (both exact); every body meets exactly the
oracle's numbers of cells and bodies over all trees (integers, exact), so
the LETs hold everything the walks need; the accelerations agree to the
float32 walk's bound (per-body relative error RMS <= 1e-5, max <= 1e-4).
One process reproduces nb_tree_forces bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import host, relerr_per_body, to_dev
from paper_1211_2292_gb300 import inputs, let, nbody

pytestmark = pytest.mark.gpu


def _run(cuda, b, P, theta, leaf_cap, group, eps):
    N = b.n

    def fn(comm):
        r = comm.rank
        lo, hi = r * N // P, (r + 1) * N // P  # a block of ids per process to start
        with nbody.NBody(max(N, 1), "fp32_comp") as nb:
            pos, vel, mass = (to_dev(a[lo:hi], cuda) for a in (b.pos, b.vel, b.mass))
            ids = torch.arange(lo, hi, dtype=torch.int64, device=cuda)
            rank = let.orb_partition(nb, comm, pos, ids)
            pos, vel, mass, ids = let.exchange(nb, comm, rank, pos, vel, mass, ids)
            acc, cnt = let.let_forces(nb, comm, pos, mass, 1.0, eps, theta, leaf_cap, group,
                                      counts=True)
            nb.sync()
            return host(rank), host(ids), host(pos), host(acc), host(cnt)

    return let.run_threads(P, fn)


@pytest.mark.parametrize("P,n_per,theta,group", [(2, 1500, 0.5, 64), (3, 1500, 0.7, 32),
                                                 (4, 5000, 0.5, 64), (4, 5000, 0.6, 32)])
def test_sharded_tree_matches_the_oracle(cuda, P, n_per, theta, group):
    b = inputs.two_plummer(n_per, seed=91)
    eps, leaf_cap = 0.002, 16
    res = _run(cuda, b, P, theta, leaf_cap, group, eps)
    ref_rank = oracle.orb(b.pos, P)
    assert np.array_equal(np.concatenate([r[0] for r in res]), ref_rank)
    ref, _, ref_cnt = oracle.bh_sharded(b.pos, b.mass, 1.0, eps, theta, leaf_cap, group,
                                        ref_rank, P)
    for r, (_, ids, pos, acc, cnt) in enumerate(res):
        mine = np.flatnonzero(ref_rank == r)
        assert np.array_equal(ids, mine) and np.array_equal(pos, b.pos[mine])
        assert np.array_equal(cnt.astype(np.int64), ref_cnt[mine, :2])
        e = relerr_per_body(acc, ref[mine])
        assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4


def test_one_process_is_the_tree_code(cuda):
    b = inputs.plummer(6000, seed=92)
    res = _run(cuda, b, 1, 0.5, 16, 64, 0.01)
    _, ids, _, acc, cnt = res[0]
    assert np.array_equal(ids, np.arange(b.n))
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a, c = nb.tree_forces(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.01, 0.5, 16,
                              counts=True, group=64)
        nb.sync()
    assert np.array_equal(acc, host(a)) and np.array_equal(cnt, host(c))


def test_let_sizes_match_the_oracle(cuda):
    # the LET one process sends another: as many nodes as the oracle marks
    # sent, and the bodies of the leaves it marks sent with their bodies
    b = inputs.two_plummer(3000, seed=93)
    rank = oracle.orb(b.pos, 4)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        for s, d, theta in ((0, 1, 0.5), (2, 0, 0.7), (3, 1, 0.4)):
            src, dst = rank == s, rank == d
            nb.let_build(to_dev(b.pos[src], cuda), to_dev(b.mass[src], cuda), 16)
            xd = b.pos[dst].astype(np.float32)
            box = np.concatenate([xd.min(0), xd.max(0)])
            buf = host(nb.let_export(theta, box))
            head = buf[:24].view(np.int64)
            ref = oracle.bh_let(b.pos[src], b.mass[src], theta, 16, box[:3], box[3:])
            leaves = ref["kind"] == 3
            assert head[1] == np.count_nonzero(ref["kind"])
            assert head[2] == int((ref["range"][leaves, 1] - ref["range"][leaves, 0]).sum())


def test_more_processes_than_bodies(cuda):
    b = inputs.plummer(3, seed=94)
    res = _run(cuda, b, 4, 0.5, 1, 32, 0.01)
    counts = [r[1].size for r in res]
    assert sorted(counts) == [0, 1, 1, 1]
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    for _, ids, _, acc, cnt in res:
        if ids.size:
            assert relerr_per_body(acc, ref[ids]).max() <= 1e-5
            assert np.all(cnt[:, 0] + cnt[:, 1] >= 1)


def test_argument_checks(cuda):
    with nbody.NBody(100, "fp32_comp") as nb:
        with pytest.raises(nbody.NBodyError):
            nb.let_export(0.5, np.zeros(6, np.float32))  # no local tree yet
        x = torch.zeros((10, 3), dtype=torch.float64, device=cuda)
        g = torch.zeros(10, dtype=torch.int32, device=cuda)
        ids = torch.arange(10, dtype=torch.int64, device=cuda)
        with pytest.raises(nbody.NBodyError):
            nb.orb_hist(x, ids, g, [0], [3], np.zeros((1, 2), np.uint64), 0)  # axis 3
        with pytest.raises(nbody.NBodyError):
            nb.orb_hist(x, ids, g, [0], [0], np.zeros((1, 2), np.uint64), 12)  # round 12
        with pytest.raises(nbody.NBodyError):
            nb.orb_cut(x, ids, g, [1], [0], np.zeros((1, 2), np.uint64), [1])  # upper not above
        with pytest.raises(nbody.NBodyError):
            nb.orb_pack(g + 5, 4, x, x, x[:, 0].contiguous(), ids)  # ranks beyond P
        m = torch.ones(10, dtype=torch.float64, device=cuda)
        nb.let_build(x, m, 16)
        junk = torch.zeros(256, dtype=torch.uint8, device=cuda)
        with pytest.raises(nbody.NBodyError):
            nb.let_forces(1.0, 0.01, 0.5, 64, [junk])  # not a LET
        nb.tree_forces(x, m, 1.0, 0.01, 0.5, 16)  # replaces the local tree
        with pytest.raises(nbody.NBodyError):
            nb.let_export(0.5, np.zeros(6, np.float32))


def test_ties_in_the_cut_coordinate(cuda):
    # Many bodies share the cut coordinate (a third coincident, and -0.0
    # against +0.0): the cut orders them by id, as the oracle does.
    b = inputs.plummer(2400, seed=95)
    pos = b.pos.copy()
    pos[::3] = [0.25, -0.5, 0.125]
    pos[1::7, 0] = 0.0
    pos[2::7, 0] = -0.0
    b = inputs.Bodies(pos, b.vel, b.mass)
    res = _run(cuda, b, 4, 0.5, 8, 32, 0.01)
    ref_rank = oracle.orb(b.pos, 4)
    assert np.array_equal(np.concatenate([r[0] for r in res]), ref_rank)
    ref, _, ref_cnt = oracle.bh_sharded(b.pos, b.mass, 1.0, 0.01, 0.5, 8, 32, ref_rank, 4)
    for r, (_, ids, _, acc, cnt) in enumerate(res):
        mine = np.flatnonzero(ref_rank == r)
        assert np.array_equal(ids, mine)
        assert np.array_equal(cnt.astype(np.int64), ref_cnt[mine, :2])
        e = relerr_per_body(acc, ref[mine])
        assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4


def test_more_trees_than_one_launch_takes(cuda):
    # 70 copies of one LET: the local tree and 63 received ones go in the
    # first launch, the rest in a second; counts add exactly and each copy
    # adds the same float64 sum
    b = inputs.two_plummer(3000, seed=96)
    rank = oracle.orb(b.pos, 2)
    src, dst = rank == 0, rank == 1
    with nbody.NBody(b.n, "fp32_comp") as other:
        other.let_build(to_dev(b.pos[src], cuda), to_dev(b.mass[src], cuda), 16)
        xd = b.pos[dst].astype(np.float32)
        let_buf = other.let_export(0.5, np.concatenate([xd.min(0), xd.max(0)]))
        other.sync()
        with nbody.NBody(b.n, "fp32_comp") as nb:
            nb.let_build(to_dev(b.pos[dst], cuda), to_dev(b.mass[dst], cuda), 16)
            runs = {}
            for k in (0, 1, 70):
                a, c = nb.let_forces(1.0, 0.01, 0.5, 64, [let_buf] * k, counts=True)
                nb.sync()
                runs[k] = (host(a), host(c).astype(np.int64))
    (a0, c0), (a1, c1), (a70, c70) = runs[0], runs[1], runs[70]
    assert np.array_equal(c70, c0 + 70 * (c1 - c0))
    d = a1 - a0
    assert np.allclose(a70, a0 + 70 * d, rtol=0, atol=1e-11 * np.abs(a70).max())
