"""Pins of the oracle's parallel tree code (paper Sec. IV-B): orthogonal
recursive bisection, per-processor trees and the locally essential tree.

None of these restates the oracle's formulas: the ORB is checked by its
counts and separating planes, the sharded walk against the single tree
(one processor), the direct sum (theta = 0) and the requirement that every
body is accounted for exactly once, and the LET by brute-force per-body
walks over the whole remote tree.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs


def _err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _parts_are_bisections(x, rank, rank0, p, idx):
    """Every cut of the ORB hierarchy separates the two parts by a plane
    across the longest side of the part's bounding box."""
    if p == 1 or idx.size == 0:
        return True
    lo_ranks = (rank[idx] >= rank0) & (rank[idx] < rank0 + p // 2)
    ext = x[idx].max(0) - x[idx].min(0)
    axis = int(np.argmax(ext))
    a, b = x[idx[lo_ranks], axis], x[idx[~lo_ranks], axis]
    if a.size and b.size and not a.max() <= b.min():
        return False
    return (_parts_are_bisections(x, rank, rank0, p // 2, idx[lo_ranks]) and
            _parts_are_bisections(x, rank, rank0 + p // 2, p - p // 2, idx[~lo_ranks]))


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("n", [0, 1, 7, 1000, 2047])
def test_orb_equal_counts_and_bisecting_planes(P, n):
    b = inputs.two_plummer(max((n + 1) // 2, 1), seed=81)
    x = b.pos[:n]
    rank = oracle.orb(x, P)
    counts = np.bincount(rank, minlength=P)
    assert counts.sum() == n and counts.max() - counts.min() <= 1
    assert _parts_are_bisections(x, rank, 0, P, np.arange(n))


def test_orb_follows_the_bodies():
    # relabelling the bodies relabels the result (distinct coordinates: no
    # ties), and a translation or a power-of-two scaling changes nothing
    b = inputs.plummer(3000, seed=82)
    rank = oracle.orb(b.pos, 6)
    perm = np.random.default_rng(3).permutation(b.n)
    assert np.array_equal(oracle.orb(b.pos[perm], 6), rank[perm])
    assert np.array_equal(oracle.orb(b.pos * 4.0 + 1.0, 6), rank)


@pytest.mark.parametrize("theta,group", [(0.3, 1), (0.5, 32), (0.8, 64)])
def test_one_processor_is_the_tree_code(theta, group):
    b = inputs.plummer(2500, seed=83)
    ref, rst, rcnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, theta, 16, group, counts=True)
    a, st, cnt = oracle.bh_sharded(b.pos, b.mass, 1.0, 0.01, theta, 16, group,
                                   np.zeros(b.n, np.int32), 1)
    assert np.array_equal(a, ref) and st == rst and np.array_equal(cnt[:, :2], rcnt)


@pytest.mark.parametrize("P", [2, 3, 5])
def test_theta_zero_is_the_direct_sum(P):
    b = inputs.two_plummer(1200, seed=84)
    rank = oracle.orb(b.pos, P)
    a, st, cnt = oracle.bh_sharded(b.pos, b.mass, 1.0, 0.005, 0.0, 8, 32, rank, P)
    assert _err(a, oracle.accel(b.pos, b.mass, 1.0, 0.005)).max() <= 1e-13
    assert np.all(cnt[:, 0] == 0) and np.all(cnt[:, 1] == b.n)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.8, 1.0])
@pytest.mark.parametrize("P", [2, 3, 4, 8])
def test_every_body_is_met_once(theta, P):
    # each body of the system appears on a body's lists exactly once, inside
    # a cell or by itself, summed over all processors' trees
    b = inputs.two_plummer(1500, seed=85)
    rank = oracle.orb(b.pos, P)
    _, st, cnt = oracle.bh_sharded(b.pos, b.mass, 1.0, 0.002, theta, 16, 64, rank, P)
    assert np.all(cnt[:, 2] == b.n)
    assert st["cell_interactions"] == cnt[:, 0].sum() and st["body_interactions"] == cnt[:, 1].sum()


def test_error_against_the_direct_sum_is_the_tree_codes():
    # splitting the tree over processors changes which cells are used, not
    # the accuracy of the method: within a factor 2 of the single tree's
    b = inputs.two_plummer(3000, seed=86)
    ex = oracle.accel(b.pos, b.mass, 1.0, 0.002)
    one, _ = oracle.bh_forces(b.pos, b.mass, 1.0, 0.002, 0.5, 16, 32)
    rms1 = np.sqrt((_err(one, ex) ** 2).mean())
    for P in (2, 4, 8):
        a, _, _ = oracle.bh_sharded(b.pos, b.mass, 1.0, 0.002, 0.5, 16, 32, oracle.orb(b.pos, P), P)
        rms = np.sqrt((_err(a, ex) ** 2).mean())
        assert 0.5 * rms1 <= rms <= 2.0 * rms1, (P, rms, rms1)


def _crit2(pos, theta):
    ext = float((pos.max(0) - pos.min(0)).max())
    ext = ext if ext > 0 else 1.0
    return [np.float32(np.float32(ext / 2 ** L) / np.float32(theta)) ** 2 for L in range(11)]


def _body_walk(d, crit2, p):
    """Per-body walk of the dumped tree (the paper's traversal): nodes tested,
    opened, listed as leaves and accepted."""
    seen, opened, leaves, accepted = [], [], [], []
    stack = [0]
    while stack:
        u = stack.pop()
        seen.append(u)
        lo, hi = d["lo"][u], d["hi"][u]
        dd = np.maximum(np.maximum(lo - p, p - hi), np.float32(0))
        d2 = np.float32(0)
        for c in range(3):
            d2 = np.float32(d2 + np.float32(dd[c] * dd[c]))
        kids = [int(k) for k in d["child"][u] if k >= 0]
        if d2 >= crit2[d["level"][u]]:
            accepted.append(u)
        elif not kids:
            leaves.append(u)
        else:
            opened.append(u)
            stack.extend(kids)
    return seen, opened, leaves, accepted


@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_let_holds_everything_a_remote_body_meets(theta):
    # brute force: every body of the destination walks the whole remote tree
    # alone; every node it tests must be sent, every node it opens sent with
    # its children, every leaf it lists sent with its bodies, and a node sent
    # alone must be accepted by every body of the destination
    b = inputs.two_plummer(2000, seed=87)
    P = 4
    rank = oracle.orb(b.pos, P)
    rng = np.random.default_rng(4)
    for s in range(P):
        src = rank == s
        for dst in range(P):
            if dst == s:
                continue
            xd = b.pos[rank == dst].astype(np.float32)
            d = oracle.bh_let(b.pos[src], b.mass[src], theta, 16, xd.min(0), xd.max(0))
            kind = d["kind"]
            assert kind[0] != 0
            crit2 = _crit2(b.pos[src], theta)
            alone = np.flatnonzero(kind == 1)
            for p in xd[rng.choice(xd.shape[0], 60, replace=False)]:
                seen, opened, leaves, accepted = _body_walk(d, crit2, p)
                assert np.all(kind[seen] != 0)
                assert np.all(kind[opened] == 2) and np.all(kind[leaves] == 3)
            # every node sent alone passes the opening test for every body
            for u in alone:
                dd = np.maximum(np.maximum(d["lo"][u] - xd, xd - d["hi"][u]), np.float32(0))
                d2 = ((dd[:, 0] * dd[:, 0]) + (dd[:, 1] * dd[:, 1])) + (dd[:, 2] * dd[:, 2])
                assert np.all(d2 >= crit2[d["level"][u]])
            # a sent node's children are sent exactly when it is opened
            for u in range(kind.size):
                kids = [k for k in d["child"][u] if k >= 0]
                if kind[u] == 2:
                    assert kids and np.all(kind[kids] != 0)
                elif kids:
                    assert np.all(kind[kids] == 0)


def test_let_of_a_far_destination_is_the_root_alone():
    b = inputs.plummer(1000, seed=88)
    far = np.array([1e4, 0.0, 0.0], dtype=np.float32)
    d = oracle.bh_let(b.pos, b.mass, 0.5, 16, far, far + 1)
    assert d["kind"][0] == 1 and np.all(d["kind"][1:] == 0)
