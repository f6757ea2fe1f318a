"""Pins of the oracle's Barnes-Hut tree code (paper Sec. IV-A) against the
direct sum and against closed forms it does not contain."""
import math

import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs


def _err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("leaf_cap,group", [(1, 1), (8, 32), (16, 32), (64, 7)])
def test_theta_zero_is_the_direct_sum(leaf_cap, group):
    # theta = 0 opens every cell: each body meets every other body directly.
    b = inputs.plummer(3000, seed=51)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    a, st, cnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, 0.0, leaf_cap, group, counts=True)
    assert _err(a, ref).max() <= 1e-13
    assert st["cell_interactions"] == 0 and np.all(cnt[:, 0] == 0) and np.all(cnt[:, 1] == b.n)
    assert st["leaves"] <= st["nodes"]


def test_error_falls_with_theta():
    b = inputs.plummer(8000, seed=52)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    rms = []
    for th in (0.8, 0.4, 0.2, 0.1):
        a, st = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, th, 16, 32)
        e = _err(a, ref)
        rms.append(np.sqrt((e ** 2).mean()))
    assert all(r1 < r0 for r0, r1 in zip(rms, rms[1:]))
    assert rms[1] < 1e-3 and rms[3] < 1e-4


def test_far_cluster_is_its_monopole():
    # A compact cluster far from one test body: the cell holding the cluster
    # is accepted and acts as its total mass at its centre of mass.
    rng = np.random.default_rng(3)
    cl = rng.uniform(0.0, 0.01, (40, 3))
    mc = rng.uniform(0.5, 1.5, 40)
    x = np.vstack([cl, [[1.0, 1.0, 1.0]]])
    m = np.append(mc, 1e-3)
    a, st, cnt = oracle.bh_forces(x, m, 1.3, 0.05, 0.5, 8, 1, counts=True)
    com = (mc[:, None] * cl).sum(0) / mc.sum()
    d = com - x[-1]
    s2 = d @ d + 0.05 ** 2
    expect = 1.3 * mc.sum() * d / (s2 * math.sqrt(s2))
    assert cnt[-1, 0] == 1 and cnt[-1, 1] == 1  # one cell, and its own leaf
    np.testing.assert_allclose(a[-1], expect, rtol=1e-13)


def test_tree_counts_and_cost():
    b = inputs.plummer(20000, seed=53)
    _, st, cnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, 0.5, 16, 32, counts=True)
    assert st["cell_interactions"] == cnt[:, 0].sum()
    assert st["body_interactions"] == cnt[:, 1].sum()
    # every body meets its own leaf, and far fewer partners than N
    assert np.all(cnt[:, 1] >= 1)
    assert (cnt.sum(1)).mean() < 0.5 * b.n


def test_bad_arguments():
    b = inputs.plummer(10, seed=1)
    with pytest.raises(ValueError):
        oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, 0.5, 0, 32)
    a, st = oracle.bh_forces(np.zeros((0, 3)), np.zeros(0), 1.0, 0.1, 0.5, 16, 32)
    assert a.shape == (0, 3)


def test_group_subset_equals_the_full_run():
    # The subset walk reuses the full tree: its bodies, lists and sums must be
    # those of the full run exactly, and idx must list the groups' bodies in
    # key order (consecutive groups tile the bodies once).
    b = inputs.plummer(3001, seed=54)
    a, _, cnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, 0.6, 8, 64, counts=True)
    ngroups = (b.n + 63) // 64
    idx, a2, c2 = oracle.bh_groups(b.pos, b.mass, 1.0, 0.01, 0.6, 8, 64, np.arange(ngroups))
    flat = idx.ravel()
    assert np.array_equal(np.sort(flat[flat >= 0]), np.arange(b.n))
    assert np.array_equal(a2, a) and np.array_equal(c2, cnt)
    sel = np.array([ngroups - 1, 3])
    idx, a3, c3 = oracle.bh_groups(b.pos, b.mass, 1.0, 0.01, 0.6, 8, 64, sel)
    assert (idx[0] >= 0).sum() == b.n - 64 * (ngroups - 1) and (idx[1] >= 0).all()
    ii = idx[idx >= 0]
    assert np.array_equal(a3[ii], a[ii]) and np.isnan(a3[np.setdiff1d(np.arange(b.n), ii)]).all()
    with pytest.raises(ValueError):
        oracle.bh_groups(b.pos, b.mass, 1.0, 0.01, 0.6, 8, 64, [ngroups])


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_grouped_walk_is_a_refinement_of_the_per_body_walk(theta):
    # group = 1 is the per-body walk the paper describes.  A group accepts a
    # cell only when every one of its bodies would, so each body's grouped
    # list refines its per-body list: more cells opened, fewer bodies
    # approximated.  Stated bounds, against the exact sum (per-body relative
    # error e_i): rms(e_grouped) <= rms(e_per_body), max(e_grouped) <=
    # 1.5 max(e_per_body), and per body |a_grouped - a_per_body| / |a_exact|
    # <= 2 max(e_per_body) (measured up to 1.35 on these inputs).
    for b, eps in ((inputs.two_plummer(4096, seed=31), 0.002), (inputs.plummer(8000, seed=32), 0.01)):
        ex = oracle.accel(b.pos, b.mass, 1.0, eps)
        pb, st1, c1 = oracle.bh_forces(b.pos, b.mass, 1.0, eps, theta, 16, 1, counts=True)
        e_pb = _err(pb, ex)
        for group in (32, 64):
            ag, stg, cg = oracle.bh_forces(b.pos, b.mass, 1.0, eps, theta, 16, group, counts=True)
            e_g = _err(ag, ex)
            assert np.sqrt((e_g ** 2).mean()) <= np.sqrt((e_pb ** 2).mean())
            assert e_g.max() <= 1.5 * e_pb.max()
            assert (np.linalg.norm(ag - pb, axis=1) / np.linalg.norm(ex, axis=1)).max() \
                <= 2.0 * e_pb.max()
            # a refinement meets at least as many bodies directly
            assert np.all(cg[:, 1] >= c1[:, 1])

