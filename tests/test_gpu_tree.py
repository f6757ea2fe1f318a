"""GPU Barnes-Hut tree code (paper Sec. IV-A) against the oracle's tree code.

Both sides build the same octree and take the same opening decisions (the
acceptance test is float32 arithmetic written out identically), so the cells
and bodies each body meets must agree exactly; the accelerations agree to
the float32 walk's rounding.  With theta = 0 the tree walk is the direct sum.
"""
import numpy as np
import pytest

import oracle
from helpers import host, relerr_per_body, to_dev
from paper_1211_2292_gb300 import inputs, nbody

pytestmark = pytest.mark.gpu

RMS_TOL, MAX_TOL = 1e-5, 1e-4  # float32 pair terms, as the direct-sum float32 forms


def _gpu_tree(cuda, b, G, eps, theta, leaf_cap, prec="fp32_comp", group=64):
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, prec) as nb:
        a, cnt = nb.tree_forces(x, m, G, eps, theta, leaf_cap, counts=True, group=group)
        nb.sync()
        st = nb.tree_stats()
    return host(a), host(cnt).astype(np.int64), st


@pytest.mark.parametrize("group", [32, 64])
@pytest.mark.parametrize("n,theta,leaf_cap", [(1000, 0.5, 16), (4099, 0.7, 8), (20000, 0.5, 16),
                                              (20000, 0.3, 32), (777, 1.0, 1)])
def test_matches_oracle_tree(cuda, n, theta, leaf_cap, group):
    b = inputs.plummer(n, seed=61)
    a, cnt, st = _gpu_tree(cuda, b, 1.0, 0.01, theta, leaf_cap, group=group)
    ref, rst, rcnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.01, theta, leaf_cap, group,
                                      counts=True)
    assert np.array_equal(cnt, rcnt)
    assert st == rst
    e = relerr_per_body(a, ref)
    assert np.sqrt((e ** 2).mean()) <= RMS_TOL and e.max() <= MAX_TOL


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_grouped_gpu_walk_against_the_per_body_walk(cuda, theta):
    # The paper's walk is per body (the oracle with group = 1); the GPU walks
    # groups of 32 or 64 bodies, accepting a cell only when all of them
    # would.  Against the exact sum, with e_i the per-body relative error:
    # rms(e_gpu) <= rms(e_per_body), max(e_gpu) <= 1.5 max(e_per_body), and
    # per body |a_gpu - a_per_body| / |a_exact| <= 2 max(e_per_body).
    for b, eps in ((inputs.two_plummer(4096, seed=31), 0.002), (inputs.plummer(8000, seed=32), 0.01)):
        ex = oracle.accel(b.pos, b.mass, 1.0, eps)
        pb, _ = oracle.bh_forces(b.pos, b.mass, 1.0, eps, theta, 16, 1)
        e_pb = relerr_per_body(pb, ex)
        for group in (32, 64):
            a, _, _ = _gpu_tree(cuda, b, 1.0, eps, theta, 16, group=group)
            e_g = relerr_per_body(a, ex)
            assert np.sqrt((e_g ** 2).mean()) <= np.sqrt((e_pb ** 2).mean())
            assert e_g.max() <= 1.5 * e_pb.max()
            assert (np.linalg.norm(a - pb, axis=1) / np.linalg.norm(ex, axis=1)).max() \
                <= 2.0 * e_pb.max()


@pytest.mark.parametrize("group", [32, 64])
def test_theta_zero_is_the_direct_sum(cuda, group):
    b = inputs.plummer(3000, seed=62)
    a, cnt, st = _gpu_tree(cuda, b, 1.0, 0.01, 0.0, 16, group=group)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    assert np.all(cnt[:, 0] == 0) and np.all(cnt[:, 1] == b.n)
    assert st["cell_interactions"] == 0 and st["body_interactions"] == b.n * b.n
    e = relerr_per_body(a, ref)
    assert np.sqrt((e ** 2).mean()) <= RMS_TOL and e.max() <= MAX_TOL


def test_two_clusters_and_every_precision_mode(cuda):
    # Two distant clusters: whole subtrees are accepted as monopoles.
    b = inputs.two_plummer(2500, seed=63)
    ref, _, rcnt = oracle.bh_forces(b.pos, b.mass, 1.0, 0.005, 0.6, 16, 64, counts=True)
    for prec in ("fp64", "fp32", "fp32_comp"):
        a, cnt, _ = _gpu_tree(cuda, b, 1.0, 0.005, 0.6, 16, prec)
        assert np.array_equal(cnt, rcnt), prec
        e = relerr_per_body(a, ref)
        assert np.sqrt((e ** 2).mean()) <= RMS_TOL and e.max() <= MAX_TOL, prec


def test_error_against_direct_sum_falls_with_theta(cuda):
    b = inputs.plummer(30000, seed=64)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    rms = []
    for th in (0.8, 0.4, 0.2):
        a, _, _ = _gpu_tree(cuda, b, 1.0, 0.01, th, 16)
        e = relerr_per_body(a, ref)
        rms.append(np.sqrt((e ** 2).mean()))
    assert rms[0] > rms[1] > rms[2] and rms[1] < 1e-3


def test_degenerate_inputs(cuda):
    # all bodies at one point: ext = 0 is read as 1, keys all 0, one chain of
    # single-child cells down to a level-10 leaf holding every body
    pos = np.zeros((100, 3)) + 0.25
    m = np.full(100, 0.01)
    b = inputs.Bodies(pos, np.zeros_like(pos), m)
    a, cnt, st = _gpu_tree(cuda, b, 1.0, 0.1, 0.5, 4)
    _, rst, rcnt = oracle.bh_forces(pos, m, 1.0, 0.1, 0.5, 4, 64, counts=True)
    assert np.all(a == 0) and np.array_equal(cnt, rcnt) and st == rst and st["nodes"] == 11
    # one body; a pair with zero softening (self pair skipped); ragged sizes
    for n, eps, group in ((1, 0.1, 64), (2, 0.0, 64), (33, 0.0, 32), (33, 0.0, 64),
                          (65, 0.0, 64), (100, 0.01, 32)):
        bb = inputs.random_system(n, seed=65 + n)
        a, cnt, _ = _gpu_tree(cuda, bb, 1.3, eps, 0.5, 1, group=group)
        ref, _, rcnt = oracle.bh_forces(bb.pos, bb.mass, 1.3, eps, 0.5, 1, group, counts=True)
        assert np.array_equal(cnt, rcnt) and np.isfinite(a).all()
        if n == 1:
            assert np.all(a == 0)
        else:
            assert relerr_per_body(a, ref).max() <= MAX_TOL


def test_deterministic_and_empty(cuda):
    b = inputs.plummer(5000, seed=66)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a1 = host(nb.tree_forces(x, m, 1.0, 0.01, 0.5, 16))
        a2 = host(nb.tree_forces(x, m, 1.0, 0.01, 0.5, 16))
        e = nb.tree_forces(x[:0], m[:0], 1.0, 0.01, 0.5, 16)
        nb.sync()
    assert np.array_equal(a1, a2) and e.shape == (0, 3)


def test_argument_checks(cuda):
    import torch
    b = inputs.plummer(64, seed=67)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    a = torch.empty((64, 3), dtype=torch.float64, device=cuda)
    with nbody.NBody(64, "fp32_comp") as nb:
        lib, before = nb.lib, nb.launches
        args = (nb.h, 64, x.data_ptr(), m.data_ptr(), 1.0, 0.01)
        assert lib.nb_tree_forces(*args, -0.1, 16, 64, a.data_ptr(), None) == 1
        assert lib.nb_tree_forces(*args, float("inf"), 16, 64, a.data_ptr(), None) == 1
        assert lib.nb_tree_forces(*args, 0.5, 0, 64, a.data_ptr(), None) == 1
        assert lib.nb_tree_forces(*args, 0.5, 65537, 64, a.data_ptr(), None) == 1
        assert lib.nb_tree_forces(*args, 0.5, 16, 48, a.data_ptr(), None) == 1
        assert lib.nb_tree_forces(nb.h, 65, x.data_ptr(), m.data_ptr(), 1.0, 0.01, 0.5, 16, 64,
                                  a.data_ptr(), None) == 1
        assert nb.launches == before


def test_tree_step_matches_oracle_kdk_at_theta_zero(cuda):
    b = inputs.plummer(2000, seed=68)
    xr, vr, _ = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 10)
    x, v, m = (to_dev(t, cuda) for t in (b.pos, b.vel, b.mass))
    acc = to_dev(np.zeros((b.n, 3)), cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        nb.tree_step(x, v, m, 1.0, 0.01, 0.0, 16, 1e-3, 10, acc)
        nb.sync()
    assert np.abs(host(x) - xr).max() <= 1e-9
    assert np.abs(host(v) - vr).max() <= 1e-6


def test_tree_step_graph_equals_eager(cuda):
    b = inputs.plummer(6000, seed=69)
    outs = []
    for graph, group in ((False, 64), (True, 64), (True, 64), (False, 32), (True, 32)):
        x, v, m = (to_dev(t, cuda) for t in (b.pos, b.vel, b.mass))
        acc = to_dev(np.zeros((b.n, 3)), cuda)
        with nbody.NBody(b.n, "fp32_comp") as nb:
            nb.tree_step(x, v, m, 1.0, 0.01, 0.6, 16, 1e-3, 3, acc, graph=graph, group=group)
            nb.tree_step(x, v, m, 1.0, 0.01, 0.6, 16, 1e-3, 3, acc, acc_valid=True, graph=graph,
                         group=group)
            nb.sync()
        outs.append((host(x), host(v), host(acc)))
    for ref, o in ((0, 1), (0, 2), (3, 4)):
        for p, q in zip(outs[ref], outs[o]):
            assert np.array_equal(p, q)
    # The two group sizes accept different cells, so they differ by the
    # approximation error itself (a few 1e-3 of |a| at theta 0.6, |a| < 10
    # here): over 6 steps of 1e-3, |dx| <= 0.5 * 0.03 * (6e-3)^2 ~ 5e-7.
    assert np.abs(outs[0][0] - outs[3][0]).max() <= 1e-6


def test_schedules_give_identical_results(cuda):
    # static / dynamic / guided dealing of the groups changes only the time
    b = inputs.two_plummer(6000, seed=70)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    outs = []
    with nbody.NBody(b.n, "fp32_comp") as nb:
        for sched, chunk in (("static", 1), ("dynamic", 1), ("dynamic", 7), ("guided", 1),
                             ("guided", 3)):
            nb.tree_schedule(sched, chunk)
            for group in (32, 64):
                a, c = nb.tree_forces(x, m, 1.0, 0.01, 0.5, 16, counts=True, group=group)
                outs.append((group, host(a), host(c)))
        with pytest.raises(nbody.NBodyError):
            nb.tree_schedule(3, 1)
        with pytest.raises(nbody.NBodyError):
            nb.tree_schedule("dynamic", 0)
    for group in (32, 64):
        ref = [o for o in outs if o[0] == group]
        for o in ref[1:]:
            assert np.array_equal(o[1], ref[0][1]) and np.array_equal(o[2], ref[0][2])


def _both(cuda, pos, mass, G, eps, theta, leaf_cap, group):
    b = inputs.Bodies(pos, np.zeros_like(pos), mass)
    a, cnt, st = _gpu_tree(cuda, b, G, eps, theta, leaf_cap, group=group)
    ref, rst, rcnt = oracle.bh_forces(pos, mass, G, eps, theta, leaf_cap, group, counts=True)
    return a, cnt, st, ref, rcnt, rst


@pytest.mark.parametrize("group", [32, 64])
def test_shapes_the_tree_can_take(cuda, group):
    rng = np.random.default_rng(71)
    # a flat disc (one axis constant), a single leaf holding everything,
    # a dense clump that reaches level 10 with more than leaf_cap bodies,
    # and massless bodies (cells of zero mass keep their centre at 0).  The
    # clump runs at eps = 0.1: for pairs closer than eps a float32 form errs
    # by about m * ulp(|x - origin|) / eps^3 per pair, which at eps = 0.01 and
    # 300 coincident bodies of mass 4e-4 reaches 5e-3 of |a| in the direct
    # float32 kernel as well (an input for the float64 form, not a tree issue).
    disc = np.column_stack([rng.normal(size=(3000, 2)), np.zeros(3000)])
    clump = np.vstack([rng.normal(size=(2000, 3)), 1e-9 * rng.normal(size=(300, 3)) + 0.3])
    cases = [
        (disc, rng.uniform(0.5, 1.5, 3000) / 3000, 0.5, 16),
        (rng.normal(size=(500, 3)), rng.uniform(0.5, 1.5, 500) / 500, 0.5, 1000),
        (clump, rng.uniform(0.5, 1.5, 2300) / 2300, 0.5, 8),
        (rng.normal(size=(2000, 3)), np.where(rng.random(2000) < 0.3, 0.0, 1.0 / 2000), 0.6, 4),
    ]
    for k, (pos, mass, theta, lc) in enumerate(cases):
        eps = 0.1 if k == 2 else 0.01
        a, cnt, st, ref, rcnt, rst = _both(cuda, pos, mass, 1.0, eps, theta, lc, group)
        assert np.array_equal(cnt, rcnt) and st == rst
        # error against the rms acceleration (the disc has bodies of near-zero
        # |a| at its centre, where a per-body ratio is ill-conditioned)
        rms = np.sqrt((np.linalg.norm(ref, axis=1) ** 2).mean())
        e = np.linalg.norm(a - ref, axis=1) / rms
        assert e.max() <= MAX_TOL and np.sqrt((e ** 2).mean()) <= RMS_TOL
    # one leaf: the walk is the direct sum for every body
    _, cnt, st, _, _, _ = _both(cuda, cases[1][0], cases[1][1], 1.0, 0.01, 0.5, 1000, group)
    assert st["nodes"] == 1 and np.all(cnt[:, 1] == 500) and np.all(cnt[:, 0] == 0)
