"""Pins of the oracle's fast multipole method (the O(N) successor of the tree
code, paper Sec. VI) against closed forms, calculus and the direct sum."""
import math

import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs


def _err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _slot(p):
    return {n: q for q, n in enumerate(oracle.fmm_multi_indices(p))}


def test_slot_order():
    mi = oracle.fmm_multi_indices(6)
    assert len(mi) == 84 and len(set(mi)) == 84
    assert [sum(n) for n in mi] == sorted(sum(n) for n in mi)
    assert mi[:4] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def test_derivatives_closed_forms():
    # g = 1/s, s^2 = |r|^2 + eps^2: grad g = -r/s^3,
    # d_a d_b g = 3 r_a r_b / s^5 - delta_ab / s^3.
    r, eps = np.array([0.3, -0.7, 1.1]), 0.25
    T = oracle.fmm_deriv(2, r, eps)
    ix = _slot(2)
    s = math.sqrt(r @ r + eps * eps)
    assert T[ix[(0, 0, 0)]] == pytest.approx(1 / s, rel=1e-15)
    for c in range(3):
        e = [0, 0, 0]
        e[c] = 1
        assert T[ix[tuple(e)]] == pytest.approx(-r[c] / s ** 3, rel=1e-14)
    for a in range(3):
        for b in range(3):
            n = [0, 0, 0]
            n[a] += 1
            n[b] += 1
            expect = 3 * r[a] * r[b] / s ** 5 - (1.0 if a == b else 0.0) / s ** 3
            assert T[ix[tuple(n)]] == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("eps", [0.0, 0.4])
def test_derivatives_finite_differences(eps):
    # every order against the next: d_c T_n = T_{n + e_c}, fourth-order
    # central differences of the lower order.
    p = 7
    r = np.array([0.9, -0.5, 0.65])
    ix = _slot(p)
    T0 = oracle.fmm_deriv(p, r, eps)
    h = 1e-3
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        f = [oracle.fmm_deriv(p, r + k * e, eps) for k in (-2, -1, 1, 2)]
        d = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        for n, q in ix.items():
            if sum(n) == p:
                continue
            up = list(n)
            up[c] += 1
            exact = T0[ix[tuple(up)]]
            scale = np.abs([T0[ix[m]] for m in ix if sum(m) == sum(n) + 1]).max()
            assert abs(d[q] - exact) <= 1e-7 * scale, (n, c)


def test_derivatives_harmonic_without_softening():
    # 1/|r| is harmonic: sum_c T_{n + 2 e_c} = 0 for every n.
    p = 9
    r = np.array([-0.4, 0.8, 0.55])
    ix = _slot(p)
    T = oracle.fmm_deriv(p, r, 0.0)
    for n in ix:
        if sum(n) > p - 2:
            continue
        lap = sum(T[ix[tuple(n[a] + 2 * (a == c) for a in range(3))]] for c in range(3))
        scale = np.abs([T[ix[m]] for m in ix if sum(m) == sum(n) + 2]).max()
        assert abs(lap) <= 1e-13 * scale, n


def _pair_case(delta, rng_seed=7):
    rng = np.random.default_rng(rng_seed)
    zA, zB = np.array([1.2, -0.4, 0.7]), np.array([-0.3, 0.2, -0.5])
    xs = zB + delta * rng.uniform(-1, 1, (12, 3))
    ms = rng.uniform(0.5, 1.5, 12)
    xt = zA + delta * rng.uniform(-1, 1, (5, 3))
    return zA, zB, xs, ms, xt


def _direct(xs, ms, xt, eps):
    d = xs[None, :, :] - xt[:, None, :]
    s2 = (d * d).sum(-1) + eps * eps
    return (ms[None, :, None] * d / (s2 * np.sqrt(s2))[..., None]).sum(1)


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_expansion_order_of_accuracy(eps):
    # The expansions truncate at total order p in the source and target
    # offsets, so the force error of a cluster pair shrinks as delta^p when
    # both clusters shrink by delta: halving them divides it by 2^p.  A wrong
    # or missing term of any order q < p would show as 2^q.
    for p in range(1, 9):
        errs = []
        for delta in (0.08, 0.04):
            zA, zB, xs, ms, xt = _pair_case(delta)
            a = oracle.fmm_pair(p, zA, zB, eps, xs, ms, xt)
            errs.append(np.abs(a - _direct(xs, ms, xt, eps)).max())
        ratio = errs[0] / errs[1]
        assert 0.75 * 2 ** p <= ratio <= 1.35 * 2 ** p, (p, ratio)


def test_expansion_converges_to_the_direct_sum():
    zA, zB, xs, ms, xt = _pair_case(0.25)
    ref = _direct(xs, ms, xt, 0.1)
    e = [np.abs(oracle.fmm_pair(p, zA, zB, 0.1, xs, ms, xt) - ref).max() / np.abs(ref).max()
         for p in range(1, 13)]
    # each order gains at least a factor 2 (the offsets reach 0.43 of the
    # centres' distance), twelve orders more than 1e6
    assert all(b < a / 2 for a, b in zip(e, e[1:]))
    assert e[-1] < 1e-6 * e[0]


@pytest.mark.parametrize("leaf_cap,p", [(1, 1), (8, 4), (16, 6), (64, 3)])
def test_theta_zero_is_the_direct_sum(leaf_cap, p):
    # theta = 0 separates no pair of cells: every pair interacts directly.
    b = inputs.plummer(2500, seed=61)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    a, st, cnt = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.01, 0.0, p, leaf_cap, counts=True)
    assert _err(a, ref).max() <= 1e-13
    assert st["expansions"] == 0 and st["direct_pairs"] == b.n ** 2
    assert np.all(cnt[:, 0] == 0) and np.all(cnt[:, 2] == b.n)


@pytest.mark.parametrize("theta", [0.3, 0.6, 0.95])
def test_every_body_meets_every_other_once(theta):
    b = inputs.two_plummer(6000, seed=62)
    _, st, cnt = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.01, theta, 3, 12, counts=True)
    assert np.all(cnt[:, 1] + cnt[:, 2] == b.n)
    assert np.all(cnt[:, 2] >= 1)
    assert st["direct_pairs"] == cnt[:, 2].sum()
    assert st["expansions"] > 0


def test_power_of_two_scaling_is_exact():
    # x -> 2x, eps -> 2 eps, m -> 8m: every expansion term scales by a power
    # of two, and a by exactly 2.
    b = inputs.plummer(3000, seed=63)
    a1, _ = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.02, 0.5, 5, 16)
    a2, _ = oracle.fmm_forces(2 * b.pos, 8 * b.mass, 1.0, 0.04, 0.5, 5, 16)
    assert np.array_equal(a2, 2 * a1)


def test_error_falls_with_theta_and_order():
    b = inputs.plummer(8000, seed=64)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    rms = {}
    for th in (0.6, 0.4):
        for p in (2, 4, 6):
            a, _ = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.01, th, p, 16)
            rms[th, p] = float(np.sqrt((_err(a, ref) ** 2).mean()))
    for th in (0.6, 0.4):
        assert rms[th, 2] > rms[th, 4] > rms[th, 6]
    for p in (2, 4, 6):
        assert rms[0.4, p] < rms[0.6, p]
    assert rms[0.4, 6] < 1e-4 and rms[0.6, 4] < 1e-2


def test_far_cluster_through_expansions_only():
    # A tight cluster in one corner of the root cube and a light body in the
    # opposite one: the body meets the cluster only through a source cell's
    # expansion acting on its (large) leaf, and sits at that leaf's corner,
    # where the local polynomial converges slowest: the error falls with p,
    # at least by 0.6 per order on average (the offsets' sum is 0.45 of the
    # centres' distance here).
    rng = np.random.default_rng(5)
    cl = rng.uniform(-1e-4, 1e-4, (30, 3))
    x = np.vstack([cl, [[40.0, 40.0, 40.0]]])
    m = np.append(rng.uniform(0.5, 1.5, 30), 1e-3)
    ref = oracle.accel(x, m, 1.0, 0.0)
    e = []
    for p in (2, 4, 8, 12):
        a, _, cnt = oracle.fmm_forces(x, m, 1.0, 0.0, 0.5, p, 4, counts=True)
        assert list(cnt[-1]) == [1, 30, 1]
        e.append(_err(a[-1:], ref[-1:])[0])
    assert all(b < a for a, b in zip(e, e[1:]))
    assert e[-1] < 0.6 ** 10 * e[0]


def test_bad_arguments():
    b = inputs.plummer(10, seed=1)
    for th, p, lc in ((0.5, 0, 16), (0.5, 13, 16), (0.5, 4, 0), (-0.1, 4, 16), (np.nan, 4, 16)):
        with pytest.raises(ValueError):
            oracle.fmm_forces(b.pos, b.mass, 1.0, 0.01, th, p, lc)
    a, st = oracle.fmm_forces(np.zeros((0, 3)), np.zeros(0), 1.0, 0.1, 0.5, 4, 16)
    assert a.shape == (0, 3)
    a, st = oracle.fmm_forces(b.pos[:1], b.mass[:1], 1.0, 0.1, 0.5, 4, 16)
    assert np.array_equal(a, np.zeros((1, 3)))
    with pytest.raises(ValueError):
        oracle.fmm_deriv(13, np.ones(3))
