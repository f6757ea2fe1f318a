"""Pins of the FP64 oracle against mathematics it does not contain.

Every check here comes from outside the oracle's own code: closed forms
(two-body and three-body configurations, circular and Kepler orbits, the
Plummer potential energy), exact invariants (Newton's third law, power-of-two
scaling laws, rotation/translation/permutation equivariance), the potential
whose gradient the force must be, brute force at 50 digits on tiny systems,
finite differences, and an independent derivative by torch autograd.  They are
chosen so that a dropped term, a wrong sign, a wrong power of s or a swapped
index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- force sum

def test_two_body_closed_form():
    # Two bodies on the x axis: a_1 = G m_2 r / (r^2+eps^2)^{3/2} toward body 2.
    G, eps, r, m1, m2 = 1.7, 0.3, 2.5, 0.25, 0.75
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    a = oracle.accel(x, np.array([m1, m2]), G, eps)
    k = r / (r * r + eps * eps) ** 1.5
    np.testing.assert_allclose(a[0], [G * m2 * k, 0, 0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(a[1], [-G * m1 * k, 0, 0], rtol=1e-15, atol=0)


def test_two_body_zero_softening():
    # eps = 0: the self pair must be skipped (no 0/0), Newton's 1/r^2 law.
    x = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    a = oracle.accel(x, np.array([1.0, 3.0]), 1.0, 0.0)
    np.testing.assert_allclose(a, [[0, 0.75, 0], [0, -0.25, 0]], rtol=1e-15, atol=0)


def test_equilateral_triangle():
    # Three equal masses on a triangle of side L: each is pulled toward the
    # centroid with magnitude sqrt(3) G m L / (L^2 + eps^2)^{3/2}.
    G, m, L, eps = 1.0, 0.4, 1.3, 0.05
    ang = np.array([90.0, 210.0, 330.0]) * math.pi / 180
    R = L / math.sqrt(3)
    x = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros(3)], axis=1)
    a = oracle.accel(x, np.full(3, m), G, eps)
    mag = math.sqrt(3) * G * m * L / (L * L + eps * eps) ** 1.5
    expect = -mag * x / R
    np.testing.assert_allclose(a, expect, rtol=1e-13, atol=1e-15)


def test_single_body_and_empty():
    assert oracle.accel(np.zeros((0, 3)), np.zeros(0), 1.0, 0.1).shape == (0, 3)
    a = oracle.accel(np.array([[1.0, 2.0, 3.0]]), np.array([2.0]), 1.0, 0.1)
    assert np.all(a == 0)


@pytest.mark.parametrize("n,eps", [(2, 0.0), (5, 0.01), (8, 0.3)])
def test_brute_force_50_digits(n, eps):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    b = inputs.random_system(n, seed=n)
    G = 1.25
    a = oracle.accel(b.pos, b.mass, G, eps)
    X = [[mpmath.mpf(float(v)) for v in row] for row in b.pos]
    M = [mpmath.mpf(float(v)) for v in b.mass]
    e2 = mpmath.mpf(eps) ** 2
    for i in range(n):
        acc = [mpmath.mpf(0)] * 3
        for j in range(n):
            if i == j:
                continue
            d = [X[j][c] - X[i][c] for c in range(3)]
            s2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + e2
            f = M[j] / (s2 * mpmath.sqrt(s2))
            acc = [acc[c] + f * d[c] for c in range(3)]
        ref = np.array([float(G * acc[c]) for c in range(3)])
        assert np.linalg.norm(a[i] - ref) <= 1e-14 * np.linalg.norm(ref)


def test_newton_third_law():
    b = inputs.plummer(2048, seed=5)
    a = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    net = (b.mass[:, None] * a).sum(0)
    scale = (b.mass * np.linalg.norm(a, axis=1)).sum()
    assert np.linalg.norm(net) <= 1e-13 * scale


def test_power_of_two_scaling_is_exact():
    # Lengths (x and eps) times 2 -> a / 4 exactly; masses or G times 2 ->
    # a * 2 exactly.  A wrong power of s or a dropped mass factor breaks these.
    b = inputs.random_system(40, seed=11)
    a = oracle.accel(b.pos, b.mass, 1.0, 0.05)
    assert np.array_equal(oracle.accel(2 * b.pos, b.mass, 1.0, 0.1), a / 4)
    assert np.array_equal(oracle.accel(b.pos, 2 * b.mass, 1.0, 0.05), 2 * a)
    assert np.array_equal(oracle.accel(b.pos, b.mass, 2.0, 0.05), 2 * a)


def test_rotation_translation_permutation():
    b = inputs.random_system(60, seed=12)
    a = oracle.accel(b.pos, b.mass, 1.0, 0.02)
    q, _ = np.linalg.qr(np.random.default_rng(0).normal(size=(3, 3)))
    ar = oracle.accel(b.pos @ q.T, b.mass, 1.0, 0.02)
    np.testing.assert_allclose(ar, a @ q.T, rtol=0, atol=1e-12 * np.abs(a).max())
    at = oracle.accel(b.pos + np.array([0.5, -0.25, 0.125]), b.mass, 1.0, 0.02)
    np.testing.assert_allclose(at, a, rtol=0, atol=1e-12 * np.abs(a).max())
    p = np.random.default_rng(1).permutation(60)
    ap = oracle.accel(b.pos[p], b.mass[p], 1.0, 0.02)
    np.testing.assert_allclose(ap, a[p], rtol=0, atol=1e-13 * np.abs(a).max())


def test_monopole_far_field():
    # A compact cluster (radius 1e-2, centre of mass at the origin) seen from
    # R = 10: a = G M / R^2 up to quadrupole terms of order (1e-2/10)^2.
    rng = np.random.default_rng(3)
    cl = rng.uniform(-1e-2, 1e-2, (50, 3))
    mc = rng.uniform(0.5, 1.5, 50)
    cl -= (mc[:, None] * cl).sum(0) / mc.sum()
    x = np.vstack([cl, [[10.0, 0.0, 0.0]]])
    m = np.append(mc, 1e-3)
    a = oracle.accel(x, m, 1.0, 0.0)[-1]
    expect = np.array([-mc.sum() / 100.0, 0.0, 0.0])
    assert np.linalg.norm(a - expect) <= 3e-6 * np.linalg.norm(expect)


def test_force_is_minus_gradient_of_potential():
    # m_i a_i = -dE_pot/dx_i.  The potential uses 1/s over i<j, the force
    # d/s^3 over j != i, so a slip in either disagrees with this derivative.
    b = inputs.random_system(7, seed=13)
    G, eps, h = 1.3, 0.07, 1e-5
    a = oracle.accel(b.pos, b.mass, G, eps)
    for i in range(b.n):
        for c in range(3):
            xp = b.pos.copy(); xp[i, c] += h
            xm = b.pos.copy(); xm[i, c] -= h
            ep = oracle.energy(xp, b.vel, b.mass, G, eps)[1]
            em = oracle.energy(xm, b.vel, b.mass, G, eps)[1]
            grad = (ep - em) / (2 * h)
            assert abs(-grad - b.mass[i] * a[i, c]) <= 1e-8 * np.abs(b.mass[:, None] * a).max()


def test_rows_match_full():
    b = inputs.plummer(700, seed=6)
    rows = np.array([0, 5, 699, 350, 5])
    full = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    part = oracle.accel_rows(b.pos, b.mass, rows, 1.0, 0.01)
    assert np.array_equal(part, full[rows])


def test_energy_closed_forms():
    # Two bodies at rest: E_pot = -G m1 m2 / sqrt(r^2 + eps^2); E_kin from v.
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    m = np.array([2.0, 0.5])
    e = oracle.energy(x, v, m, 1.5, 0.5)
    np.testing.assert_allclose(e[0], 0.5 * 2 * 1 + 0.5 * 0.5 * 4, rtol=1e-15)
    np.testing.assert_allclose(e[1], -1.5 * 1.0 / math.sqrt(25.25), rtol=1e-15)
    np.testing.assert_allclose(e[2], e[0] + e[1], rtol=1e-15)
    np.testing.assert_allclose(e[3:6], [2.0, 0.0, 1.0], rtol=1e-15)
    assert np.abs(e[6:9]).max() < 1e-15


# --------------------------------------------------------------- integrator

def _circular_pair(m=0.5, r=1.0, eps=0.1, G=1.0):
    w = math.sqrt(2 * G * m / (r * r + eps * eps) ** 1.5)
    x = np.array([[-r / 2, 0, 0], [r / 2, 0, 0]], dtype=float)
    v = np.array([[0, -w * r / 2, 0], [0, w * r / 2, 0]], dtype=float)
    return x, v, np.array([m, m]), w


def test_circular_orbit_phase_error_is_second_order():
    # Softened circular two-body orbit: omega^2 = 2 G m / (r^2+eps^2)^{3/2}
    # exactly for any eps.  KDK keeps it circular; its phase error is O(dt^2).
    x, v, m, w = _circular_pair()
    T = 3.0
    errs = []
    for dt in (0.02, 0.01, 0.005):
        xs, _, _ = oracle.kdk(x, v, m, 1.0, 0.1, dt, int(round(T / dt)))
        d = xs[1] - xs[0]
        ph = math.atan2(d[1], d[0])
        errs.append(abs((ph - w * T + math.pi) % (2 * math.pi) - math.pi))
        assert abs(np.linalg.norm(d) - 1.0) < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


def _kepler_relative(t, a=1.0, e=0.5, mu=1.0):
    # Kepler's equation E - e sin E = n t, solved by Newton's method.
    n = math.sqrt(mu / a ** 3)
    M = n * t
    E = M
    for _ in range(50):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def test_kepler_orbit_zero_softening():
    # eps = 0, eccentricity 0.5, G (m1+m2) = 1, started at pericentre.
    m = np.array([0.3, 0.7])
    e, a_k = 0.5, 1.0
    rp = a_k * (1 - e)
    vp = math.sqrt((1 + e) / (a_k * (1 - e)))
    rel_x = np.array([rp, 0, 0]); rel_v = np.array([0, vp, 0])
    x = np.stack([-m[1] * rel_x, m[0] * rel_x])
    v = np.stack([-m[1] * rel_v, m[0] * rel_v])
    T = 2.0
    errs = []
    for dt in (2e-3, 1e-3):
        xs, _, _ = oracle.kdk(x, v, m, 1.0, 0.0, dt, int(round(T / dt)))
        errs.append(np.linalg.norm((xs[1] - xs[0]) - _kepler_relative(T)))
    assert errs[1] < 1e-5
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_time_reversibility():
    b = inputs.plummer(64, seed=7)
    x1, v1, _ = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 100)
    x2, v2, _ = oracle.kdk(x1, -v1, b.mass, 1.0, 0.01, 1e-3, 100)
    assert np.abs(x2 - b.pos).max() < 1e-12
    assert np.abs(-v2 - b.vel).max() < 1e-11


def test_energy_error_second_order_and_bounded():
    # Eccentric softened pair: the KDK energy error scales as dt^2 and does
    # not grow secularly over many orbits.
    m = np.array([0.5, 0.5])
    x = np.array([[-0.25, 0, 0], [0.25, 0, 0]])
    v = np.array([[0, -0.9, 0], [0, 0.9, 0]])
    eps = 0.05
    e0 = oracle.energy(x, v, m, 1.0, eps)[2]

    def max_err(dt, steps, chunk):
        xs, vs = x, v
        errs = []
        for _ in range(steps // chunk):
            xs, vs, _ = oracle.kdk(xs, vs, m, 1.0, eps, dt, chunk)
            errs.append(abs(oracle.energy(xs, vs, m, 1.0, eps)[2] - e0))
        return np.array(errs)

    e1 = max_err(2e-3, 2000, 10).max()
    e2 = max_err(1e-3, 4000, 20).max()
    assert 3.0 < e1 / e2 < 5.0
    long = max_err(2e-3, 10000, 10)
    assert long[-100:].max() < 2.0 * long[:100].max()


def test_kdk_zero_steps_is_force_only():
    b = inputs.plummer(32, seed=8)
    x, v, a = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 0)
    assert np.array_equal(x, b.pos) and np.array_equal(v, b.vel)
    assert np.array_equal(a, oracle.accel(b.pos, b.mass, 1.0, 0.01))


# ------------------------------------------------------------------ adjoint

def test_force_vjp_central_differences():
    b = inputs.random_system(16, seed=14)
    G, eps, h = 1.1, 0.05, 1e-6
    lam = np.random.default_rng(2).normal(size=(16, 3))
    gx, gm = oracle.force_vjp(b.pos, b.mass, lam, G, eps)

    def L(x, m):
        return float((lam * oracle.accel(x, m, G, eps)).sum())

    fx = np.zeros_like(gx)
    for i in range(16):
        for c in range(3):
            xp = b.pos.copy(); xp[i, c] += h
            xm = b.pos.copy(); xm[i, c] -= h
            fx[i, c] = (L(xp, b.mass) - L(xm, b.mass)) / (2 * h)
    fm = np.zeros_like(gm)
    for i in range(16):
        mp = b.mass.copy(); mp[i] += h
        mm = b.mass.copy(); mm[i] -= h
        fm[i] = (L(b.pos, mp) - L(b.pos, mm)) / (2 * h)
    assert _rel(gx, fx) < 1e-6
    assert _rel(gm, fm) < 1e-6


def _torch_rollout(x, v, m, G, eps, dt, nsteps):
    import torch

    def F(x):
        d = x[None, :, :] - x[:, None, :]            # d[i, j] = x_j - x_i
        s2 = (d * d).sum(-1) + eps * eps
        w = m[None, :] / (s2 * torch.sqrt(s2))
        w = w * (1 - torch.eye(x.shape[0], dtype=x.dtype))
        return G * (w[:, :, None] * d).sum(1)

    a = F(x)
    for _ in range(nsteps):
        v = v + 0.5 * dt * a
        x = x + dt * v
        a = F(x)
        v = v + 0.5 * dt * a
    return x, v, F


def test_force_vjp_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    b = inputs.random_system(12, seed=15)
    G, eps = 0.9, 0.03
    lam = np.random.default_rng(4).normal(size=(12, 3))
    x = torch.tensor(b.pos, requires_grad=True)
    m = torch.tensor(b.mass, requires_grad=True)
    _, _, F = _torch_rollout(x, x, m, G, eps, 0.0, 0)
    (F(x) * torch.tensor(lam)).sum().backward()
    gx, gm = oracle.force_vjp(b.pos, b.mass, lam, G, eps)
    np.testing.assert_allclose(gx, x.grad.numpy(), rtol=1e-10, atol=1e-12 * np.abs(gx).max())
    np.testing.assert_allclose(gm, m.grad.numpy(), rtol=1e-10, atol=1e-12 * np.abs(gm).max())


def test_kdk_grad_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    b = inputs.plummer(10, seed=16)
    G, eps, dt, K = 1.0, 0.05, 1e-2, 25
    tgt = b.pos + 0.01
    x0 = torch.tensor(b.pos, requires_grad=True)
    v0 = torch.tensor(b.vel, requires_grad=True)
    m = torch.tensor(b.mass, requires_grad=True)
    xT, vT, _ = _torch_rollout(x0, v0, m, G, eps, dt, K)
    loss = ((xT - torch.tensor(tgt)) ** 2).sum(-1).mean() + (vT ** 2).sum() * 0.1
    loss.backward()
    xTn, vTn, _ = oracle.kdk(b.pos, b.vel, b.mass, G, eps, dt, K)
    gxT = 2.0 / b.n * (xTn - tgt)
    gvT = 0.2 * vTn
    gx, gv, gm = oracle.kdk_grad(b.pos, b.vel, b.mass, G, eps, dt, K, gxT, gvT)
    assert _rel(gx, x0.grad.numpy()) < 1e-10
    assert _rel(gv, v0.grad.numpy()) < 1e-10
    assert _rel(gm, m.grad.numpy()) < 1e-10


def test_kdk_grad_central_differences():
    b = inputs.plummer(6, seed=17)
    G, eps, dt, K, h = 1.0, 0.05, 1e-2, 10, 1e-6
    tgt = np.zeros_like(b.pos)

    def loss(x, v, m):
        xT, _, _ = oracle.kdk(x, v, m, G, eps, dt, K)
        return ((xT - tgt) ** 2).sum(-1).mean()

    xT, _, _ = oracle.kdk(b.pos, b.vel, b.mass, G, eps, dt, K)
    gx, gv, gm = oracle.kdk_grad(b.pos, b.vel, b.mass, G, eps, dt, K,
                                 2.0 / b.n * (xT - tgt), np.zeros_like(xT))
    for arr, g in ((0, gx), (1, gv)):
        fd = np.zeros_like(g)
        for i in range(b.n):
            for c in range(3):
                args_p = [b.pos.copy(), b.vel.copy(), b.mass]
                args_m = [b.pos.copy(), b.vel.copy(), b.mass]
                args_p[arr][i, c] += h
                args_m[arr][i, c] -= h
                fd[i, c] = (loss(*args_p) - loss(*args_m)) / (2 * h)
        assert _rel(g, fd) < 1e-6
    fdm = np.zeros_like(gm)
    for i in range(b.n):
        mp = b.mass.copy(); mp[i] += h
        mm = b.mass.copy(); mm[i] -= h
        fdm[i] = (loss(b.pos, b.vel, mp) - loss(b.pos, b.vel, mm)) / (2 * h)
    assert _rel(gm, fdm) < 1e-6


# ---------------------------------------------------------------- generator

def test_plummer_radius_distribution_ks():
    scipy_stats = pytest.importorskip("scipy.stats")
    b = inputs.plummer(20000, seed=21)
    r = np.linalg.norm(b.pos, axis=1)
    R = inputs.R_TRUNC
    norm = R ** 3 / (1 + R * R) ** 1.5

    def cdf(x):
        x = np.minimum(x, R)
        return x ** 3 / (1 + x * x) ** 1.5 / norm

    assert scipy_stats.kstest(r, cdf).pvalue > 1e-3
    assert r.max() <= R + 0.05


def test_plummer_virial_and_potential_energy():
    integrate = pytest.importorskip("scipy.integrate")
    n = 16384
    b = inputs.plummer(n, seed=22)
    e = oracle.energy(b.pos, b.vel, b.mass, 1.0, 1e-4)
    q = 2 * e[0] / abs(e[1])
    assert abs(q - 1.0) < 3.0 / math.sqrt(n)
    # Potential energy of the Plummer model truncated at R (mass renormalised
    # to 1): W = -G int M(r) dM(r) / r.  Untruncated this is -3 pi / 32.
    R = inputs.R_TRUNC
    Mr = lambda r: r ** 3 / (1 + r * r) ** 1.5
    dM = lambda r: 3 * r * r / (1 + r * r) ** 2.5
    W = -integrate.quad(lambda r: Mr(r) * dM(r) / r, 0, R)[0] / Mr(R) ** 2
    assert abs(integrate.quad(lambda r: Mr(r) * dM(r) / r, 0, np.inf)[0] - 3 * math.pi / 32) < 1e-10
    assert abs(e[1] - W) < 3.0 / math.sqrt(n) * abs(W)
    assert np.abs(e[3:6]).max() < 1e-14


def test_two_plummer_layout():
    b = inputs.two_plummer(n_per=2048, seed=2)
    assert b.n == 4096
    np.testing.assert_allclose(b.mass.sum(), 1.0, rtol=1e-14)
    MA, MB = b.mass[:2048].sum(), b.mass[2048:].sum()
    ca = (b.mass[:2048, None] * b.pos[:2048]).sum(0) / MA
    cb = (b.mass[2048:, None] * b.pos[2048:]).sum(0) / MB
    np.testing.assert_allclose(ca, [-5, 0, 0], atol=1e-12)
    np.testing.assert_allclose(cb, [5, 0, 0], atol=1e-12)
    va = (b.mass[:2048, None] * b.vel[:2048]).sum(0) / MA
    vb = (b.mass[2048:, None] * b.vel[2048:]).sum(0) / MB
    np.testing.assert_allclose(va - vb, [0.5, 0, 0], atol=1e-12)
    np.testing.assert_allclose((b.mass[:, None] * b.vel).sum(0), 0, atol=1e-14)


def test_batch_sizes_log_uniform():
    s = inputs.batch_sizes(512, seed=3)
    assert s.min() >= 64 and s.max() <= 8192 and s.size == 512
    lg = np.log(s)
    assert abs(lg.mean() - 0.5 * (math.log(64) + math.log(8192))) < 0.2
    bodies, off = inputs.plummer_batch(sizes=[64, 100, 7])
    assert list(off) == [0, 64, 164, 171]
    np.testing.assert_allclose(bodies.mass[64:164].sum(), 1.0, rtol=1e-14)
