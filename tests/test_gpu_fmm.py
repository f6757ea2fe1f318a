"""GPU fast multipole method against the oracle's (paper Sec. VI names the FMM
as its tree code's O(N) successor).

Both sides build the same tree and decide well-separatedness exactly (integer
centres), so the source cells and direct partners of every body agree
exactly; the GPU translates float32 expansions that the oracle evaluates by
their float64 definitions, so the accelerations agree to float32 rounding.
With theta = 0 the FMM is the direct sum.
"""
import numpy as np
import pytest

import oracle
from helpers import host, relerr_per_body, to_dev
from paper_1211_2292_gb300 import inputs, nbody

pytestmark = pytest.mark.gpu

RMS_TOL, MAX_TOL = 1e-5, 1e-4  # float32 expansions and pair terms


def _gpu_fmm(cuda, pos, mass, G, eps, theta, order, leaf_cap, prec="fp32_comp"):
    x, m = to_dev(pos, cuda), to_dev(mass, cuda)
    with nbody.NBody(len(mass), prec) as nb:
        a, cnt = nb.fmm_forces(x, m, G, eps, theta, order, leaf_cap, counts=True)
        nb.sync()
        st = nb.fmm_stats()
    return host(a), host(cnt).astype(np.int64), st


def _check(a, cnt, st, ref, rcnt, rst, rms_tol=RMS_TOL, max_tol=MAX_TOL):
    assert np.array_equal(cnt, rcnt)
    assert st == rst
    # error against the rms acceleration (per-body ratios are ill-conditioned
    # where |a| nearly vanishes)
    rms = np.sqrt((np.linalg.norm(ref, axis=1) ** 2).mean())
    e = np.linalg.norm(a - ref, axis=1) / rms
    assert np.sqrt((e ** 2).mean()) <= rms_tol and e.max() <= max_tol, (e.max(),
                                                                         np.sqrt((e ** 2).mean()))


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("n,theta,leaf_cap,eps", [(3001, 0.5, 16, 0.01), (20000, 0.6, 32, 0.005),
                                                  (777, 0.9, 1, 0.02), (12000, 0.35, 64, 0.0)])
def test_matches_oracle_fmm(cuda, n, theta, leaf_cap, eps, order):
    b = inputs.plummer(n, seed=81)
    a, cnt, st = _gpu_fmm(cuda, b.pos, b.mass, 1.0, eps, theta, order, leaf_cap)
    ref, rst, rcnt = oracle.fmm_forces(b.pos, b.mass, 1.0, eps, theta, order, leaf_cap,
                                       counts=True)
    _check(a, cnt, st, ref, rcnt, rst)
    assert np.all(cnt[:, 1] + cnt[:, 2] == n)


def test_theta_zero_is_the_direct_sum(cuda):
    b = inputs.plummer(3000, seed=82)
    a, cnt, st = _gpu_fmm(cuda, b.pos, b.mass, 1.0, 0.01, 0.0, 4, 16)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    assert np.all(cnt[:, 0] == 0) and np.all(cnt[:, 2] == b.n)
    assert st["expansions"] == 0 and st["direct_pairs"] == b.n * b.n
    e = relerr_per_body(a, ref)
    assert np.sqrt((e ** 2).mean()) <= RMS_TOL and e.max() <= MAX_TOL


def test_two_clusters_and_every_precision_mode(cuda):
    b = inputs.two_plummer(4000, seed=83)
    ref, rst, rcnt = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.005, 0.5, 5, 32, counts=True)
    for prec in ("fp64", "fp32", "fp32_comp", "df64"):
        a, cnt, st = _gpu_fmm(cuda, b.pos, b.mass, 1.0, 0.005, 0.5, 5, 32, prec)
        _check(a, cnt, st, ref, rcnt, rst)


def test_error_against_direct_sum_falls_with_order(cuda):
    b = inputs.plummer(30000, seed=84)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    rms = []
    for order in (2, 4, 6):
        a, _, _ = _gpu_fmm(cuda, b.pos, b.mass, 1.0, 0.01, 0.5, order, 32)
        e = relerr_per_body(a, ref)
        rms.append(np.sqrt((e ** 2).mean()))
    assert rms[0] > rms[1] > rms[2] and rms[2] < 3e-4


def test_degenerate_inputs(cuda):
    # all bodies at one point: one chain of single-child cells down to a
    # level-10 leaf holding all 100 bodies (more than the 64 a pass takes)
    pos = np.zeros((100, 3)) + 0.25
    m = np.full(100, 0.01)
    a, cnt, st = _gpu_fmm(cuda, pos, m, 1.0, 0.1, 0.5, 4, 4)
    _, rst, rcnt = oracle.fmm_forces(pos, m, 1.0, 0.1, 0.5, 4, 4, counts=True)
    assert np.all(a == 0) and np.array_equal(cnt, rcnt) and st == rst and st["nodes"] == 11
    for n, eps, lc in ((1, 0.1, 8), (2, 0.0, 1), (33, 0.0, 1), (65, 0.0, 64), (100, 0.01, 2)):
        bb = inputs.random_system(n, seed=85 + n)
        a, cnt, st = _gpu_fmm(cuda, bb.pos, bb.mass, 1.3, eps, 0.5, 3, lc)
        ref, rst, rcnt = oracle.fmm_forces(bb.pos, bb.mass, 1.3, eps, 0.5, 3, lc, counts=True)
        assert np.array_equal(cnt, rcnt) and st == rst and np.isfinite(a).all()
        if n == 1:
            assert np.all(a == 0)
        else:
            assert relerr_per_body(a, ref).max() <= MAX_TOL


def test_shapes_the_tree_can_take(cuda):
    rng = np.random.default_rng(86)
    disc = np.column_stack([rng.normal(size=(3000, 2)), np.zeros(3000)])
    clump = np.vstack([rng.normal(size=(2000, 3)), 1e-9 * rng.normal(size=(300, 3)) + 0.3])
    cases = [
        (disc, rng.uniform(0.5, 1.5, 3000) / 3000, 0.5, 16, 0.01),
        (rng.normal(size=(60, 3)), rng.uniform(0.5, 1.5, 60) / 60, 0.5, 64, 0.01),
        (clump, rng.uniform(0.5, 1.5, 2300) / 2300, 0.5, 8, 0.1),
        (rng.normal(size=(2000, 3)), np.where(rng.random(2000) < 0.3, 0.0, 1.0 / 2000), 0.6, 4,
         0.01),
    ]
    for pos, mass, theta, lc, eps in cases:
        a, cnt, st = _gpu_fmm(cuda, pos, mass, 1.0, eps, theta, 5, lc)
        ref, rst, rcnt = oracle.fmm_forces(pos, mass, 1.0, eps, theta, 5, lc, counts=True)
        _check(a, cnt, st, ref, rcnt, rst)


def test_deterministic_and_empty(cuda):
    b = inputs.plummer(20000, seed=87)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a1 = host(nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 5, 32))
        a2 = host(nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 5, 32))
        a3 = host(nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 4, 32))  # smaller order, same scratch
        e = nb.fmm_forces(x[:0], m[:0], 1.0, 0.01, 0.5, 5, 32)
        nb.sync()
    assert np.array_equal(a1, a2) and e.shape == (0, 3)
    ref, _ = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.01, 0.5, 4, 32)
    assert relerr_per_body(a3, ref).max() <= MAX_TOL


def test_argument_checks(cuda):
    import torch
    b = inputs.plummer(64, seed=88)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    a = torch.empty((64, 3), dtype=torch.float64, device=cuda)
    with nbody.NBody(64, "fp32_comp") as nb:
        lib, before = nb.lib, nb.launches
        args = (nb.h, 64, x.data_ptr(), m.data_ptr(), 1.0, 0.01)
        assert lib.nb_fmm_forces(*args, -0.1, 4, 16, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(*args, float("nan"), 4, 16, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(*args, 0.5, 1, 16, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(*args, 0.5, 7, 16, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(*args, 0.5, 4, 0, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(*args, 0.5, 4, 65, a.data_ptr(), None) == 1
        assert lib.nb_fmm_forces(nb.h, 65, x.data_ptr(), m.data_ptr(), 1.0, 0.01, 0.5, 4, 16,
                                 a.data_ptr(), None) == 1
        assert nb.launches == before


def test_pool_overflow_reruns_with_a_larger_pool(cuda):
    # A pool of 16 candidate ids overflows at the first non-leaf cells; the
    # host doubles it and reruns the passes until it suffices, and the result
    # is bit-identical to the run with the default pool.
    b = inputs.plummer(20000, seed=89)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a1, c1 = nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 4, 16, counts=True)
        nb.sync()
        st1 = nb.fmm_stats()
        nb.fmm_reserve(16)
        a2, c2 = nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 4, 16, counts=True)
        nb.sync()
        st2 = nb.fmm_stats()
        with pytest.raises(nbody.NBodyError):
            nb.fmm_reserve(0)
    assert np.array_equal(host(a1), host(a2)) and np.array_equal(host(c1), host(c2))
    assert st1 == st2


def test_fmm_step_matches_oracle_kdk_at_theta_zero(cuda):
    # theta = 0: every evaluation is the direct sum, so ten FMM steps follow
    # the oracle's leapfrog.
    b = inputs.plummer(2000, seed=90)
    xr, vr, _ = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 10)
    x, v, m = (to_dev(t, cuda) for t in (b.pos, b.vel, b.mass))
    acc = to_dev(np.zeros((b.n, 3)), cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        nb.fmm_step(x, v, m, 1.0, 0.01, 0.0, 4, 16, 1e-3, 10, acc)
        nb.sync()
    assert np.abs(host(x) - xr).max() <= 1e-9
    assert np.abs(host(v) - vr).max() <= 1e-6


def test_fmm_step_is_the_kick_drift_kick_of_fmm_forces(cuda):
    # One step at theta 0.5 checked against fmm_forces: x' = x + dt (v + dt/2
    # a(x)), acc = a(x') exactly, v' = v + dt/2 (a(x) + a(x')); a second step
    # with acc_valid starts from that cached acc; graphs are refused.
    import torch
    b = inputs.plummer(5000, seed=91)
    dt = 2e-3
    x, v, m = (to_dev(t, cuda) for t in (b.pos, b.vel, b.mass))
    acc = to_dev(np.zeros((b.n, 3)), cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a0 = nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 5, 32)
        x0, v0 = x.clone(), v.clone()
        nb.fmm_step(x, v, m, 1.0, 0.01, 0.5, 5, 32, dt, 1, acc)
        a1 = nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 5, 32)
        nb.sync()
        assert torch.equal(acc, a1)
        assert torch.allclose(x, x0 + dt * (v0 + 0.5 * dt * a0), rtol=0, atol=1e-13)
        assert torch.allclose(v, v0 + 0.5 * dt * (a0 + a1), rtol=0, atol=1e-13)
        x1, v1 = x.clone(), v.clone()
        nb.fmm_step(x, v, m, 1.0, 0.01, 0.5, 5, 32, dt, 1, acc, acc_valid=True)
        a2 = nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 5, 32)
        nb.sync()
        assert torch.equal(acc, a2)
        assert torch.allclose(v, v1 + 0.5 * dt * (a1 + a2), rtol=0, atol=1e-13)
        assert nb.lib.nb_fmm_step(nb.h, b.n, x.data_ptr(), v.data_ptr(), m.data_ptr(), 1.0, 0.01,
                                  0.5, 5, 32, dt, 1, acc.data_ptr(), 2) == 1  # graph refused


@pytest.mark.parametrize("method", ["tree", "fmm"])
def test_nonfinite_input_is_reported(cuda, method):
    # An infinite coordinate makes the box infinite: every key quantises to a
    # valid cell (the structure stays consistent), the sums turn non-finite
    # and nb_sync reports NB_ENONFINITE once.
    b = inputs.plummer(300, seed=92)
    pos = b.pos.copy()
    pos[7, 1] = np.inf
    with nbody.NBody(b.n, "fp32_comp") as nb:
        x, m = to_dev(pos, cuda), to_dev(b.mass, cuda)
        if method == "tree":
            nb.tree_forces(x, m, 1.0, 0.01, 0.5, 16)
        else:
            nb.fmm_forces(x, m, 1.0, 0.01, 0.5, 4, 16)
        with pytest.raises(nbody.NBodyError) as ei:
            nb.sync()
        assert ei.value.status == 4
        nb.sync()  # flag cleared
