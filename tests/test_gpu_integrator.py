"""Leapfrog (KDK) and diagnostics on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_2292_gb300 import inputs, nbody
from helpers import host, relerr_per_body, to_dev

pytestmark = pytest.mark.gpu


def _run(cuda, prec, b, G, eps, dt, nsteps, graph=False, nb=None):
    own = nb is None
    nb = nb or nbody.NBody(b.n, prec)
    x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
    a = torch.empty_like(x)
    nb.step(x, v, m, G, eps, dt, nsteps, a, graph=graph)
    nb.sync()
    out = host(x), host(v), host(a)
    if own:
        nb.close()
    return out


def test_plain_fp64_config_n1024(cuda):
    # N = 1024 equal-mass Plummer sphere, seed 0, G = 1, eps = 0.01, 10 KDK
    # steps of dt = 1e-3: accelerations, positions and total energy.
    b = inputs.plummer(1024, seed=0)
    rx, rv, ra = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 10)
    x, v, a = _run(cuda, "fp64", b, 1.0, 0.01, 1e-3, 10)
    assert relerr_per_body(a, ra).max() <= 1e-12
    assert np.abs(x - rx).max() <= 1e-13
    assert np.abs(v - rv).max() <= 1e-12
    with nbody.NBody(1024, "fp64") as nb:
        e = nb.energy(to_dev(x, cuda), to_dev(v, cuda), to_dev(b.mass, cuda), 1.0, 0.01)
    re = oracle.energy(rx, rv, b.mass, 1.0, 0.01)
    assert abs(e[2] - re[2]) <= 1e-12 * abs(re[2])
    assert abs(e[0] - re[0]) <= 1e-13 * abs(re[0])
    assert abs(e[1] - re[1]) <= 1e-12 * abs(re[1])
    assert np.abs(np.array(e[3:6]) - re[3:6]).max() <= 1e-15
    assert np.abs(e[6:9]).max() <= 1e-13


def test_plain_config_in_double_float(cuda):
    # The same run through the double-float form: float64 accuracy (forces
    # <= 1e-12) from the float32 pipe, Morton-ordered, over 10 steps
    b = inputs.plummer(1024, seed=0)
    rx, rv, ra = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 10)
    x, v, a = _run(cuda, "df64", b, 1.0, 0.01, 1e-3, 10)
    assert relerr_per_body(a, ra).max() <= 1e-12
    assert np.abs(x - rx).max() <= 1e-13
    assert np.abs(v - rv).max() <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32_comp", "df64"])
@pytest.mark.parametrize("n", [1, 2, 33, 1000])
def test_energy_matches_oracle(cuda, prec, n):
    b = inputs.plummer(n, seed=30 + n)
    with nbody.NBody(n, prec) as nb:
        e = nb.energy(to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda), 1.0, 0.02)
    re = oracle.energy(b.pos, b.vel, b.mass, 1.0, 0.02)
    for q in (0, 1, 2):
        assert abs(e[q] - re[q]) <= 1e-12 * max(abs(re[q]), 1e-300)
    assert np.abs(np.array(e[3:]) - re[3:]).max() <= 1e-13


def test_energy_zero_softening(cuda):
    b = inputs.random_system(50, seed=4)
    with nbody.NBody(50, "fp64") as nb:
        e = nb.energy(to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda), 1.0, 0.0)
    re = oracle.energy(b.pos, b.vel, b.mass, 1.0, 0.0)
    assert abs(e[1] - re[1]) <= 1e-12 * abs(re[1])


def test_fp32_comp_steps_track_oracle(cuda):
    b = inputs.plummer(4096, seed=5)
    rx, rv, ra = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.005, 5e-4, 20)
    x, v, a = _run(cuda, "fp32_comp", b, 1.0, 0.005, 5e-4, 20)
    e = relerr_per_body(a, ra)
    assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4
    assert np.abs(x - rx).max() <= 1e-9
    assert np.abs(v - rv).max() <= 1e-6


def test_zero_steps_is_force_only(cuda):
    b = inputs.plummer(300, seed=6)
    x, v, a = _run(cuda, "fp64", b, 1.0, 0.01, 1e-3, 0)
    assert np.array_equal(x, b.pos) and np.array_equal(v, b.vel)
    assert relerr_per_body(a, oracle.accel(b.pos, b.mass, 1.0, 0.01)).max() <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32_comp", "df64"])
def test_graph_matches_eager_and_acc_valid(cuda, prec):
    b = inputs.plummer(777, seed=7)
    x1, v1, a1 = _run(cuda, prec, b, 1.0, 0.01, 1e-3, 6)
    x2, v2, a2 = _run(cuda, prec, b, 1.0, 0.01, 1e-3, 6, graph=True)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(a1, a2)
    # 3 steps, then 3 more with the cached force: same as 6 in one call
    with nbody.NBody(b.n, prec) as nb:
        x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
        a = torch.empty_like(x)
        nb.step(x, v, m, 1.0, 0.01, 1e-3, 3, a)
        nb.step(x, v, m, 1.0, 0.01, 1e-3, 3, a, acc_valid=True, graph=True)
        nb.step(x, v, m, 1.0, 0.01, 1e-3, 0, a, acc_valid=True)
        assert np.array_equal(host(x), x1) and np.array_equal(host(v), v1)


def test_rollout_records(cuda):
    b = inputs.plummer(200, seed=8)
    with nbody.NBody(b.n, "fp64") as nb:
        x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
        a = torch.empty_like(x)
        rp = torch.full((4, b.n, 3), np.nan, dtype=torch.float64, device=cuda)
        rv = torch.full_like(rp, np.nan)
        nb.rollout(x, v, m, 1.0, 0.01, 1e-3, 10, a, 3, rp, rv)
        rp, rv = host(rp), host(rv)
    for r, k in enumerate((0, 3, 6, 9)):
        ox, ov, _ = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, k)
        assert np.abs(rp[r] - ox).max() <= 1e-13
        assert np.abs(rv[r] - ov).max() <= 1e-12


def test_momentum_conserved_fp64(cuda):
    b = inputs.plummer(2000, seed=9)
    x, v, _ = _run(cuda, "fp64", b, 1.0, 0.01, 1e-3, 20)
    p0 = (b.mass[:, None] * b.vel).sum(0)
    p1 = (b.mass[:, None] * v).sum(0)
    assert np.abs(p1 - p0).max() <= 1e-14
