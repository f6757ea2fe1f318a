"""GPU force kernels against the FP64 oracle, through the C ABI.

Tolerances (per-body relative error e_i = |a_i - a_i^ref| / |a_i^ref|):
  FP64 form:        max e_i <= 1e-12
  double-float:     max e_i <= 1e-12, RMS e_i <= 1e-13 (48-bit pair arithmetic)
  FP32 compensated: RMS e_i <= 1e-5, max e_i <= 1e-4
  FP32 plain:       RMS e_i <= 1e-4 at N <= 4097 (one float32 running sum)
Sizes span one and several tiles with ragged tails; every compiled variant
and forced j-splits are exercised.
"""
import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs, nbody
from helpers import host, relerr_per_body, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 31, 32, 33, 127, 1000, 1024, 4097]


def _forces(cuda, prec, b, G, eps, variant=None, split=0):
    with nbody.NBody(max(b.n, 1), prec) as nb:
        if variant is not None:
            nb.tune_set(nbody.KIND_FORCE, 0, 1 << 40, variant, split)
        a = nb.forces(to_dev(b.pos, cuda), to_dev(b.mass, cuda), G, eps)
        nb.sync()
        return host(a)


@pytest.mark.parametrize("n", SIZES)
def test_fp64_matches_oracle(cuda, n):
    b = inputs.plummer(n, seed=n)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    a = _forces(cuda, "fp64", b, 1.0, 0.01)
    if n == 1:
        assert np.all(a == 0)
        return
    assert relerr_per_body(a, ref).max() <= 1e-12


@pytest.mark.parametrize("sep", [1e-20, 1e-45, 1e-60, 1e20, 1e45, 1e60])
def test_fp64_separations_outside_the_float32_range(cuda, sep):
    # eps = 0: r^2 = sep^2 lies outside float32's normal range, where a
    # float32 seed of the float64 rsqrt would flush to zero or overflow.
    # Two bodies: a closed form, a_0 = G m_1 d / r^3 (and the oracle agrees).
    pos = np.array([[0.0, 0.0, 0.0], [sep * 0.6, -sep * 0.8, 0.0]])
    mass = np.array([0.75, 0.25])
    b = inputs.Bodies(pos, np.zeros_like(pos), mass)
    a = _forces(cuda, "fp64", b, 1.0, 0.0)
    d = pos[1] - pos[0]
    r = np.linalg.norm(d)
    exact = np.array([mass[1] * d / r ** 3, -mass[0] * d / r ** 3])
    assert np.all(np.isfinite(a))
    assert relerr_per_body(a, exact).max() <= 1e-12
    assert relerr_per_body(oracle.accel(pos, mass, 1.0, 0.0), exact).max() <= 1e-14
    with nbody.NBody(2, "fp64") as nb:
        e = nb.energy(to_dev(pos, cuda), to_dev(np.zeros_like(pos), cuda), to_dev(mass, cuda),
                      1.0, 0.0)
    assert abs(e[1] - (-mass[0] * mass[1] / r)) <= 1e-12 * abs(mass[0] * mass[1] / r)


@pytest.mark.parametrize("n", SIZES)
def test_df64_matches_oracle(cuda, n):
    b = inputs.plummer(n, seed=300 + n)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    a = _forces(cuda, "df64", b, 1.0, 0.01)
    if n == 1:
        assert np.all(a == 0)
        return
    e = relerr_per_body(a, ref)
    assert e.max() <= 1e-12 and np.sqrt((e ** 2).mean()) <= 1e-13


def test_df64_at_the_precision_and_throughput_workloads(cuda):
    # N = 65,536 Plummer (eps 0.005) and the first 262,144 bodies of the
    # two-sphere workload (eps 0.002): 2048 sampled bodies each
    for b, eps in ((inputs.plummer(65536, seed=1), 0.005),
                   (inputs.two_plummer(131072, seed=2), 0.002)):
        rows = inputs.sample_rows(b.n, 2048, seed=1)
        ref = oracle.accel_rows(b.pos, b.mass, rows, 1.0, eps)
        e = relerr_per_body(_forces(cuda, "df64", b, 1.0, eps)[rows], ref)
        assert e.max() <= 1e-12 and np.sqrt((e ** 2).mean()) <= 1e-13


@pytest.mark.parametrize("n", SIZES)
def test_fp32_comp_matches_oracle(cuda, n):
    b = inputs.plummer(n, seed=100 + n)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.005)
    a = _forces(cuda, "fp32_comp", b, 1.0, 0.005)
    if n == 1:
        assert np.all(a == 0)
        return
    e = relerr_per_body(a, ref)
    assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4


@pytest.mark.parametrize("n", [33, 1000, 4097])
def test_fp32_plain_matches_oracle(cuda, n):
    b = inputs.plummer(n, seed=200 + n)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    e = relerr_per_body(_forces(cuda, "fp32", b, 1.0, 0.01), ref)
    assert np.sqrt((e ** 2).mean()) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_comp", "df64"])
def test_every_variant_and_forced_splits(cuda, prec):
    b = inputs.plummer(3001, seed=7)
    ref = oracle.accel(b.pos, b.mass, 1.3, 0.02)
    tol = 1e-12 if prec in ("fp64", "df64") else 1e-4
    nvar = len(nbody.variants(nbody.KIND_FORCE, prec))
    for v in range(nvar):
        for split in (1, 3, 7):
            a = _forces(cuda, prec, b, 1.3, 0.02, variant=v, split=split)
            e = relerr_per_body(a, ref)
            assert e.max() <= tol, (v, split, e.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_comp", "df64"])
def test_zero_softening_skips_self_pair(cuda, prec):
    x = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    m = np.array([1.0, 3.0])
    b = inputs.Bodies(x, np.zeros_like(x), m)
    a = _forces(cuda, prec, b, 1.0, 0.0)
    rtol = {"fp64": 1e-15, "df64": 1e-13}.get(prec, 1e-6)
    np.testing.assert_allclose(a, [[0, 0.75, 0], [0, -0.25, 0]], rtol=rtol)
    b = inputs.random_system(33, seed=3)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.0)
    e = relerr_per_body(_forces(cuda, prec, b, 1.0, 0.0), ref)
    assert np.isfinite(e).all() and e.max() <= (1e-12 if prec in ("fp64", "df64") else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32_comp", "df64"])
def test_deterministic_across_calls(cuda, prec):
    b = inputs.plummer(5000, seed=9)
    with nbody.NBody(b.n, prec) as nb:
        nb.tune_set(nbody.KIND_FORCE, 0, 1 << 40, 0, 5)
        x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
        a1 = host(nb.forces(x, m, 1.0, 0.01))
        a2 = host(nb.forces(x, m, 1.0, 0.01))
    assert np.array_equal(a1, a2)


def test_scaling_laws_fp64(cuda):
    # Power-of-two scalings: G and mass linear, lengths (x and eps) as
    # length^-2.  A wrong power of s or a dropped factor breaks these.
    b = inputs.plummer(700, seed=10)
    a = _forces(cuda, "fp64", b, 1.0, 0.05)
    a2 = _forces(cuda, "fp64", inputs.Bodies(2 * b.pos, b.vel, b.mass), 1.0, 0.1)
    np.testing.assert_allclose(a2, a / 4, rtol=1e-14, atol=0)
    a3 = _forces(cuda, "fp64", b, 2.0, 0.05)
    np.testing.assert_array_equal(a3, 2 * a)


def test_empty_and_n_max(cuda):
    import torch
    with nbody.NBody(16, "fp32_comp") as nb:
        z = torch.zeros((0, 3), dtype=torch.float64, device=cuda)
        nb.forces(z, torch.zeros(0, dtype=torch.float64, device=cuda), 1.0, 0.1, out=z)
        b = inputs.plummer(16, seed=1)
        a = host(nb.forces(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.1))
        ref = oracle.accel(b.pos, b.mass, 1.0, 0.1)
        assert relerr_per_body(a, ref).max() < 1e-4
        b17 = inputs.plummer(17, seed=1)
        with pytest.raises(nbody.NBodyError) as ei:
            nb.forces(to_dev(b17.pos, cuda), to_dev(b17.mass, cuda), 1.0, 0.1)
        assert ei.value.status == 1


def test_argument_checks_reject_before_launch(cuda):
    import ctypes
    import torch
    lib = nbody.load()
    with nbody.NBody(64, "fp32_comp") as nb:
        x = torch.zeros((64, 3), dtype=torch.float64, device=cuda)
        m = torch.ones(64, dtype=torch.float64, device=cuda)
        a = torch.zeros((64, 3), dtype=torch.float64, device=cuda)
        before = nb.launches
        # host memory instead of device memory
        hx = np.zeros((64, 3))
        st = lib.nb_forces(nb.h, 64, hx.ctypes.data, m.data_ptr(), 1.0, 0.1, a.data_ptr())
        assert st == 1
        # misaligned pointer
        st = lib.nb_forces(nb.h, 63, x.data_ptr() + 4, m.data_ptr(), 1.0, 0.1, a.data_ptr())
        assert st == 1
        # NULL, NaN G, negative eps, n out of range
        assert lib.nb_forces(nb.h, 64, None, m.data_ptr(), 1.0, 0.1, a.data_ptr()) == 1
        assert lib.nb_forces(nb.h, 64, x.data_ptr(), m.data_ptr(), float("nan"), 0.1, a.data_ptr()) == 1
        assert lib.nb_forces(nb.h, 64, x.data_ptr(), m.data_ptr(), 1.0, -0.1, a.data_ptr()) == 1
        assert lib.nb_forces(nb.h, 65, x.data_ptr(), m.data_ptr(), 1.0, 0.1, a.data_ptr()) == 1
        assert lib.nb_forces(nb.h, -1, x.data_ptr(), m.data_ptr(), 1.0, 0.1, a.data_ptr()) == 1
        torch.cuda.synchronize()
        assert nb.launches == before
        nb.sync()


def test_nonfinite_flag_reported(cuda):
    b = inputs.plummer(100, seed=2)
    pos = b.pos.copy()
    pos[5, 0] = np.inf
    with nbody.NBody(100, "fp64") as nb:
        nb.forces(to_dev(pos, cuda), to_dev(b.mass, cuda), 1.0, 0.01)
        with pytest.raises(nbody.NBodyError) as ei:
            nb.sync()
        assert ei.value.status == 4
        nb.sync()  # flag cleared


@pytest.mark.parametrize("prec", ["fp32", "fp32_comp"])
@pytest.mark.parametrize("n", [1, 2, 33, 1000, 4097])
def test_morton_order_matches_oracle_and_is_deterministic(cuda, prec, n):
    b = inputs.plummer(n, seed=300 + n)
    ref = oracle.accel(b.pos, b.mass, 1.0, 0.01)
    with nbody.NBody(n, prec) as nb:
        nb.set_order(1)
        x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
        a1 = host(nb.forces(x, m, 1.0, 0.01))
        a2 = host(nb.forces(x, m, 1.0, 0.01))
    assert np.array_equal(a1, a2)
    if n > 1:
        assert relerr_per_body(a1, ref).max() <= 1e-4


def test_morton_order_fixes_offset_close_pairs(cuda):
    # Two spheres at (+-5, 0, 0), eps = 0.002: with bodies in input order the
    # float32 rounding of |x| ~ 5 dominates close pairs; spatially ordered
    # i-tiles with tile-local origins remove it.
    b = inputs.two_plummer(n_per=16384, seed=2)
    rows = inputs.sample_rows(b.n, 2048, seed=1)
    ref = oracle.accel_rows(b.pos, b.mass, rows, 1.0, 0.002)
    errs = {}
    for mode in (0, 1):
        with nbody.NBody(b.n, "fp32_comp") as nb:
            nb.set_order(mode)
            a = host(nb.forces(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.002))[rows]
        errs[mode] = relerr_per_body(a, ref)
    assert errs[1].max() <= 1e-4 and np.sqrt((errs[1] ** 2).mean()) <= 1e-5
    assert errs[1].max() < 0.5 * errs[0].max()


def test_morton_order_in_step_loop(cuda):
    b = inputs.plummer(3000, seed=301)
    rx, rv, ra = oracle.kdk(b.pos, b.vel, b.mass, 1.0, 0.01, 1e-3, 5)
    for graph in (False, True):
        with nbody.NBody(b.n, "fp32_comp") as nb:
            nb.set_order(1)
            x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
            a = torch_empty_like(x)
            nb.step(x, v, m, 1.0, 0.01, 1e-3, 5, a, graph=graph)
            e = relerr_per_body(host(a), ra)
            assert e.max() <= 1e-4
            assert np.abs(host(x) - rx).max() <= 1e-9


def torch_empty_like(x):
    import torch
    return torch.empty_like(x)
