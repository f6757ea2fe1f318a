"""Batched persistent force kernel and graph-captured stepping."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_2292_gb300 import inputs, nbody
from helpers import host, relerr_per_body, to_dev

pytestmark = pytest.mark.gpu

SIZES = [64, 0, 1, 2, 100, 1000, 8192, 37, 513]


def _check_systems(a, bodies, off, eps, idx=None):
    for k in (range(len(off) - 1) if idx is None else idx):
        s, e = off[k], off[k + 1]
        if e - s < 2:
            assert np.all(a[s:e] == 0)
            continue
        ref = oracle.accel(bodies.pos[s:e], bodies.mass[s:e], 1.0, eps)
        err = relerr_per_body(a[s:e], ref)
        assert np.sqrt((err ** 2).mean()) <= 1e-5 and err.max() <= 1e-4, (k, err.max())


@pytest.mark.parametrize("variant", list(range(11)))
def test_batched_forces_match_oracle(cuda, variant):
    bodies, off = inputs.plummer_batch(sizes=SIZES, seed=3)
    with nbody.NBody(bodies.n, "fp32_comp") as nb:
        nb.tune_set(nbody.KIND_BATCHED, 0, 1 << 40, variant)
        nb.batch_plan(off)
        a = host(nb.forces_batched(to_dev(bodies.pos, cuda), to_dev(bodies.mass, cuda), 1.0, 0.01))
        nb.sync()
    _check_systems(a, bodies, off, 0.01)


def test_batched_zero_softening(cuda):
    bodies, off = inputs.plummer_batch(sizes=[5, 70, 300], seed=2)
    with nbody.NBody(bodies.n, "fp32") as nb:
        nb.batch_plan(off)
        a = host(nb.forces_batched(to_dev(bodies.pos, cuda), to_dev(bodies.mass, cuda), 1.0, 0.0))
    for k in range(3):
        s, e = off[k], off[k + 1]
        ref = oracle.accel(bodies.pos[s:e], bodies.mass[s:e], 1.0, 0.0)
        assert relerr_per_body(a[s:e], ref).max() <= 1e-3


def test_batched_bitwise_equals_solo_when_tiles_match(cuda):
    # Batched variant 1 and solo variant 0 share (T, I, J) = (128, 4, 128);
    # a system of whole tiles runs with one lane per body and (with few
    # items) unsplit j ranges, so both perform the same operations in the
    # same order.
    assert nbody.variants(nbody.KIND_BATCHED, "fp32_comp")[1] == nbody.variants(
        nbody.KIND_FORCE, "fp32_comp")[0]
    b = inputs.plummer(3072, seed=11)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        nb.tune_set(nbody.KIND_FORCE, 0, 1 << 40, 0, 1)
        solo = host(nb.forces(x, m, 1.0, 0.01))
        nb.tune_set(nbody.KIND_BATCHED, 0, 1 << 40, 1)
        nb.batch_plan([0, b.n])
        bat = host(nb.forces_batched(x, m, 1.0, 0.01))
    assert np.array_equal(solo, bat)


def test_chunked_pieces_equal_the_solo_j_split(cuda):
    # 400 systems of 2048 bodies: more pieces than resident CTAs, so each
    # piece's j range is split into chunks (2 to 4 here, by the item cap)
    # whose partial sums the last chunk adds in order -- the solo kernel's
    # j-split with the same count, bit for bit.
    bodies, off = inputs.plummer_batch(sizes=[2048] * 400, seed=14)
    x, m = to_dev(bodies.pos, cuda), to_dev(bodies.mass, cuda)
    with nbody.NBody(bodies.n, "fp32_comp") as nb:
        nb.tune_set(nbody.KIND_BATCHED, 0, 1 << 40, 1, 4)
        nb.batch_plan(off)
        a = host(nb.forces_batched(x, m, 1.0, 0.01))
        nb.sync()
    with nbody.NBody(2048, "fp32_comp") as nb:
        for k in (0, 177, 399):
            s_, e_ = off[k], off[k + 1]
            match = []
            for S in (1, 2, 3, 4):
                nb.tune_set(nbody.KIND_FORCE, 0, 1 << 40, 0, S)
                if np.array_equal(host(nb.forces(x[s_:e_], m[s_:e_], 1.0, 0.01)), a[s_:e_]):
                    match.append(S)
            assert match and match[0] > 1, (k, match)
    _check_systems(a, bodies, off, 0.01, idx=[0, 5, 177, 250, 399])


def test_batched_steps_match_oracle_and_graph(cuda):
    bodies, off = inputs.plummer_batch(sizes=[300, 64, 1500, 0, 700], seed=12)
    res = []
    for graph in (False, True):
        with nbody.NBody(bodies.n, "fp32_comp") as nb:
            nb.batch_plan(off)
            x, v, m = (to_dev(bodies.pos, cuda), to_dev(bodies.vel, cuda),
                       to_dev(bodies.mass, cuda))
            a = torch.empty_like(x)
            nb.step_batched(x, v, m, 1.0, 0.01, 1e-3, 8, a, graph=graph)
            if graph:  # a second launch of the cached graph continues the run
                nb.step_batched(x, v, m, 1.0, 0.01, 1e-3, 8, a, acc_valid=True, graph=True)
            else:
                nb.step_batched(x, v, m, 1.0, 0.01, 1e-3, 8, a, acc_valid=True)
            nb.sync()
            res.append((host(x), host(v), host(a)))
    for p, q in zip(*res):
        assert np.array_equal(p, q)
    x, v, a = res[0]
    for k in range(len(off) - 1):
        s, e = off[k], off[k + 1]
        if e == s:
            continue
        ox, ov, oa = oracle.kdk(bodies.pos[s:e], bodies.vel[s:e], bodies.mass[s:e], 1.0, 0.01,
                                1e-3, 16)
        assert np.abs(x[s:e] - ox).max() <= 1e-9
        err = relerr_per_body(a[s:e], oa)
        assert err.max() <= 1e-4


def test_plan_rejects_bad_offsets(cuda):
    with nbody.NBody(100, "fp32_comp") as nb:
        for bad in ([1, 10], [0, 10, 5], [0, 101]):
            with pytest.raises(nbody.NBodyError):
                nb.batch_plan(bad)
    with nbody.NBody(100, "fp64") as nb:
        with pytest.raises(nbody.NBodyError):
            nb.batch_plan([0, 10])


def test_queue_resets_between_launches(cuda):
    # Many launches in a row: each must see a fresh queue (self-reset).
    bodies, off = inputs.plummer_batch(sizes=[200] * 40, seed=13)
    with nbody.NBody(bodies.n, "fp32_comp") as nb:
        nb.batch_plan(off)
        x, m = to_dev(bodies.pos, cuda), to_dev(bodies.mass, cuda)
        first = host(nb.forces_batched(x, m, 1.0, 0.01))
        for _ in range(20):
            again = host(nb.forces_batched(x, m, 1.0, 0.01))
            assert np.array_equal(first, again)
