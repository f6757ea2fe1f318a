"""Force VJP and leapfrog adjoint on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_2292_gb300 import inputs, nbody
from paper_1211_2292_gb300.autograd import rollout
from helpers import host, to_dev

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_comp", 5e-5), ("fp32", 5e-5),
                                      ("df64", 1e-12)])
@pytest.mark.parametrize("n", [2, 33, 1000, 2049])
def test_force_vjp_matches_oracle(cuda, prec, tol, n):
    # FP32 tolerance: the float32 rounding of the positions perturbs each
    # close-pair term by about ulp(|x - c|)/|d| relative (c the tile origin),
    # and the VJP sums cancel (random-sign cotangents), so 5e-5 relative in
    # norm; the direct float32 arithmetic itself contributes ~1e-6.
    b = inputs.plummer(n, seed=40 + n)
    lam = np.random.default_rng(n).normal(size=(n, 3))
    rgx, rgm = oracle.force_vjp(b.pos, b.mass, lam, 1.2, 0.01)
    with nbody.NBody(n, prec) as nb:
        gx, gm = nb.forces_backward(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.2, 0.01,
                                    to_dev(lam, cuda))
        nb.sync()
    assert _rel(host(gx), rgx) <= tol
    assert _rel(host(gm), rgm) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32_comp"])
def test_vjp_variants_and_splits(cuda, prec):
    b = inputs.plummer(1500, seed=41)
    lam = np.random.default_rng(1).normal(size=(1500, 3))
    rgx, rgm = oracle.force_vjp(b.pos, b.mass, lam, 1.0, 0.02)
    tol = 1e-12 if prec == "fp64" else 5e-5
    for v in range(len(nbody.variants(nbody.KIND_VJP, prec))):
        for split in (1, 4, 7):
            with nbody.NBody(1500, prec) as nb:
                nb.tune_set(nbody.KIND_VJP, 0, 1 << 40, v, split)
                gx, gm = nb.forces_backward(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.02,
                                            to_dev(lam, cuda))
                nb.sync()
            assert _rel(host(gx), rgx) <= tol and _rel(host(gm), rgm) <= tol, (v, split)


def test_vjp_smooth_cotangent_fp32(cuda):
    # A smooth cotangent field (as the adjoint's dt*lam_v is) makes
    # w = m_k mu_j - m_j mu_k small for close pairs: the direct w form keeps
    # the float32 VJP accurate there.
    b = inputs.plummer(3000, seed=48)
    lam = np.stack([np.sin(b.pos[:, 0]), np.cos(b.pos[:, 1]), b.pos[:, 2] * 0.5], axis=1) + 1.0
    rgx, rgm = oracle.force_vjp(b.pos, b.mass, lam, 1.0, 0.01)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        gx, gm = nb.forces_backward(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.01,
                                    to_dev(lam, cuda))
    assert _rel(host(gx), rgx) <= 5e-5 and _rel(host(gm), rgm) <= 5e-5


def _vjp32(cuda, pos, mass, lam, G, eps, variant=None):
    with nbody.NBody(len(mass), "fp32_comp") as nb:
        if variant is not None:
            nb.tune_set(nbody.KIND_VJP, 0, 1 << 40, variant, 0)
        gx, gm = nb.forces_backward(to_dev(pos, cuda), to_dev(mass, cuda), G, eps,
                                    to_dev(lam, cuda))
        nb.sync()
        return host(gx), host(gm)


@pytest.mark.parametrize("variant", [0, 5])
def test_vjp_massless_bodies_fp32(cuda, variant):
    # Bodies of zero mass: the float32 kernel cannot form mu_k/m_k, so every
    # CTA holding one takes the m_k mu_j - m_j mu_k form; the others keep the
    # mu_j - m_j mu_k/m_k form.  Both against the oracle.
    b = inputs.plummer(1500, seed=49)
    mass = b.mass.copy()
    mass[:300:7] = 0.0  # the first CTAs hold massless bodies, the later ones none
    lam = np.random.default_rng(49).normal(size=(b.n, 3))
    rgx, rgm = oracle.force_vjp(b.pos, mass, lam, 1.0, 0.01)
    gx, gm = _vjp32(cuda, b.pos, mass, lam, 1.0, 0.01, variant)
    assert _rel(gx, rgx) <= 5e-5 and _rel(gm, rgm) <= 5e-5


@pytest.mark.parametrize("variant", [0, 5])
def test_vjp_tiny_mass_large_cotangent_fp32(cuda, variant):
    # m_j mu_k/m_k beyond the float32 range for a light body k with a large
    # cotangent next to heavy bodies j (mu_k/m_k itself finite): the lanes
    # whose tile sums overflow evaluate that tile again in the
    # m_k mu_j - m_j mu_k form, which stays finite, as the oracle does.
    b = inputs.plummer(1000, seed=50)
    mass = b.mass.copy()
    mass[[10, 400]] = 10.0
    mass[600] = 1e-30
    lam = np.random.default_rng(50).normal(size=(b.n, 3))
    lam[600] = [1e8, -2e8, 5e7]
    assert np.isfinite(np.float32(lam[600, 1]) / np.float32(mass[600]))
    rgx, rgm = oracle.force_vjp(b.pos, mass, lam, 1.0, 0.01)
    gx, gm = _vjp32(cuda, b.pos, mass, lam, 1.0, 0.01, variant)
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gm))
    assert _rel(gx, rgx) <= 5e-5 and _rel(gm, rgm) <= 5e-5


def test_vjp_zero_softening(cuda):
    b = inputs.random_system(40, seed=3)
    lam = np.random.default_rng(3).normal(size=(40, 3))
    rgx, rgm = oracle.force_vjp(b.pos, b.mass, lam, 1.0, 0.0)
    with nbody.NBody(40, "fp64") as nb:
        gx, gm = nb.forces_backward(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.0,
                                    to_dev(lam, cuda))
    assert _rel(host(gx), rgx) <= 1e-12 and _rel(host(gm), rgm) <= 1e-12


def _grads(cuda, prec, b, G, eps, dt, K, every, tgt):
    with nbody.NBody(b.n, prec) as nb:
        x0 = to_dev(b.pos, cuda).requires_grad_()
        v0 = to_dev(b.vel, cuda).requires_grad_()
        m = to_dev(b.mass, cuda).requires_grad_()
        xT, vT = rollout(nb, x0, v0, m, G, eps, dt, K, every)
        loss = ((xT - to_dev(tgt, cuda)) ** 2).sum(-1).mean()
        loss.backward()
        return host(x0.grad), host(v0.grad), host(m.grad), float(loss.detach())


@pytest.mark.parametrize("K,every", [(30, 7), (30, 30), (1, 1)])
def test_rollout_grad_matches_oracle_fp64(cuda, K, every):
    b = inputs.plummer(64, seed=44)
    G, eps, dt = 1.0, 0.01, 1e-3
    tgt = b.pos + 0.01
    gx, gv, gm, _ = _grads(cuda, "fp64", b, G, eps, dt, K, every, tgt)
    xT, _, _ = oracle.kdk(b.pos, b.vel, b.mass, G, eps, dt, K)
    ox, ov, om = oracle.kdk_grad(b.pos, b.vel, b.mass, G, eps, dt, K,
                                 2.0 / b.n * (xT - tgt), np.zeros_like(xT))
    assert _rel(gx, ox) <= 1e-10 and _rel(gv, ov) <= 1e-10 and _rel(gm, om) <= 1e-10


def test_rollout_grad_central_differences_n64(cuda):
    # Central differences of the oracle's loss at N = 64 (FP64, h = 1e-6).
    b = inputs.plummer(64, seed=45)
    G, eps, dt, K = 1.0, 0.01, 1e-3, 200
    rng = np.random.default_rng(5)
    tgt = b.pos + rng.normal(0, 1e-3, b.pos.shape)
    gx, gv, gm, _ = _grads(cuda, "fp64", b, G, eps, dt, K, 20, tgt)

    def loss(x, v, m):
        xT, _, _ = oracle.kdk(x, v, m, G, eps, dt, K)
        return ((xT - tgt) ** 2).sum(-1).mean()

    h = 1e-6
    idx = rng.choice(64, 6, replace=False)
    for i in idx:
        for c in range(3):
            xp, xm = b.pos.copy(), b.pos.copy()
            xp[i, c] += h; xm[i, c] -= h
            fd = (loss(xp, b.vel, b.mass) - loss(xm, b.vel, b.mass)) / (2 * h)
            assert abs(fd - gx[i, c]) <= 1e-6 * np.abs(gx).max()
            vp, vm = b.vel.copy(), b.vel.copy()
            vp[i, c] += h; vm[i, c] -= h
            fd = (loss(b.pos, vp, b.mass) - loss(b.pos, vm, b.mass)) / (2 * h)
            assert abs(fd - gv[i, c]) <= 1e-6 * np.abs(gv).max()
        mp, mm = b.mass.copy(), b.mass.copy()
        mp[i] += h; mm[i] -= h
        fd = (loss(b.pos, b.vel, mp) - loss(b.pos, b.vel, mm)) / (2 * h)
        assert abs(fd - gm[i]) <= 1e-6 * np.abs(gm).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32_comp", 1e-3), ("df64", 1e-10)])
def test_rollout_grad_oracle_adjoint_n1024(cuda, prec, tol):
    # Differentiation workload at N = 1024: 200 steps of dt = 1e-3, eps = 0.01,
    # checkpoints every 20 steps, target from the oracle run of a perturbed start.
    b, dx = inputs.plummer_with_perturbation(1024, seed=4)
    G, eps, dt, K = 1.0, 0.01, 1e-3, 200
    tgt, _, _ = oracle.kdk(b.pos + dx, b.vel, b.mass, G, eps, dt, K)
    gx, gv, gm, _ = _grads(cuda, prec, b, G, eps, dt, K, 20, tgt)
    xT, _, _ = oracle.kdk(b.pos, b.vel, b.mass, G, eps, dt, K)
    ox, ov, om = oracle.kdk_grad(b.pos, b.vel, b.mass, G, eps, dt, K,
                                 2.0 / b.n * (xT - tgt), np.zeros_like(xT))
    assert _rel(gx, ox) <= tol and _rel(gv, ov) <= tol and _rel(gm, om) <= tol


def test_checkpoint_interval_does_not_change_gradients(cuda):
    b = inputs.plummer(300, seed=46)
    tgt = b.pos * 1.01
    ref = _grads(cuda, "fp32_comp", b, 1.0, 0.01, 1e-3, 40, 40, tgt)
    for every in (1, 7, 20):
        g = _grads(cuda, "fp32_comp", b, 1.0, 0.01, 1e-3, 40, every, tgt)
        for a, r in zip(g[:3], ref[:3]):
            assert np.array_equal(a, r)


def test_zero_steps_passes_gradients_through(cuda):
    b = inputs.plummer(20, seed=47)
    with nbody.NBody(20, "fp64") as nb:
        x0 = to_dev(b.pos, cuda).requires_grad_()
        v0 = to_dev(b.vel, cuda).requires_grad_()
        m = to_dev(b.mass, cuda).requires_grad_()
        xT, vT = rollout(nb, x0, v0, m, 1.0, 0.01, 1e-3, 0, 20)
        (xT.sum() + 2 * vT.sum()).backward()
    assert np.all(host(x0.grad) == 1) and np.all(host(v0.grad) == 2)
    assert np.all(host(m.grad) == 0)
