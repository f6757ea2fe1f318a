"""The workloads at full size, in the library's tuned configuration (the
packaged GB300 tuning table, as bench.py uses it), checked against the FP64
oracle on sampled outputs it computes one by one, or through properties that
hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_2292_gb300 import inputs, nbody, tune
from paper_1211_2292_gb300.autograd import rollout
from helpers import host, relerr_per_body, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _ctx(n, prec):
    nb = nbody.NBody(n, prec)
    tune.apply(nb)
    return nb


def test_precision_workload_n65536(cuda):
    # N = 65,536 Plummer sphere, seed 1, eps = 0.005: FP32 compensated forces on
    # 4096 sampled bodies vs the oracle; 100 steps of dt = 5e-4 in FP32 and FP64,
    # energy compared with the FP64 GPU run.
    b = inputs.plummer(65536, seed=1)
    G, eps, dt, K = 1.0, 0.005, 5e-4, 100
    rows = inputs.sample_rows(b.n, 4096, seed=1)
    ref = oracle.accel_rows(b.pos, b.mass, rows, G, eps)
    res = {}
    for prec in ("fp32_comp", "fp64"):
        with _ctx(b.n, prec) as nb:
            x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
            a = nb.forces(x, m, G, eps)
            e = relerr_per_body(host(a)[rows], ref)
            if prec == "fp64":
                assert e.max() <= 1e-12
            else:
                assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4
            e0 = nb.energy(x, v, m, G, eps)
            nb.step(x, v, m, G, eps, dt, K, a, acc_valid=True)
            e1 = nb.energy(x, v, m, G, eps)
            res[prec] = (e0, e1, host(x))
    e0, e1, _ = res["fp64"]
    f0, f1, _ = res["fp32_comp"]
    assert e0[2] == f0[2]  # the diagnostics are float64 in every mode
    drift64 = abs(e1[2] - e0[2]) / abs(e0[2])
    drift32 = abs(f1[2] - f0[2]) / abs(f0[2])
    assert drift64 < 1e-5
    assert abs(f1[2] - e1[2]) <= 1e-7 * abs(e0[2]), (drift32, drift64)
    assert np.abs(res["fp32_comp"][2] - res["fp64"][2]).max() <= 1e-8


def test_throughput_workload_n2p20(cuda):
    # Two Plummer spheres, N = 2^20, eps = 0.002, seed 2, FP32 compensated with
    # Morton-ordered tiles: forces on 4096 sampled bodies vs the oracle, then
    # one bench step (1 + 10 force evaluations) and its invariants.
    b = inputs.two_plummer(524288, seed=2)
    G, eps, dt = 1.0, 0.002, 1e-3
    rows = inputs.sample_rows(b.n, 4096, seed=1)
    ref = oracle.accel_rows(b.pos, b.mass, rows, G, eps)
    with _ctx(b.n, "fp32_comp") as nb:
        x, v, m = to_dev(b.pos, cuda), to_dev(b.vel, cuda), to_dev(b.mass, cuda)
        a0 = host(nb.forces(x, m, G, eps))
        e = relerr_per_body(a0[rows], ref)
        assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4
        acc = torch.empty_like(x)
        nb.step(x, v, m, G, eps, dt, 10, acc)
        nb.sync()
        a_loop = host(acc)
        a_again = host(nb.forces(x, m, G, eps))
    # the cached force after the loop is F(final positions), bit for bit
    assert np.array_equal(a_loop, a_again)
    xs, vs = host(x), host(v)
    assert np.isfinite(xs).all() and np.isfinite(vs).all()
    # momentum: sum m a vanishes up to the float32 force error
    p0 = (b.mass[:, None] * b.vel).sum(0)
    p1 = (b.mass[:, None] * vs).sum(0)
    scale = (b.mass * np.linalg.norm(a0, axis=1)).sum() * 10 * dt
    assert np.abs(p1 - p0).max() <= 1e-5 * scale


def test_batched_workload_512_systems(cuda):
    # 512 systems, N_k log-uniform in [64, 8192], seed 3, eps = 0.01, FP32
    # compensated, 100 steps of dt = 1e-3 as one graph launch.
    bodies, off = inputs.plummer_batch(512, 64, 8192, seed=3)
    G, eps, dt, K = 1.0, 0.01, 1e-3, 100
    sizes = np.diff(off)
    pick = list(np.argsort(sizes)[:3]) + list(np.argsort(sizes)[-2:]) + [17, 250]
    out = []
    for graph in (True, False):
        with _ctx(bodies.n, "fp32_comp") as nb:
            nb.batch_plan(off)
            x, v, m = (to_dev(bodies.pos, cuda), to_dev(bodies.vel, cuda),
                       to_dev(bodies.mass, cuda))
            a = nb.forces_batched(x, m, G, eps)
            a0 = host(a)
            nb.step_batched(x, v, m, G, eps, dt, K, a, acc_valid=True, graph=graph)
            nb.sync()
            out.append((a0, host(x), host(v)))
    for p, q in zip(*out):
        assert np.array_equal(p, q)
    a0, xs, _ = out[0]
    for k in pick:
        s, e = off[k], off[k + 1]
        ref = oracle.accel(bodies.pos[s:e], bodies.mass[s:e], G, eps)
        err = relerr_per_body(a0[s:e], ref)
        assert np.sqrt((err ** 2).mean()) <= 1e-5 and err.max() <= 1e-4, (k, err.max())
    for k in np.argsort(sizes)[:2]:  # the smallest systems, run through by the oracle
        s, e = off[k], off[k + 1]
        ox, _, _ = oracle.kdk(bodies.pos[s:e], bodies.vel[s:e], bodies.mass[s:e], G, eps, dt, K)
        assert np.abs(xs[s:e] - ox).max() <= 1e-8


def test_differentiation_workload_n16384(cuda):
    # N = 16,384, eps = 0.01, 200 steps of dt = 1e-3, seed 4; loss = mean over
    # bodies of |x_T - x*|^2 with x* the oracle run of the perturbed start;
    # gradients from the adjoint kernels with checkpoints every 20 steps.  The
    # oracle's loss is differenced along the gradient direction of each input.
    b, dx = inputs.plummer_with_perturbation(16384, seed=4)
    G, eps, dt, K = 1.0, 0.01, 1e-3, 200
    tgt, _, _ = oracle.kdk(b.pos + dx, b.vel, b.mass, G, eps, dt, K)
    with _ctx(b.n, "fp32_comp") as nb:
        x0 = to_dev(b.pos, cuda).requires_grad_()
        v0 = to_dev(b.vel, cuda).requires_grad_()
        m = to_dev(b.mass, cuda).requires_grad_()
        xT, _ = rollout(nb, x0, v0, m, G, eps, dt, K, 20)
        loss = ((xT - to_dev(tgt, cuda)) ** 2).sum(-1).mean()
        loss.backward()
        gx, gv, gm = host(x0.grad), host(v0.grad), host(m.grad)

    def L(x, v, mm):
        xt, _, _ = oracle.kdk(x, v, mm, G, eps, dt, K)
        return ((xt - tgt) ** 2).sum(-1).mean()

    base = L(b.pos, b.vel, b.mass)
    assert abs(base - float(loss.detach())) <= 1e-6 * base
    for g, which in ((gx, 0), (gv, 1), (gm, 2)):
        u = g / np.linalg.norm(g)
        h = 1e-3 * (np.abs(b.pos).mean() if which == 0 else
                    np.abs(b.vel).mean() if which == 1 else b.mass.mean())
        args_p = [b.pos, b.vel, b.mass]
        args_m = [b.pos, b.vel, b.mass]
        args_p[which] = args_p[which] + h * u
        args_m[which] = args_m[which] - h * u
        fd = (L(*args_p) - L(*args_m)) / (2 * h)
        assert abs(fd - np.linalg.norm(g)) <= 1e-3 * np.linalg.norm(g), (which, fd, np.linalg.norm(g))


@pytest.mark.parametrize("group", [64, 32])
def test_tree_workload_n2p20_sampled_groups(cuda, group):
    # The tree bench's workload and launch configuration (two-Plummer 2^20,
    # theta 0.5, leaves <= 16, dynamic schedule): every body of 48 seeded
    # groups meets exactly the oracle tree's lists, with forces within the
    # float32 bound; the totals agree with the per-body counts.
    b = inputs.two_plummer(524_288, seed=2)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a, cnt = nb.tree_forces(x, m, 1.0, 0.002, 0.5, 16, counts=True, group=group)
        nb.sync()
        st = nb.tree_stats()
    a, cnt = host(a), host(cnt).astype(np.int64)
    ngroups = (b.n + group - 1) // group
    sel = np.sort(np.random.default_rng(5).choice(ngroups, 48, replace=False))
    idx, ra, rc = oracle.bh_groups(b.pos, b.mass, 1.0, 0.002, 0.5, 16, group, sel)
    ii = idx[idx >= 0]
    assert ii.size == 48 * group
    assert np.array_equal(cnt[ii], rc[ii])
    e = relerr_per_body(a[ii], ra[ii])
    assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4
    assert st["cell_interactions"] == cnt[:, 0].sum()
    assert st["body_interactions"] == cnt[:, 1].sum()


def test_fmm_workload_n2p20_whole_run(cuda):
    # The FMM bench's workload and configuration (two-Plummer 2^20, theta 0.6,
    # order 6, leaves <= 64): the whole oracle FMM (about 20 s on the host
    # cores) against the GPU's, body by body: the same source cells, bodies
    # and direct partners for every body, the same totals, forces within the
    # float32 bound of the rms acceleration; every body meets all others once.
    b = inputs.two_plummer(524_288, seed=2)
    x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    with nbody.NBody(b.n, "fp32_comp") as nb:
        a, cnt = nb.fmm_forces(x, m, 1.0, 0.002, 0.6, 6, 64, counts=True)
        nb.sync()
        st = nb.fmm_stats()
    a, cnt = host(a), host(cnt).astype(np.int64)
    ra, rst, rc = oracle.fmm_forces(b.pos, b.mass, 1.0, 0.002, 0.6, 6, 64, counts=True)
    assert st == rst
    assert np.array_equal(cnt, rc)
    assert np.all(cnt[:, 1] + cnt[:, 2] == b.n)
    rms = np.sqrt((np.linalg.norm(ra, axis=1) ** 2).mean())
    e = np.linalg.norm(a - ra, axis=1) / rms
    assert np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4
