"""nb_forces_noalloc: the allocation-free force entry point.

Some callers cannot allocate device memory: code whose device memory
belongs to another allocator or to a fixed budget, and latency-critical
loops where a cudaMalloc could block.  This test calls the entry point
through the C ABI on two calls in a row and compares each result with
nb_forces (the context-based entry point, same float32 compensated
arithmetic) and with the FP64 oracle, within the float32 tolerance of the
parity tests (per-body relative difference RMS <= 1e-5, max <= 1e-4).  The
file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1211_2292_gb300 import inputs, nbody
from helpers import host, relerr_per_body, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(lib, x, m, G, eps, out):
    st = lib.nb_forces_noalloc(m.shape[0], x.data_ptr(), m.data_ptr(), G, eps, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    return st


def _within_fp32_bound(a, ref):
    e = relerr_per_body(a, ref)
    return bool(np.isfinite(e).all() and np.sqrt((e ** 2).mean()) <= 1e-5 and e.max() <= 1e-4)


def test_noalloc_matches_nb_forces_and_oracle_on_two_calls(cuda):
    lib = nbody.load()
    # two different systems in a row: the shared scratch must not leak state
    for n, seed, eps in ((5000, 71, 0.01), (777, 72, 0.02)):
        b = inputs.plummer(n, seed=seed)
        x, m = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
        with nbody.NBody(n, "fp32_comp") as nb:
            ref = host(nb.forces(x, m, 1.0, eps))
        out = torch.full((n, 3), float("nan"), dtype=torch.float64, device=cuda)
        assert _noalloc(lib, x, m, 1.0, eps, out) == 0
        torch.cuda.synchronize()
        got = host(out)
        assert _within_fp32_bound(got, ref)
        assert _within_fp32_bound(got, oracle.accel(b.pos, b.mass, 1.0, eps))


def test_noalloc_limits(cuda):
    lib = nbody.load()
    n_max = 65536
    x = torch.zeros((n_max + 1, 3), dtype=torch.float64, device=cuda)
    m = torch.ones(n_max + 1, dtype=torch.float64, device=cuda)
    a = torch.zeros_like(x)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.nb_forces_noalloc(n_max + 1, x.data_ptr(), m.data_ptr(), 1.0, 0.1, a.data_ptr(), s) == 1
    assert lib.nb_forces_noalloc(-1, x.data_ptr(), m.data_ptr(), 1.0, 0.1, a.data_ptr(), s) == 1
    assert lib.nb_forces_noalloc(0, None, None, 1.0, 0.1, None, s) == 0
    hx = np.zeros((4, 3))
    assert lib.nb_forces_noalloc(4, hx.ctypes.data, m.data_ptr(), 1.0, 0.1, a.data_ptr(), s) == 1
    # the largest allowed size runs
    b = inputs.plummer(n_max, seed=73)
    xb, mb = to_dev(b.pos, cuda), to_dev(b.mass, cuda)
    out = torch.empty((n_max, 3), dtype=torch.float64, device=cuda)
    assert _noalloc(lib, xb, mb, 1.0, 0.01, out) == 0
    with nbody.NBody(n_max, "fp32_comp") as nb:
        nb.set_order(0)
        ref = host(nb.forces(xb, mb, 1.0, 0.01))
    got = host(out)
    assert _within_fp32_bound(got, ref)
    rows = inputs.sample_rows(n_max, 512, seed=74)
    assert _within_fp32_bound(got[rows], oracle.accel_rows(b.pos, b.mass, rows, 1.0, 0.01))
