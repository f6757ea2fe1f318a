"""Host-side checks of libnbody.so that need no GPU: every symbol declared in
include/nbody.h is exported, the host scheduling helpers behave, and calls
without a device fail with a status instead of crashing."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1211_2292_gb300 import nbody

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = nbody.load()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(nbody.SIGNATURES), set(names) ^ set(nbody.SIGNATURES)


def test_null_context_is_rejected():
    lib = nbody.load()
    assert lib.nb_forces(None, 1, None, None, 1.0, 0.1, None) == 1
    assert lib.nb_sync(None) == 1
    assert lib.nb_destroy(None) == 0
    assert lib.nb_launch_count(None) == 0


def test_create_without_device_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = nbody.load()
    h = ctypes.c_void_p()
    st = lib.nb_create(ctypes.byref(h), 100, 2, 0, None)
    assert st == 2 and h.value is None
    assert lib.nb_last_error(None)
    assert lib.nb_create(None, 100, 2, 0, None) == 1
    assert lib.nb_create(ctypes.byref(h), -1, 2, 0, None) == 1
    assert lib.nb_create(ctypes.byref(h), 100, 7, 0, None) == 1


def test_variant_tables():
    for prec in ("fp64", "fp32", "fp32_comp", "df64"):
        v = nbody.variants(nbody.KIND_FORCE, prec)
        assert v and all(t % 32 == 0 and j % t == 0 for t, i, j in v)
        if prec != "fp64":
            assert all(i % 2 == 0 for _, i, _ in v)  # float32x2 pairs
    assert nbody.variants(nbody.KIND_BATCHED, "fp64") == []
    assert nbody.variants(nbody.KIND_BATCHED, "df64") == []
    # the double-float context differentiates in float64
    assert nbody.variants(nbody.KIND_VJP, "df64") == nbody.variants(nbody.KIND_VJP, "fp64")
    assert nbody.load().nb_variant_count(9, 0) == 0
    assert nbody.load().nb_variant_count(0, 4) == 0


def _waves_eff(items, slots):
    w = items / slots
    return w / math.ceil(w)


@pytest.mark.parametrize("n,tile,jt,slots", [(1 << 20, 512, 128, 760), (65536, 512, 128, 760),
                                             (1024, 512, 128, 760), (3000, 256, 256, 1216),
                                             (16384, 256, 128, 608)])
def test_choose_split(n, tile, jt, slots):
    it, jtiles = -(-n // tile), -(-n // jt)
    cap = 1 << 22
    s = nbody.choose_split(it, jtiles, slots, cap, tile)
    assert 1 <= s <= jtiles
    assert s == 1 or s * it * tile <= cap
    # never worse than no split, in the scheduler's own model
    per = jtiles / s
    assert _waves_eff(it * s, slots) * per / (per + 1) >= _waves_eff(it, slots) * jtiles / (jtiles + 1) - 1e-12
    if n >= 65536:
        assert _waves_eff(it * s, slots) > 0.9


def test_choose_split_degenerate():
    assert nbody.choose_split(0, 10, 100, 1 << 20, 256) == 1
    assert nbody.choose_split(10, 0, 100, 1 << 20, 256) == 1
    assert nbody.choose_split(4, 1000, 608, 1024, 256) == 1  # no room for partials


@pytest.mark.parametrize("cap", [0, 200_000])
@pytest.mark.parametrize("T,I,J", [(128, 2, 128), (128, 4, 128), (256, 2, 256), (64, 4, 128),
                                   (128, 6, 256), (64, 6, 128)])
def test_plan_batch_covers_every_pair_once(T, I, J, cap):
    from paper_1211_2292_gb300 import inputs
    sizes = [0, 1, 2, 64, 100, 255, 256, 257, 8192] + list(inputs.batch_sizes(60, seed=3))
    off = np.concatenate([[0], np.cumsum(sizes)])
    items = nbody.plan_batch_host(off, T, I, J, cap)
    TI = T * I
    lmax = min(32, T, J)
    jcover = np.zeros(off[-1], dtype=np.int64)  # j bodies met, summed over a body's items
    costs = []
    pieces = {}
    for i0, i_end, j0, j1, lanes, sys, ctr, pbase, chunk, nchunks in items:
        s_, e_ = off[sys], off[sys + 1]
        assert s_ <= i0 < i_end <= e_ and s_ <= j0 < j1 <= e_
        assert (j0 - s_) % J == 0  # chunks start on j-tile boundaries
        assert lanes in (1, 2, 4, 8, 16, 32) and lanes <= lmax
        assert i_end - i0 <= TI // lanes
        jcover[i0:i_end] += j1 - j0
        costs.append(-(-(j1 - j0) // J) * J // lanes)
        if nchunks == 1:
            assert ctr == -1 and (j0, j1) == (s_, e_)
        else:
            pieces.setdefault(ctr, []).append((chunk, nchunks, pbase, i0, i_end, j0, j1))
        if cap and nchunks == 1:
            # an unsplit piece stays under the cap unless it is one j-tile
            assert (TI // lanes) * (j1 - j0) <= cap or j1 - j0 <= J
    # every body meets every body of its system once
    assert np.array_equal(jcover, np.repeat(np.diff(off), np.diff(off)))
    assert costs == sorted(costs, reverse=True)
    # chunks of a split piece: one counter, contiguous slots, consecutive j ranges
    assert sorted(pieces) == list(range(len(pieces)))
    slots = []
    for ctr, ch in pieces.items():
        ch.sort()
        nch, pbase = ch[0][1], ch[0][2]
        assert [c[0] for c in ch] == list(range(nch)) and all(c[1:5] == ch[0][1:5] for c in ch)
        assert all(a[6] == b[5] for a, b in zip(ch, ch[1:]))
        slots.append((pbase, nch))
    slots.sort()
    assert not slots or slots[0][0] == 0
    assert all(a[0] + a[1] == b[0] for a, b in zip(slots, slots[1:]))
    if cap:
        assert pieces  # the 8192-body system is split
    # remainders go in pieces of TI / lanes bodies: little is left unfilled
    filled = sum(it[1] - it[0] for it in items if it[8] == 0)
    slots_ = sum(TI // it[4] for it in items if it[8] == 0)
    assert filled >= 0.75 * slots_


def test_plan_batch_rejects_bad_offsets():
    with pytest.raises(ValueError):
        nbody.plan_batch_host([1, 5], 128, 2, 128)
    with pytest.raises(ValueError):
        nbody.plan_batch_host([0, 5, 3], 128, 2, 128)
    assert nbody.plan_batch_host([0], 128, 2, 128) == []


def test_oracle_and_cuda_path_share_nothing():
    # Neither side imports the other; only tests, the smoke check and the
    # bench's CPU leg touch the oracle.
    pkg = os.path.join(ROOT, "paper_1211_2292_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "nbody_oracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1211_2292_gb300" not in text and "nbody.h" not in text, f
