"""FP64 CPU oracle for the softened direct-sum n-body path (ctypes shim).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may call this module; the product path never
does.  The arithmetic lives in ``nbody_oracle.c`` (plain C, FP64, OpenMP over
bodies), which shares nothing with the CUDA library.

Every function takes and returns float64 numpy arrays: positions and
velocities (n, 3), masses (n,).  Function-level citations are in the C file:
the force sum is the exact form of the paper's force calculation (Sec. IV-A,
IV-B); the leapfrog is the reading of "Move_bodies" (Sec. IV-B pseudo-code);
the diagnostics and adjoints have no counterpart in the paper and follow from
the same formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    i64, dbl = ctypes.c_int64, ctypes.c_double
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_accel.argtypes = [i64, _D, _D, dbl, dbl, _D]
    lib.oracle_accel_rows.argtypes = [i64, _D, _D, dbl, dbl, i64, _I, _D]
    lib.oracle_energy.argtypes = [i64, _D, _D, _D, dbl, dbl, _D]
    lib.oracle_kdk.argtypes = [i64, _D, _D, _D, dbl, dbl, dbl, i64, _D]
    lib.oracle_force_vjp.argtypes = [i64, _D, _D, dbl, dbl, _D, _D, _D]
    lib.oracle_kdk_grad.argtypes = [i64, _D, _D, _D, dbl, dbl, dbl, i64,
                                    _D, _D, _D, _D, _D]
    lib.oracle_kdk_grad.restype = ctypes.c_int
    lib.oracle_bh_forces.argtypes = [i64, _D, _D, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                     _D, _I, _I]
    lib.oracle_bh_forces.restype = ctypes.c_int
    lib.oracle_bh_groups.argtypes = [i64, _D, _D, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                     i64, _I, _I, _D, _I]
    lib.oracle_bh_groups.restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.oracle_orb.argtypes = [i64, _D, ctypes.c_int, i32p]
    lib.oracle_orb.restype = ctypes.c_int
    lib.oracle_bh_sharded.argtypes = [i64, _D, _D, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, i32p, _D, _I, _I]
    lib.oracle_bh_sharded.restype = ctypes.c_int
    lib.oracle_bh_let.argtypes = [i64, _D, _D, dbl, ctypes.c_int, f32p, f32p, i64, _I, i32p,
                                  i32p, _I, _I, _I, f32p, f32p, _I]
    lib.oracle_bh_let.restype = ctypes.c_int
    lib.oracle_fmm_forces.argtypes = [i64, _D, _D, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                      _D, _I, _I]
    lib.oracle_fmm_forces.restype = ctypes.c_int
    lib.oracle_fmm_deriv.argtypes = [ctypes.c_int, _D, dbl, _D]
    lib.oracle_fmm_deriv.restype = ctypes.c_int
    lib.oracle_fmm_pair.argtypes = [ctypes.c_int, _D, _D, dbl, i64, _D, _D, i64, _D, _D]
    lib.oracle_fmm_pair.restype = ctypes.c_int
    for f in (lib.oracle_accel, lib.oracle_accel_rows, lib.oracle_energy,
              lib.oracle_kdk, lib.oracle_force_vjp):
        f.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(_D)


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def accel(pos, mass, G=1.0, eps=0.0):
    """a_i = G sum_{j != i} m_j d_ij / (|d_ij|^2 + eps^2)^{3/2}, (n, 3)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    out = np.zeros((n, 3))
    _load().oracle_accel(n, _p(x), _p(m), float(G), float(eps), _p(out))
    return out


def accel_rows(pos, mass, rows, G=1.0, eps=0.0):
    """Accelerations of the bodies listed in ``rows`` only, (len(rows), 3)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    r = np.ascontiguousarray(rows, dtype=np.int64)
    if r.size and (r.min() < 0 or r.max() >= n):
        raise IndexError("row index out of range")
    out = np.zeros((r.size, 3))
    _load().oracle_accel_rows(n, _p(x), _p(m), float(G), float(eps), r.size,
                              r.ctypes.data_as(_I), _p(out))
    return out


def energy(pos, vel, mass, G=1.0, eps=0.0):
    """[E_kin, E_pot, E_tot, Px, Py, Pz, Fx, Fy, Fz] (F = sum m a)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    v = _f64(vel, (n, 3))
    out = np.zeros(9)
    _load().oracle_energy(n, _p(x), _p(v), _p(m), float(G), float(eps), _p(out))
    return out


def kdk(pos, vel, mass, G, eps, dt, nsteps):
    """nsteps KDK leapfrog steps; returns (pos, vel, acc) at the end."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3)).copy()
    v = _f64(vel, (n, 3)).copy()
    a = np.zeros((n, 3))
    _load().oracle_kdk(n, _p(x), _p(v), _p(m), float(G), float(eps), float(dt),
                       int(nsteps), _p(a))
    return x, v, a


def force_vjp(pos, mass, lam, G=1.0, eps=0.0):
    """(dL/dx, dL/dm) of L through a = F(x, m), given lam = dL/da."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    l = _f64(lam, (n, 3))
    gx = np.zeros((n, 3))
    gm = np.zeros(n)
    _load().oracle_force_vjp(n, _p(x), _p(m), float(G), float(eps), _p(l),
                             _p(gx), _p(gm))
    return gx, gm


def kdk_grad(pos, vel, mass, G, eps, dt, nsteps, gxT, gvT):
    """Gradients (dL/dx0, dL/dv0, dL/dm) through nsteps KDK steps."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    v = _f64(vel, (n, 3))
    gx = _f64(gxT, (n, 3))
    gv = _f64(gvT, (n, 3))
    ox = np.zeros((n, 3)); ov = np.zeros((n, 3)); om = np.zeros(n)
    rc = _load().oracle_kdk_grad(n, _p(x), _p(v), _p(m), float(G), float(eps),
                                 float(dt), int(nsteps), _p(gx), _p(gv),
                                 _p(ox), _p(ov), _p(om))
    if rc != 0:
        raise MemoryError("oracle_kdk_grad: allocation failed")
    return ox, ov, om


def bh_forces(pos, mass, G=1.0, eps=0.0, theta=0.5, leaf_cap=16, group=32, counts=False):
    """Barnes-Hut accelerations (paper Sec. IV-A, readings in nbody_oracle.c).

    Returns acc (n, 3), stats {nodes, leaves, cell_interactions,
    body_interactions} and, with counts=True, per-body (cells, bodies) list
    sizes (n, 2).
    """
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    out = np.zeros((n, 3))
    st = np.zeros(4, dtype=np.int64)
    cnt = np.zeros((n, 2), dtype=np.int64) if counts else None
    rc = _load().oracle_bh_forces(n, _p(x), _p(m), float(G), float(eps), float(theta),
                                  int(leaf_cap), int(group), _p(out), st.ctypes.data_as(_I),
                                  cnt.ctypes.data_as(_I) if counts else None)
    if rc != 0:
        raise ValueError("oracle_bh_forces: bad leaf_cap/group")
    stats = dict(zip(("nodes", "leaves", "cell_interactions", "body_interactions"),
                     (int(v) for v in st)))
    return (out, stats, cnt) if counts else (out, stats)


def bh_groups(pos, mass, G, eps, theta, leaf_cap, group, sel):
    """The tree code of bh_forces for the groups `sel` only (indices in key
    order), over the tree of all bodies.  Returns (idx, acc, counts): idx
    (len(sel), group) body indices (-1 past the last body), acc (n, 3) and
    counts (n, 2) filled for those bodies (NaN / -1 elsewhere)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    idx = np.full((sel.size, group), -1, dtype=np.int64)
    acc = np.full((n, 3), np.nan)
    cnt = np.full((n, 2), -1, dtype=np.int64)
    rc = _load().oracle_bh_groups(n, _p(x), _p(m), float(G), float(eps), float(theta),
                                  int(leaf_cap), int(group), sel.size, sel.ctypes.data_as(_I),
                                  idx.ctypes.data_as(_I), _p(acc), cnt.ctypes.data_as(_I))
    if rc != 0:
        raise ValueError("oracle_bh_groups: bad leaf_cap/group or group index")
    return idx, acc, cnt


def orb(pos, P):
    """Processor of each body under orthogonal recursive bisection into P
    equal-count domains (paper Sec. IV-B; readings in nbody_oracle.c)."""
    x = _f64(pos)
    n = x.shape[0]
    out = np.zeros(n, dtype=np.int32)
    if _load().oracle_orb(n, _p(x), int(P), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))):
        raise ValueError("oracle_orb: P must be >= 1")
    return out


def bh_sharded(pos, mass, G, eps, theta, leaf_cap, group, rank, P):
    """The parallel tree code's accelerations (paper Sec. IV-B): every
    processor's tree over its own bodies, walked by every processor's groups.
    Returns acc (n, 3), stats {nodes, leaves, cell_interactions,
    body_interactions} and per body (cells, bodies met, bodies covered)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    r = np.ascontiguousarray(rank, dtype=np.int32)
    out = np.zeros((n, 3))
    st = np.zeros(4, dtype=np.int64)
    cnt = np.zeros((n, 3), dtype=np.int64)
    rc = _load().oracle_bh_sharded(n, _p(x), _p(m), float(G), float(eps), float(theta),
                                   int(leaf_cap), int(group), int(P),
                                   r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _p(out),
                                   st.ctypes.data_as(_I), cnt.ctypes.data_as(_I))
    if rc != 0:
        raise ValueError("oracle_bh_sharded: bad arguments")
    stats = dict(zip(("nodes", "leaves", "cell_interactions", "body_interactions"),
                     (int(v) for v in st)))
    return out, stats, cnt


def bh_let(pos, mass, theta, leaf_cap, box_lo, box_hi):
    """The tree over (pos, mass) and each node's kind in the locally
    essential tree sent to a destination whose bodies lie in the float32 box
    [box_lo, box_hi]: 0 not sent, 1 sent alone, 2 sent with its children,
    3 a leaf sent with its bodies.  Returns a dict of per-node arrays (build
    order: kind, level, prefix, child (k, 8), range (k, 2), lo, hi (k, 3)
    float32) and perm (key order -> body)."""
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    blo = np.ascontiguousarray(box_lo, dtype=np.float32)
    bhi = np.ascontiguousarray(box_hi, dtype=np.float32)
    lib = _load()
    f32p = ctypes.POINTER(ctypes.c_float)
    i32p = ctypes.POINTER(ctypes.c_int32)
    nn = np.zeros(1, dtype=np.int64)
    none = ctypes.POINTER(ctypes.c_int64)()
    if lib.oracle_bh_let(n, _p(x), _p(m), float(theta), int(leaf_cap), blo.ctypes.data_as(f32p),
                         bhi.ctypes.data_as(f32p), 0, nn.ctypes.data_as(_I), None, None, none,
                         none, none, None, None, none):
        raise ValueError("oracle_bh_let: bad arguments")
    k = int(nn[0])
    d = {"kind": np.zeros(k, np.int32), "level": np.zeros(k, np.int32),
         "prefix": np.zeros(k, np.int64), "child": np.zeros((k, 8), np.int64),
         "range": np.zeros((k, 2), np.int64), "lo": np.zeros((k, 3), np.float32),
         "hi": np.zeros((k, 3), np.float32), "perm": np.zeros(n, np.int64)}
    lib.oracle_bh_let(n, _p(x), _p(m), float(theta), int(leaf_cap), blo.ctypes.data_as(f32p),
                      bhi.ctypes.data_as(f32p), k, nn.ctypes.data_as(_I),
                      d["kind"].ctypes.data_as(i32p), d["level"].ctypes.data_as(i32p),
                      d["prefix"].ctypes.data_as(_I), d["child"].ctypes.data_as(_I),
                      d["range"].ctypes.data_as(_I), d["lo"].ctypes.data_as(f32p),
                      d["hi"].ctypes.data_as(f32p), d["perm"].ctypes.data_as(_I))
    return d


def fmm_multi_indices(p):
    """Multi-indices (a, b, c) of order <= p in the oracle's slot order
    (order by order; within an order a descending, then b descending)."""
    return [(a, k - a - c, c) for k in range(p + 1) for a in range(k, -1, -1)
            for c in range(0, k - a + 1)]


def fmm_deriv(p, r, eps=0.0):
    """d^n g(r) for g(r) = (|r|^2 + eps^2)^{-1/2}, every |n| <= p, in the
    slot order of fmm_multi_indices."""
    r = _f64(r, (3,))
    out = np.zeros((p + 1) * (p + 2) * (p + 3) // 6)
    if _load().oracle_fmm_deriv(int(p), _p(r), float(eps), _p(out)) != 0:
        raise ValueError("oracle_fmm_deriv: order out of range")
    return out


def fmm_pair(p, zA, zB, eps, xs, ms, xt):
    """The FMM's expansion chain alone: sources (xs, ms) expanded about zB,
    translated to a local expansion about zA and differentiated at the
    targets xt; accelerations (G = 1), (len(xt), 3)."""
    ms = _f64(ms)
    xs = _f64(xs, (ms.shape[0], 3))
    xt = np.ascontiguousarray(xt, dtype=np.float64).reshape(-1, 3)
    zA, zB = _f64(zA, (3,)), _f64(zB, (3,))
    out = np.zeros((xt.shape[0], 3))
    if _load().oracle_fmm_pair(int(p), _p(zA), _p(zB), float(eps), ms.shape[0], _p(xs), _p(ms),
                               xt.shape[0], _p(xt), _p(out)) != 0:
        raise ValueError("oracle_fmm_pair: order out of range")
    return out


def fmm_forces(pos, mass, G=1.0, eps=0.0, theta=0.5, order=4, leaf_cap=16, counts=False):
    """Fast-multipole accelerations (readings in nbody_oracle.c).

    Returns acc (n, 3), stats {nodes, leaves, expansions, direct_pairs} and,
    with counts=True, per body (source cells, bodies in them, direct
    partners) (n, 3).
    """
    m = _f64(mass)
    n = m.shape[0]
    x = _f64(pos, (n, 3))
    out = np.zeros((n, 3))
    st = np.zeros(4, dtype=np.int64)
    cnt = np.zeros((n, 3), dtype=np.int64) if counts else None
    rc = _load().oracle_fmm_forces(n, _p(x), _p(m), float(G), float(eps), float(theta),
                                   int(order), int(leaf_cap), _p(out), st.ctypes.data_as(_I),
                                   cnt.ctypes.data_as(_I) if counts else None)
    if rc != 0:
        raise ValueError(f"oracle_fmm_forces: bad arguments ({rc})")
    stats = dict(zip(("nodes", "leaves", "expansions", "direct_pairs"), (int(v) for v in st)))
    return (out, stats, cnt) if counts else (out, stats)
