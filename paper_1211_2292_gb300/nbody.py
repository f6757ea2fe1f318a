"""Thin ctypes binding of libnbody.so (the C ABI in include/nbody.h).

Argument marshalling only: every array is a contiguous float64 CUDA tensor
whose device pointer is handed to the library, and every step of the
computation runs in the library's CUDA kernels.  There is no CPU path: if
the library cannot be loaded, or a call fails, an exception is raised.

The functions keep the C names (``nb_forces`` ...); :class:`NBody` wraps a
context for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

NB_FP64, NB_FP32, NB_FP32_COMP, NB_DF64 = 0, 1, 2, 3
PRECISIONS = {"fp64": NB_FP64, "fp32": NB_FP32, "fp32_comp": NB_FP32_COMP, "df64": NB_DF64}
NB_ACC_VALID, NB_USE_GRAPH = 1, 2
NB_BWD_AT_END, NB_BWD_AT_START = 1, 2
KIND_FORCE, KIND_BATCHED, KIND_VJP = 0, 1, 2
STATUS = {0: "NB_OK", 1: "NB_EINVAL", 2: "NB_ECUDA", 3: "NB_ENOMEM", 4: "NB_ENONFINITE",
          5: "NB_ETIMEOUT"}

_lock = threading.Lock()
_lib = None

_c_i64, _c_dbl, _c_vp, _c_int, _c_uint = (ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_uint)

# name -> (restype, argtypes); mirrors include/nbody.h
SIGNATURES = {
    "nb_create": (_c_int, [ctypes.POINTER(_c_vp), _c_i64, _c_int, _c_int, _c_vp]),
    "nb_destroy": (_c_int, [_c_vp]),
    "nb_set_stream": (_c_int, [_c_vp, _c_vp]),
    "nb_last_error": (ctypes.c_char_p, [_c_vp]),
    "nb_sync": (_c_int, [_c_vp]),
    "nb_forces": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_vp]),
    "nb_step": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_i64,
                         _c_vp, _c_uint]),
    "nb_rollout": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_i64,
                            _c_vp, _c_uint, _c_i64, _c_vp, _c_vp]),
    "nb_energy": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl,
                           ctypes.POINTER(_c_dbl)]),
    "nb_forces_backward": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_vp, _c_vp,
                                    _c_vp]),
    "nb_step_backward": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_i64,
                                  _c_vp, _c_vp, _c_vp, _c_uint]),
    "nb_batch_plan": (_c_int, [_c_vp, _c_i64, ctypes.POINTER(_c_i64)]),
    "nb_forces_batched": (_c_int, [_c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_vp]),
    "nb_step_batched": (_c_int, [_c_vp, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_i64,
                                 _c_vp, _c_uint]),
    "nb_variant_count": (_c_int, [_c_int, _c_int]),
    "nb_variant_info": (_c_int, [_c_int, _c_int, _c_int, ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "nb_tune_set": (_c_int, [_c_vp, _c_int, _c_i64, _c_i64, _c_int, _c_int]),
    "nb_tune_get": (_c_int, [_c_vp, _c_int, _c_i64, ctypes.POINTER(_c_int),
                             ctypes.POINTER(_c_int)]),
    "nb_launch_count": (_c_i64, [_c_vp]),
    "nb_set_order": (_c_int, [_c_vp, _c_int, _c_i64]),
    "nb_profile": (_c_int, [_c_vp, _c_int]),
    "nb_profile_read": (_c_int, [_c_vp, _c_int, ctypes.POINTER(_c_i64), ctypes.POINTER(_c_dbl)]),
    "nb_device_info": (_c_int, [_c_vp, _c_i64, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "nb_tree_forces": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int, _c_int,
                                _c_vp, _c_vp]),
    "nb_tree_step": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int,
                              _c_int, _c_dbl, _c_i64, _c_vp, _c_uint]),
    "nb_tree_stats": (_c_int, [_c_vp, ctypes.POINTER(_c_i64)]),
    "nb_tree_schedule": (_c_int, [_c_vp, _c_int, _c_int]),
    "nb_fmm_forces": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int, _c_int,
                               _c_vp, _c_vp]),
    "nb_fmm_stats": (_c_int, [_c_vp, ctypes.POINTER(_c_i64)]),
    "nb_fmm_reserve": (_c_int, [_c_vp, _c_i64]),
    "nb_fmm_step": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int,
                             _c_int, _c_dbl, _c_i64, _c_vp, _c_uint]),
    "nb_forces_noalloc": (_c_int, [_c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_vp, _c_vp]),
    "nb_orb_box": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_int, ctypes.POINTER(_c_dbl)]),
    "nb_orb_hist": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_int,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_uint64), _c_int, ctypes.POINTER(_c_i64)]),
    "nb_orb_cut": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_int,
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)]),
    "nb_orb_pack": (_c_int, [_c_vp, _c_i64, _c_vp, _c_int, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                             _c_vp, _c_vp, _c_vp, ctypes.POINTER(_c_i64)]),
    "nb_orb_order": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                              _c_vp]),
    "nb_let_build": (_c_int, [_c_vp, _c_i64, _c_vp, _c_vp, _c_int, ctypes.POINTER(ctypes.c_float)]),
    "nb_let_export": (_c_int, [_c_vp, _c_dbl, ctypes.POINTER(ctypes.c_float), _c_vp, _c_i64,
                               ctypes.POINTER(_c_i64)]),
    "nb_let_forces": (_c_int, [_c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int, _c_i64,
                               ctypes.POINTER(_c_vp), _c_vp, _c_vp]),
    "nb_choose_split": (_c_int, [_c_i64, _c_i64, _c_i64, _c_i64, _c_i64]),
    "nb_plan_batch_host": (_c_i64, [_c_i64, ctypes.POINTER(_c_i64), _c_int, _c_int, _c_int,
                                    _c_i64, ctypes.POINTER(ctypes.c_int32), _c_i64]),
}


class NBodyError(RuntimeError):
    def __init__(self, func, status, msg):
        super().__init__(f"{func}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnbody.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with "
                               "`python -m paper_1211_2292_gb300.build`")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(t, name, n3=None):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n3 is not None and t.numel() < n3:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n3}")
    return t.data_ptr() if t.numel() else None


def _ptr_i32(t, name, numel):
    """Device pointer of a contiguous int32 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32
            and t.is_contiguous() and t.numel() >= numel):
        raise ValueError(f"{name} must be a contiguous int32 CUDA tensor of {numel} elements")
    return t.data_ptr() if t.numel() else None


def _ptr_typed(t, name, dtype, numel):
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
            and t.is_contiguous() and t.numel() >= numel):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor of {numel} elements")
    return t.data_ptr() if t.numel() else None


def _host_array(ctype, values):
    vals = [int(v) for v in values]
    return (ctype * max(len(vals), 1))(*vals)


def _check(ctx, func, status):
    if status != 0:
        msg = load().nb_last_error(ctx).decode(errors="replace")
        raise NBodyError(func, status, msg)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class NBody:
    """A library context: precision, device, stream and scratch for n <= n_max."""

    def __init__(self, n_max: int, precision: str = "fp32_comp", device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1211_2292_gb300 needs a CUDA device; none is available")
        self.lib = load()
        self.precision = precision
        self.device = device
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            st = self.lib.nb_create(ctypes.byref(h), int(n_max), PRECISIONS[precision], device,
                                    _stream_ptr(stream))
        if st != 0:
            raise NBodyError("nb_create", st, self.lib.nb_last_error(None).decode())
        self.h = h.value
        self.n_max = int(n_max)

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _call(self, name, *args):
        _check(self.h, name, getattr(self.lib, name)(self.h, *args))

    # ------------------------------------------------------------------ API
    def set_stream(self, stream=None):
        self._call("nb_set_stream", _stream_ptr(stream))

    def sync(self):
        self._call("nb_sync")

    @property
    def launches(self) -> int:
        return int(self.lib.nb_launch_count(self.h))

    def forces(self, pos, mass, G, eps, out=None):
        import torch
        n = mass.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        self._call("nb_forces", n, _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n), float(G),
                   float(eps), _ptr(out, "acc", 3 * n))
        return out

    def step(self, pos, vel, mass, G, eps, dt, nsteps, acc, acc_valid=False, graph=False):
        n = mass.shape[0]
        flags = (NB_ACC_VALID if acc_valid else 0) | (NB_USE_GRAPH if graph else 0)
        self._call("nb_step", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), float(dt), int(nsteps),
                   _ptr(acc, "acc", 3 * n), flags)

    def rollout(self, pos, vel, mass, G, eps, dt, nsteps, acc, record_every, rec_pos,
                rec_vel=None, acc_valid=False, graph=False):
        n = mass.shape[0]
        flags = (NB_ACC_VALID if acc_valid else 0) | (NB_USE_GRAPH if graph else 0)
        nrec = int(nsteps) // int(record_every) + 1 if record_every > 0 else 0
        self._call("nb_rollout", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), float(dt), int(nsteps),
                   _ptr(acc, "acc", 3 * n), flags, int(record_every),
                   _ptr(rec_pos, "rec_pos", 3 * n * nrec),
                   _ptr(rec_vel, "rec_vel", 3 * n * nrec))

    def energy(self, pos, vel, mass, G, eps):
        """[E_kin, E_pot, E_tot, Px, Py, Pz, Fx, Fy, Fz] (synchronises)."""
        n = mass.shape[0]
        out = (ctypes.c_double * 9)()
        self._call("nb_energy", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), out)
        return list(out)

    def forces_backward(self, pos, mass, G, eps, grad_acc, grad_pos=None, grad_mass=None):
        import torch
        n = mass.shape[0]
        if grad_pos is None:
            grad_pos = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        if grad_mass is None:
            grad_mass = torch.empty((n,), dtype=torch.float64, device=pos.device)
        self._call("nb_forces_backward", n, _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n),
                   float(G), float(eps), _ptr(grad_acc, "grad_acc", 3 * n),
                   _ptr(grad_pos, "grad_pos", 3 * n), _ptr(grad_mass, "grad_mass", n))
        return grad_pos, grad_mass

    def step_backward(self, traj, mass, G, eps, dt, nsteps, lam_x, lam_v, lam_m,
                      at_start=False, at_end=False):
        n = mass.shape[0]
        flags = (NB_BWD_AT_START if at_start else 0) | (NB_BWD_AT_END if at_end else 0)
        self._call("nb_step_backward", n, _ptr(traj, "traj", 3 * n * (int(nsteps) + 1)),
                   _ptr(mass, "mass", n), float(G), float(eps), float(dt), int(nsteps),
                   _ptr(lam_x, "lam_x", 3 * n), _ptr(lam_v, "lam_v", 3 * n),
                   _ptr(lam_m, "lam_m", n), flags)

    def batch_plan(self, offsets):
        offs = [int(o) for o in offsets]
        arr = (ctypes.c_int64 * len(offs))(*offs)
        self._call("nb_batch_plan", len(offs) - 1, arr)
        self.batch_n = offs[-1]

    def forces_batched(self, pos, mass, G, eps, out=None):
        import torch
        n = self.batch_n
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        self._call("nb_forces_batched", _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n), float(G),
                   float(eps), _ptr(out, "acc", 3 * n))
        return out

    def step_batched(self, pos, vel, mass, G, eps, dt, nsteps, acc, acc_valid=False,
                     graph=False):
        n = self.batch_n
        flags = (NB_ACC_VALID if acc_valid else 0) | (NB_USE_GRAPH if graph else 0)
        self._call("nb_step_batched", _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), float(dt), int(nsteps),
                   _ptr(acc, "acc", 3 * n), flags)

    def tune_set(self, kind, lo, hi, variant, split=0):
        self._call("nb_tune_set", int(kind), int(lo), int(hi), int(variant), int(split))

    def tune_get(self, kind, n):
        v, s = ctypes.c_int(), ctypes.c_int()
        self._call("nb_tune_get", int(kind), int(n), ctypes.byref(v), ctypes.byref(s))
        return v.value, s.value

    def set_order(self, mode: int, min_n: int = 131072):
        """Float32 body order: 0 input order, 1 Morton, 2 Morton when n >= min_n."""
        self._call("nb_set_order", int(mode), int(min_n))

    def profile(self, enable: bool):
        """Start (clearing earlier records) or stop event timing of pair kernels."""
        self._call("nb_profile", 1 if enable else 0)

    def profile_read(self, kind: int):
        """(launches, total milliseconds) recorded for kind 0 force, 1 batched,
        2 VJP, 3 energy, 4 tree walk, 5 tree build, 6 fast multipole upward and
        downward passes, 7 fast multipole near field."""
        cnt, ms = ctypes.c_int64(), ctypes.c_double()
        self._call("nb_profile_read", int(kind), ctypes.byref(cnt), ctypes.byref(ms))
        return cnt.value, ms.value

    def tree_forces(self, pos, mass, G, eps, theta, leaf_cap=16, out=None, counts=False,
                    group=64):
        """Barnes-Hut accelerations (paper Sec. IV-A), bodies walking the tree
        `group` (32 or 64) at a time; with counts=True also the int32 [n, 2]
        cells and bodies each body met."""
        import torch
        n = mass.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        cnt = None
        if counts:
            cnt = torch.empty((n, 2), dtype=torch.int32, device=pos.device)
        self._call("nb_tree_forces", n, _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n), float(G),
                   float(eps), float(theta), int(leaf_cap), int(group), _ptr(out, "acc", 3 * n),
                   _ptr_i32(cnt, "counts", 2 * n))
        return (out, cnt) if counts else out

    def tree_step(self, pos, vel, mass, G, eps, theta, leaf_cap, dt, nsteps, acc,
                  acc_valid=False, graph=False, group=64):
        n = mass.shape[0]
        flags = (NB_ACC_VALID if acc_valid else 0) | (NB_USE_GRAPH if graph else 0)
        self._call("nb_tree_step", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), float(theta), int(leaf_cap),
                   int(group), float(dt), int(nsteps), _ptr(acc, "acc", 3 * n), flags)

    def tree_schedule(self, sched="dynamic", chunk=1):
        """Walk schedule: "static", "dynamic" or "guided" (or 0, 1, 2), chunk >= 1."""
        names = {"static": 0, "dynamic": 1, "guided": 2}
        self._call("nb_tree_schedule", names.get(sched, sched), int(chunk))

    def fmm_forces(self, pos, mass, G, eps, theta=0.6, order=6, leaf_cap=64, out=None,
                   counts=False):
        """Fast-multipole accelerations (order 2..6 Cartesian expansions over
        the tree, leaves of up to leaf_cap <= 64 bodies); with counts=True also
        the int32 [n, 3] source cells acting on each body's leaf and its
        ancestors, the bodies they hold, and the bodies met directly."""
        import torch
        n = mass.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        cnt = None
        if counts:
            cnt = torch.empty((n, 3), dtype=torch.int32, device=pos.device)
        self._call("nb_fmm_forces", n, _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n), float(G),
                   float(eps), float(theta), int(order), int(leaf_cap), _ptr(out, "acc", 3 * n),
                   _ptr_i32(cnt, "counts", 3 * n))
        return (out, cnt) if counts else out

    def fmm_step(self, pos, vel, mass, G, eps, theta, order, leaf_cap, dt, nsteps, acc,
                 acc_valid=False):
        """Kick-drift-kick steps with FMM forces (eager; the FMM synchronises)."""
        n = mass.shape[0]
        self._call("nb_fmm_step", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), float(G), float(eps), float(theta), int(order),
                   int(leaf_cap), float(dt), int(nsteps), _ptr(acc, "acc", 3 * n),
                   NB_ACC_VALID if acc_valid else 0)

    def fmm_reserve(self, entries):
        """Replace the FMM candidate pool by one of `entries` ints."""
        self._call("nb_fmm_reserve", int(entries))

    def fmm_stats(self):
        """{nodes, leaves, expansions, direct_pairs} of the last FMM call."""
        out = (ctypes.c_int64 * 4)()
        self._call("nb_fmm_stats", out)
        return dict(zip(("nodes", "leaves", "expansions", "direct_pairs"), out))

    def tree_stats(self):
        """{nodes, leaves, cell_interactions, body_interactions} of the last tree call."""
        out = (ctypes.c_int64 * 4)()
        self._call("nb_tree_stats", out)
        return dict(zip(("nodes", "leaves", "cell_interactions", "body_interactions"), out))

    # ------------------------------------- parallel tree code (ORB, LET)
    def orb_box(self, pos, group, ngroups):
        """Per group g < ngroups: [min xyz, max xyz] of this context's bodies
        of g (numpy float64 (ngroups, 6); +inf/-inf when none)."""
        import numpy as np
        import torch
        n = group.shape[0]
        out = np.zeros((ngroups, 6))
        self._call("nb_orb_box", n, _ptr(pos, "pos", 3 * n), _ptr_typed(group, "group", torch.int32, n),
                   int(ngroups), out.ctypes.data_as(ctypes.POINTER(_c_dbl)))
        return out

    def orb_hist(self, pos, ids, group, active, axis, prefix, rnd):
        """Digit histograms (numpy int64 (len(active), 256)) of round rnd."""
        import numpy as np
        import torch
        n = group.shape[0]
        na = len(active)
        out = np.zeros((max(na, 1), 256), dtype=np.int64)
        pre = (ctypes.c_uint64 * max(2 * na, 1))(*[int(v) for v in np.asarray(prefix, dtype=np.uint64).ravel()])
        self._call("nb_orb_hist", n, _ptr(pos, "pos", 3 * n), _ptr_typed(ids, "ids", torch.int64, n),
                   _ptr_typed(group, "group", torch.int32, n), na,
                   _host_array(ctypes.c_int32, active), _host_array(ctypes.c_int32, axis), pre,
                   int(rnd), out.ctypes.data_as(ctypes.POINTER(_c_i64)))
        return out[:na]

    def orb_cut(self, pos, ids, group, active, axis, split, upper):
        """Move the bodies of each active part at or above its split key to
        its upper group (in place on `group`)."""
        import numpy as np
        import torch
        n = group.shape[0]
        na = len(active)
        spl = (ctypes.c_uint64 * max(2 * na, 1))(*[int(v) for v in np.asarray(split, dtype=np.uint64).ravel()])
        self._call("nb_orb_cut", n, _ptr(pos, "pos", 3 * n), _ptr_typed(ids, "ids", torch.int64, n),
                   _ptr_typed(group, "group", torch.int32, n), na,
                   _host_array(ctypes.c_int32, active), _host_array(ctypes.c_int32, axis), spl,
                   _host_array(ctypes.c_int32, upper))

    def orb_pack(self, rank, P, pos, vel, mass, ids):
        """Bodies ordered by rank (stable) and the counts per rank."""
        import numpy as np
        import torch
        n = rank.shape[0]
        outs = [torch.empty_like(t) for t in (pos, vel, mass, ids)]
        counts = np.zeros(P, dtype=np.int64)
        self._call("nb_orb_pack", n, _ptr_typed(rank, "rank", torch.int32, n), int(P),
                   _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n), _ptr(mass, "mass", n),
                   _ptr_typed(ids, "ids", torch.int64, n), _ptr(outs[0], "pos_out", 3 * n),
                   _ptr(outs[1], "vel_out", 3 * n), _ptr(outs[2], "mass_out", n),
                   _ptr_typed(outs[3], "id_out", torch.int64, n),
                   counts.ctypes.data_as(ctypes.POINTER(_c_i64)))
        return (*outs, counts)

    def orb_order(self, pos, vel, mass, ids):
        """Bodies ordered by id."""
        import torch
        n = ids.shape[0]
        outs = [torch.empty_like(t) for t in (pos, vel, mass, ids)]
        self._call("nb_orb_order", n, _ptr(pos, "pos", 3 * n), _ptr(vel, "vel", 3 * n),
                   _ptr(mass, "mass", n), _ptr_typed(ids, "ids", torch.int64, n),
                   _ptr(outs[0], "pos_out", 3 * n), _ptr(outs[1], "vel_out", 3 * n),
                   _ptr(outs[2], "mass_out", n), _ptr_typed(outs[3], "id_out", torch.int64, n))
        return tuple(outs)

    def let_build(self, pos, mass, leaf_cap):
        """Build the local tree; returns the float32 box of the bodies (6,)."""
        import numpy as np
        n = mass.shape[0]
        box = np.zeros(6, dtype=np.float32)
        self._call("nb_let_build", n, _ptr(pos, "pos", 3 * n), _ptr(mass, "mass", n),
                   int(leaf_cap), box.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        self._let_n = n
        return box

    def let_export(self, theta, box):
        """The LET of the local tree for a destination box, as a uint8 CUDA tensor."""
        import numpy as np
        import torch
        b = np.ascontiguousarray(box, dtype=np.float32)
        size = _c_i64()
        bp = b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        self._call("nb_let_export", float(theta), bp, None, 0, ctypes.byref(size))
        out = torch.empty(size.value, dtype=torch.uint8, device=f"cuda:{self.device}")
        self._call("nb_let_export", float(theta), bp, out.data_ptr(), size.value, ctypes.byref(size))
        return out

    def let_forces(self, G, eps, theta, group, lets, out=None, counts=False):
        """Accelerations of the local bodies from the local tree and the
        received LETs (uint8 CUDA tensors, in the order to add them)."""
        import torch
        n = self._let_n
        dev = f"cuda:{self.device}"
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=dev)
        cnt = torch.empty((n, 2), dtype=torch.int32, device=dev) if counts else None
        arr = (_c_vp * max(len(lets), 1))(*[t.data_ptr() for t in lets])
        self._call("nb_let_forces", float(G), float(eps), float(theta), int(group), len(lets), arr,
                   _ptr(out, "acc", 3 * n), _ptr_i32(cnt, "counts", 2 * n) if counts else None)
        return (out, cnt) if counts else out

    def device_info(self, n):
        sms, occ = ctypes.c_int(), ctypes.c_int()
        self._call("nb_device_info", int(n), ctypes.byref(sms), ctypes.byref(occ))
        return sms.value, occ.value


def variants(kind: int, precision: str):
    """[(threads, bodies_per_thread, jtile)] of the compiled variants."""
    lib = load()
    p = PRECISIONS[precision]
    out = []
    for v in range(lib.nb_variant_count(kind, p)):
        t, i, j = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.nb_variant_info(kind, p, v, ctypes.byref(t), ctypes.byref(i), ctypes.byref(j))
        out.append((t.value, i.value, j.value))
    return out


def choose_split(n_itiles, n_jtiles, slots, max_split_bodies, tile_bodies) -> int:
    return int(load().nb_choose_split(n_itiles, n_jtiles, slots, max_split_bodies, tile_bodies))


BATCH_ITEM_INTS = 12


def plan_batch_host(offsets, threads, bodies_per_thread, jtile, max_item_pairs=0):
    """Work items the batched kernel would run, largest cost first:
    [(i0, i_end, j0, j1, lanes, sys, ctr, pbase, chunk, nchunks)]."""
    lib = load()
    offs = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    nsys = len(offsets) - 1
    cnt = lib.nb_plan_batch_host(nsys, offs, threads, bodies_per_thread, jtile,
                                 int(max_item_pairs), None, 0)
    if cnt < 0:
        raise ValueError("invalid offsets")
    w = BATCH_ITEM_INTS
    buf = (ctypes.c_int32 * (w * max(cnt, 1)))()
    lib.nb_plan_batch_host(nsys, offs, threads, bodies_per_thread, jtile, int(max_item_pairs),
                           buf, cnt)
    return [tuple(buf[w * q: w * q + 10]) for q in range(cnt)]
