"""Autotuner for the pair kernels: CTA shape, bodies per thread, j-tile and
j-split count, per precision and size bucket.

Each candidate (variant, split) is timed through the library itself: the
variant is forced with ``nb_tune_set`` and its launches are timed with the
library's CUDA events (``nb_profile``) on synthetic Plummer inputs.  The best
candidate per size becomes an entry {kind, precision, lo, hi, variant,
split}; buckets meet at the geometric midpoints between tuned sizes.  The
table is saved as JSON and applied to a context with :func:`apply`.

  python -m paper_1211_2292_gb300.tune --out tuning.json [--sizes 4096,65536,...]
"""
from __future__ import annotations

import argparse
import json
import math
import os

from . import inputs, nbody

DEFAULT_SIZES = {
    nbody.KIND_FORCE: [1024, 4096, 16384, 65536, 262144, 1048576],
    nbody.KIND_VJP: [1024, 4096, 16384, 65536],
}
# item caps tried for the batched kernel (1/d of an even per-CTA share of the pairs)
BATCH_DIVISORS = (1, 2, 4, 8)
DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def _time_call(nb, fn, kind, reps):
    fn()  # warm-up (and first-use setup)
    nb.profile(True)
    for _ in range(reps):
        fn()
    cnt, ms = nb.profile_read(kind)
    nb.profile(False)
    return ms / max(cnt, 1)


def time_candidates(kind, precision, n, splits=(0,), reps=3, seed=0, device=0, log=None):
    """[(ms per launch, variant, split)] for every compiled variant at size n."""
    import torch
    dev = torch.device("cuda", device)
    b = inputs.plummer(n, seed=seed)
    x = torch.as_tensor(b.pos, device=dev).contiguous()
    m = torch.as_tensor(b.mass, device=dev).contiguous()
    out = []
    with nbody.NBody(n, precision, device=device) as nb:
        if kind == nbody.KIND_FORCE:
            acc = torch.empty_like(x)
            fn = lambda: nb.forces(x, m, 1.0, 0.01, out=acc)  # noqa: E731
        elif kind == nbody.KIND_VJP:
            lam = torch.ones_like(x)
            gx, gm = torch.empty_like(x), torch.empty_like(m)
            fn = lambda: nb.forces_backward(x, m, 1.0, 0.01, lam, gx, gm)  # noqa: E731
        else:
            raise ValueError("kind must be KIND_FORCE or KIND_VJP (use tune_batched)")
        for v in range(len(nbody.variants(kind, precision))):
            for s in splits:
                nb.tune_set(kind, 0, 1 << 40, v, s)
                ms = _time_call(nb, fn, kind, reps)
                out.append((ms, v, s))
                if log:
                    log(f"kind={kind} {precision} n={n} variant={v}"
                        f"{nbody.variants(kind, precision)[v]} split={s}: {ms:.4f} ms")
                nb.tune_set(kind, 0, 1, -1, 0)
    return sorted(out)


def time_batched(precision, offsets, bodies, reps=3, device=0, log=None, divisors=(0,)):
    """[(ms per launch, variant, divisor)] of the batched kernel on one set of
    systems; the divisor (a tuning entry's split field, 0 = the default 4)
    caps a work item at 1/divisor of an even per-CTA share of the pairs."""
    import torch
    dev = torch.device("cuda", device)
    x = torch.as_tensor(bodies.pos, device=dev).contiguous()
    m = torch.as_tensor(bodies.mass, device=dev).contiguous()
    out = []
    with nbody.NBody(max(bodies.n, 1), precision, device=device) as nb:
        acc = torch.empty_like(x)
        for v in range(len(nbody.variants(nbody.KIND_BATCHED, precision))):
            for d in divisors:
                nb.tune_set(nbody.KIND_BATCHED, 0, 1 << 40, v, d)
                nb.batch_plan(offsets)
                ms = _time_call(nb, lambda: nb.forces_batched(x, m, 1.0, 0.01, out=acc),
                                nbody.KIND_BATCHED, reps)
                out.append((ms, v, d))
                if log:
                    log(f"batched {precision} variant={v}"
                        f"{nbody.variants(nbody.KIND_BATCHED, precision)[v]} divisor={d}:"
                        f" {ms:.4f} ms")
                nb.tune_set(nbody.KIND_BATCHED, 0, 1, -1, 0)
    return sorted(out)


def _buckets(sizes):
    sizes = sorted(sizes)
    edges = [0]
    for a, b in zip(sizes, sizes[1:]):
        edges.append(int(math.sqrt(a * b)))
    edges.append(1 << 40)
    return list(zip(sizes, edges[:-1], edges[1:]))


def autotune(precisions=("fp32_comp", "fp32", "fp64", "df64"),
             kinds=(nbody.KIND_FORCE, nbody.KIND_VJP), sizes=None, splits=(0,), reps=3,
             batch=True, device=0, log=print):
    """Time every variant (and each split in `splits`) at the tuned sizes of
    each precision and kind; the fastest per size becomes a table entry whose
    bucket reaches to the geometric midpoints between tuned sizes.  The
    float64-state modes (fp64, df64) are tuned up to 2^18 bodies, their last
    bucket covering every larger size."""
    import torch
    table = {"device": torch.cuda.get_device_name(device), "entries": []}
    for prec in precisions:
        for kind in kinds:
            szs = (sizes or {}).get(kind, DEFAULT_SIZES[kind])
            if prec in ("fp64", "df64"):  # ~10-100x slower than float32: up to 2^18 bodies
                szs = [z for z in szs if z <= 262144] or szs[:1]
            for n, lo, hi in _buckets(szs):
                res = time_candidates(kind, prec, n, splits, reps, device=device, log=log)
                ms, v, s = res[0]
                table["entries"].append({"kind": kind, "precision": prec, "lo": lo, "hi": hi,
                                         "n": n, "variant": v, "split": s, "ms": ms})
        if batch and prec not in ("fp64", "df64"):  # the batched kernel is float32 only
            bodies, off = inputs.plummer_batch(512, 64, 8192, seed=3)
            res = time_batched(prec, off, bodies, reps, device=device, log=log,
                               divisors=BATCH_DIVISORS)
            ms, v, d = res[0]
            table["entries"].append({"kind": nbody.KIND_BATCHED, "precision": prec, "lo": 0,
                                     "hi": 1 << 40, "n": bodies.n, "variant": v, "split": d,
                                     "ms": ms})
    return table


def load(path=DEFAULT_TABLE):
    with open(path) as f:
        return json.load(f)


def apply(nb: nbody.NBody, table=None) -> int:
    """Install the table's entries for nb's precision; returns how many."""
    if table is None:
        if not os.path.exists(DEFAULT_TABLE):
            return 0
        table = load(DEFAULT_TABLE)
    elif isinstance(table, str):
        table = load(table)
    k = 0
    for e in table.get("entries", []):
        if e["precision"] != nb.precision:
            continue
        if e["variant"] >= len(nbody.variants(e["kind"], nb.precision)):
            continue
        nb.tune_set(e["kind"], e["lo"], e["hi"], e["variant"], e["split"])
        k += 1
    return k


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--precisions", default="fp32_comp,fp32,fp64,df64")
    ap.add_argument("--sizes", default="", help="force sizes, comma separated")
    ap.add_argument("--splits", default="0")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kinds", default="force,vjp,batched",
                    help="which kernel families to tune")
    ap.add_argument("--merge", default="",
                    help="existing table whose entries for other precisions are kept")
    a = ap.parse_args()
    sizes = None
    if a.sizes:
        sizes = {nbody.KIND_FORCE: [int(x) for x in a.sizes.split(",")],
                 nbody.KIND_VJP: DEFAULT_SIZES[nbody.KIND_VJP]}
    precs = tuple(a.precisions.split(","))
    names = {"force": nbody.KIND_FORCE, "vjp": nbody.KIND_VJP, "batched": nbody.KIND_BATCHED}
    kinds = [names[k] for k in a.kinds.split(",") if k]
    t = autotune(precs, kinds=tuple(k for k in kinds if k != nbody.KIND_BATCHED), sizes=sizes,
                 splits=tuple(int(s) for s in a.splits.split(",")), reps=a.reps,
                 batch=nbody.KIND_BATCHED in kinds)
    if a.merge and os.path.exists(a.merge):
        old = load(a.merge)
        t["entries"] = [e for e in old.get("entries", [])
                        if not (e["precision"] in precs and e["kind"] in kinds)] + t["entries"]
    with open(a.out, "w") as f:
        json.dump(t, f, indent=1)
    print(f"wrote {len(t['entries'])} entries to {a.out}")


if __name__ == "__main__":
    main()
