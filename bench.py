#!/usr/bin/env python
"""Throughput benchmark of the softened direct-sum n-body path on GB300.

Default workload ("throughput"): two Plummer spheres of 524,288 bodies each
(N = 1,048,576), centres at (+-5, 0, 0) approaching at relative velocity
0.5, lognormal (sigma 0.5) masses normalised to 1, eps = 0.002, seed 2.  One
bench step is one force evaluation plus 10 kick-drift-kick steps (11 force
evaluations) in the float32 Kahan-compensated form with float64 state.
Metric: pairwise interactions per second, N^2 per force evaluation.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload throughput|batched|precision|plain|differentiation|tree|fmm|let]

The other workloads (single-GPU lines with the same metric): "precision"
(N = 65,536 Plummer, eps 0.005, FP32 compensated, 1 + 100 steps of dt 5e-4,
with the force error against the oracle and the energy drift against the
FP64 GPU run), "plain" (N = 1024 Plummer, FP64, 1 + 10 steps of dt 1e-3, one
graph launch, checked against the oracle), "differentiation" (N = 16,384,
200 steps with checkpoints every 20: forward, recompute and reverse sweep),
"tree" (the default workload's bodies through the Barnes-Hut tree code,
theta 0.5, leaves of at most 16 bodies: 1 + 10 KDK steps with the tree
rebuilt for every force evaluation; its metric counts the cell and body
interactions the walk computes), "let" (the same bodies through the parallel
tree code: ORB domains and locally essential trees over P processes, one per
GPU under torchrun, or emulated by threads on one GPU).

Multi-GPU (torchrun, one rank per GPU): for "throughput" every rank runs its
own replica (the single-system path is not sharded); for "batched" the 512
independent systems are dealt to ranks largest first, with no collective on
the data path.  value = interactions of all ranks / slowest rank's time.

The JSON line also carries the float32 force error against the FP64 oracle on
4096 sampled bodies, the force kernel's roofline (event-timed inside the timed
region), the same workload in the FP64 form (one force evaluation of all
bodies) and in the double-float form (1 + 10 steps), each with its force
error on the same sampled bodies; the batched, adjoint and precision forms
beside the plain FP64 GPU form of the same work and their errors against it
or the oracle; the tree and FMM forms; the oracle's CPU rate, an end-to-end
rate with host buffers, the SM clocks sampled during the timed region and the
number of library kernels launched.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_INTERACTION = 20          # the usual convention for one softened pair
FP32_LANES_PER_SM = 128             # Blackwell SM: 4 partitions x 32 FP32 lanes
NOMINAL_SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2

WORKLOAD = {
    "name": "two-plummer N=1048576, 1 force eval + 10 KDK steps, fp32 Kahan-compensated",
    "n_per": 524_288, "seed": 2, "G": 1.0, "eps": 0.002, "dt": 1e-3, "steps": 10,
}
BATCHED = {
    "name": "512 Plummer systems, N log-uniform in [64, 8192], 100 KDK steps per graph launch, "
            "fp32 Kahan-compensated",
    "nsys": 512, "lo": 64, "hi": 8192, "seed": 3, "G": 1.0, "eps": 0.01, "dt": 1e-3, "steps": 100,
}
ADJOINT = {"n": 16384, "seed": 4, "eps": 0.01, "dt": 1e-3, "steps": 200, "every": 20}
METRIC = "pairwise interactions/s (G/s)"
UNIT = "Ginteractions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="throughput",
                    choices=["throughput", "batched", "precision", "plain", "differentiation",
                             "tree", "fmm", "let"])
    ap.add_argument("--procs", type=int, default=8,
                    help="let workload on one GPU: processes emulated by threads")
    ap.add_argument("--theta", type=float, default=None, help="tree workload: opening angle")
    ap.add_argument("--leaf-cap", type=int, default=None, help="tree workload: leaf capacity")
    ap.add_argument("--order", type=int, default=None, help="fmm workload: expansion order 2..6")
    ap.add_argument("--group", type=int, default=None, choices=[32, 64],
                    help="tree workload: bodies walking the tree together")
    ap.add_argument("--tree-sched", default="dynamic", choices=["static", "dynamic", "guided"],
                    help="tree workload: walk schedule of the timed steps")
    ap.add_argument("--tree-chunk", type=int, default=1, help="tree workload: schedule chunk")
    ap.add_argument("--fp64-n", type=int, default=None,
                    help="bodies for the float64 and double-float forms (default: the whole "
                         "workload; a smaller value takes the first bodies, for profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched/adjoint form measurements")
    ap.add_argument("--n-per", type=int, default=WORKLOAD["n_per"],
                    help="bodies per sphere (smaller cases for profiling)")
    ap.add_argument("--force-variant", type=int, default=-1,
                    help="run the force kernel variant with this index (profiling)")
    ap.add_argument("--tuning", default="default",
                    help="kernel tuning table (JSON from paper_1211_2292_gb300.tune), "
                         "'default' for the packaged GB300 table, 'none' for built-in defaults")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region.  A reader
    thread collects the samples; wait_ready() returns once the first one has
    arrived, so that nvidia-smi's start-up (NVML initialisation) is over
    before the timed region begins."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        import threading
        self.proc = None
        self.lines = []
        self.ready = threading.Event()
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd[1:1] = ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            self.ready.set()
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)
            self.ready.set()
        self.ready.set()

    def wait_ready(self, timeout=10.0):
        self.ready.wait(timeout)
        self.skip = len(self.lines)  # samples taken before the timed region

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[getattr(self, "skip", 0):] or self.lines[-1:]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def traffic_from_profile(profile="force_f32comp_two_plummer_n1048576.md", source="force_f32.cuh"):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel's source file changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", profile)
    src = os.path.join(ROOT, "paper_1211_2292_gb300", "csrc", source)
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].rsplit(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get(f"{source} sha256[:16]") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def oracle_rate(pos, mass, G, eps, target_s, seed=8):
    """Oracle interactions/s on host cores over a bounded sample of force rows."""
    import oracle
    from paper_1211_2292_gb300 import inputs
    n = mass.shape[0]
    probe = inputs.sample_rows(n, 64, seed=7)
    t0 = time.perf_counter()
    oracle.accel_rows(pos, mass, probe, G, eps)
    rate = probe.size * n / max(time.perf_counter() - t0, 1e-6)
    rows = int(min(n, max(256, rate * target_s / n)))
    idx = inputs.sample_rows(n, rows, seed=seed)
    t0 = time.perf_counter()
    oracle.accel_rows(pos, mass, idx, G, eps)
    el = time.perf_counter() - t0
    return idx.size * n / el, el, rows


def reference_arm(args, ws, rank):
    """The FP64 CPU oracle timed on the host cores, same metric and workload;
    each step is a bounded sample of force rows of that workload."""
    if rank != 0:
        return 0
    import oracle
    from paper_1211_2292_gb300 import inputs
    if args.workload == "let":
        w = LET_W
        b = inputs.two_plummer(TREE["cpu_n_per"], seed=w["seed"])
        P = args.procs
        rank_of = oracle.orb(b.pos, P)
        for _ in range(args.warmup):
            oracle.bh_sharded(b.pos, b.mass, 1.0, w["eps"], w["theta"], w["leaf_cap"],
                              w["group"], rank_of, P)
        tot, inter = 0.0, 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, st, _ = oracle.bh_sharded(b.pos, b.mass, 1.0, w["eps"], w["theta"],
                                         w["leaf_cap"], w["group"], rank_of, P)
            tot += time.perf_counter() - t0
            inter += st["cell_interactions"] + st["body_interactions"]
        value = inter / tot / 1e9
        sample = (f"the oracle's parallel tree code on two-plummer N={b.n} (same recipe) over "
                  f"{P} ORB domains, theta {w['theta']}, leaves <= {w['leaf_cap']}, groups of "
                  f"{w['group']}, per step")
        line = {
            "impl": "reference", "metric": TREE_METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": w["name"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "tree":
        w = TREE
        theta = w["theta"] if args.theta is None else args.theta
        lc = w["leaf_cap"] if args.leaf_cap is None else args.leaf_cap
        grp = w["group"] if args.group is None else args.group
        b = inputs.two_plummer(w["cpu_n_per"], seed=w["seed"])
        for _ in range(args.warmup):
            oracle.bh_forces(b.pos, b.mass, 1.0, w["eps"], theta, lc, grp)
        tot, inter = 0.0, 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, st = oracle.bh_forces(b.pos, b.mass, 1.0, w["eps"], theta, lc, grp)
            tot += time.perf_counter() - t0
            inter += st["cell_interactions"] + st["body_interactions"]
        value = inter / tot / 1e9
        sample = (f"one tree build + walk of two-plummer N={b.n} (same recipe), theta {theta}, "
                  f"leaves <= {lc}, groups of {grp}, per step")
        line = {
            "impl": "reference", "metric": TREE_METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": w["name"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "fmm":
        w = FMM
        theta = w["theta"] if args.theta is None else args.theta
        lc = w["leaf_cap"] if args.leaf_cap is None else args.leaf_cap
        order = w["order"] if args.order is None else args.order
        b = inputs.two_plummer(w["cpu_n_per"], seed=w["seed"])
        for _ in range(args.warmup):
            oracle.fmm_forces(b.pos, b.mass, 1.0, w["eps"], theta, order, lc)
        tot = 0.0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            oracle.fmm_forces(b.pos, b.mass, 1.0, w["eps"], theta, order, lc)
            tot += time.perf_counter() - t0
        value = float(b.n) * args.steps / tot / 1e9
        sample = (f"one fast-multipole evaluation of two-plummer N={b.n} (same recipe), theta "
                  f"{theta}, order {order}, leaves <= {lc}, per step")
        line = {
            "impl": "reference", "metric": FMM_METRIC, "value": value, "unit": FMM_UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": w["name"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": FMM_UNIT, "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": FMM_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "batched":
        w = BATCHED
        bodies, off = inputs.plummer_batch(w["nsys"], w["lo"], w["hi"], seed=w["seed"])
        k = int(max(range(len(off) - 1), key=lambda q: off[q + 1] - off[q]))
        pos, mass = bodies.pos[off[k]:off[k + 1]], bodies.mass[off[k]:off[k + 1]]
        name, sample_of = w["name"], f"system {k} (N={off[k + 1] - off[k]})"
    elif args.workload in ("precision", "plain", "differentiation"):
        w = {"precision": PRECISION, "plain": PLAIN,
             "differentiation": dict(ADJOINT, name="differentiation, N=16384")}[args.workload]
        w = dict(w, G=1.0)
        b = (inputs.plummer_with_perturbation(w["n"], seed=w["seed"])[0]
             if args.workload == "differentiation" else inputs.plummer(w["n"], seed=w["seed"]))
        pos, mass = b.pos, b.mass
        name, sample_of = w["name"], f"N={b.n}"
    else:
        w = WORKLOAD
        b = inputs.two_plummer(w["n_per"], seed=w["seed"])
        pos, mass = b.pos, b.mass
        name, sample_of = w["name"], f"N={b.n}"
    n = mass.shape[0]
    probe = inputs.sample_rows(n, min(64, n), seed=7)
    t0 = time.perf_counter()
    oracle.accel_rows(pos, mass, probe, w["G"], w["eps"])
    rate = probe.size * n / max(time.perf_counter() - t0, 1e-6)
    rows = int(min(n, max(128, rate * 6.0 / n)))
    idx = inputs.sample_rows(n, rows, seed=9)
    for _ in range(args.warmup):
        oracle.accel_rows(pos, mass, idx, w["G"], w["eps"])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.accel_rows(pos, mass, idx, w["G"], w["eps"])
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = rows * n * args.steps / tot / 1e9
    sample = f"{rows} force rows x {n} bodies of {sample_of} per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Plummer spheres)",
        "config": {"workload": name, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class Timer:
    """CUDA-event timing on one stream, bracketed by barrier + synchronize."""

    def __init__(self, torch, dev, stream, barrier):
        self.torch, self.dev, self.stream, self.barrier = torch, dev, stream, barrier

    def __enter__(self):
        self.barrier()
        self.torch.cuda.synchronize(self.dev)
        self.e0 = self.torch.cuda.Event(enable_timing=True)
        self.e1 = self.torch.cuda.Event(enable_timing=True)
        self.e0.record(self.stream)
        return self

    def __exit__(self, *exc):
        self.e1.record(self.stream)
        self.torch.cuda.synchronize(self.dev)
        self.barrier()
        self.ms = self.e0.elapsed_time(self.e1)


def measure_forms(torch, dev, tune, table, peak_tflops, tree_bodies=None, tuning="default"):
    """Rates of the batched, adjoint, precision and tree forms (rank-local,
    after the timed region), the first three beside the plain FP64 GPU form
    of the same work at its accuracy."""
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody
    from paper_1211_2292_gb300.autograd import rollout
    stream = torch.cuda.current_stream(dev)
    out = {}
    w = BATCHED
    bodies, off = inputs.plummer_batch(w["nsys"], w["lo"], w["hi"], seed=w["seed"])
    sizes = np.diff(off)
    pairs = float(sum(int(z) ** 2 for z in sizes))
    with nbody.NBody(bodies.n, "fp32_comp", device=dev.index) as nb:
        tune.apply(nb, table)
        nb.batch_plan(off)
        x, v, m = (torch.as_tensor(a, device=dev).contiguous()
                   for a in (bodies.pos, bodies.vel, bodies.mass))
        a = nb.forces_batched(x, m, w["G"], w["eps"])
        ab = a.cpu().numpy()
        nb.step_batched(x, v, m, w["G"], w["eps"], w["dt"], w["steps"], a, acc_valid=True,
                        graph=True)
        with Timer(torch, dev, stream, lambda: None) as t:
            nb.step_batched(x, v, m, w["G"], w["eps"], w["dt"], w["steps"], a, acc_valid=True,
                            graph=True)
        nb.profile(True)
        nb.forces_batched(x, m, w["G"], w["eps"], out=a)
        kn, kms = nb.profile_read(1)
        nb.profile(False)
    # the plain FP64 GPU form of the same evaluation: one NB_FP64 call per
    # system, in order, on the initial state
    x, m = (torch.as_tensor(a_, device=dev).contiguous() for a_ in (bodies.pos, bodies.mass))
    with nbody.NBody(int(sizes.max()), "fp64", device=dev.index) as nb64:
        tune.apply(nb64, table)
        a64 = torch.empty_like(x)

        def fp64_batch():
            for k in range(len(sizes)):
                s_, e_ = int(off[k]), int(off[k + 1])
                nb64.forces(x[s_:e_], m[s_:e_], w["G"], w["eps"], out=a64[s_:e_])

        fp64_batch()
        nb64.profile(True)
        with Timer(torch, dev, stream, lambda: None) as t64:
            fp64_batch()
        k64, ms64 = nb64.profile_read(0)
        nb64.profile(False)
        nb64.sync()
    a64 = a64.cpu().numpy()
    # accuracy on sampled systems (the largest and 15 seeded others) vs the oracle
    rng = np.random.default_rng(6)
    sel = sorted(set(rng.choice(len(sizes), 15, replace=False).tolist()) |
                 {int(np.argmax(sizes))})
    e32, e64 = [], []
    for k in sel:
        s_, e_ = int(off[k]), int(off[k + 1])
        ref = oracle.accel(bodies.pos[s_:e_], bodies.mass[s_:e_], w["G"], w["eps"])
        e32.append(_relerr(ab[s_:e_], ref))
        e64.append(_relerr(a64[s_:e_], ref))
    e32, e64 = np.concatenate(e32), np.concatenate(e64)
    kernel_ms = kms / max(kn, 1)
    batched_rate = pairs / (kernel_ms / 1e3) / 1e9
    fp64_rate = pairs / (t64.ms / 1e3) / 1e9
    sample = (f"{len(sel)} systems ({e32.size} bodies: the largest and 15 seeded others), "
              "per-body relative error vs the FP64 oracle")
    out["batched"] = {"value": pairs * w["steps"] / (t.ms / 1e3) / 1e9, "unit": UNIT,
                      "systems": w["nsys"], "bodies": bodies.n, "pairs_per_eval": pairs,
                      "ms_per_100_steps_graph": t.ms, "kernel_ms": kernel_ms,
                      "kernel_value": batched_rate,
                      "kernel_frac_of_fp32_peak": FLOPS_PER_INTERACTION * pairs
                      / (kernel_ms / 1e3) / 1e12 / peak_tflops,
                      "force_error": {"rms": float(np.sqrt((e32 ** 2).mean())),
                                      "max": float(e32.max()), "sample": sample},
                      "fp64_form": {"value": fp64_rate, "unit": UNIT, "ms_per_eval": t64.ms,
                                    "kernel_ms_sum": ms64, "launches": k64,
                                    "force_error": {"rms": float(np.sqrt((e64 ** 2).mean())),
                                                    "max": float(e64.max())},
                                    "note": "one NB_FP64 force call per system, in order "
                                            "(pack + kernel each), on the same stream"},
                      "kernel_over_fp64": batched_rate / fp64_rate}
    # adjoint: the 200-step gradient in the float32 form, and in the FP64 and
    # double-float contexts (float64 adjoint), with the gradients' differences
    a_ = ADJOINT
    b, dx = inputs.plummer_with_perturbation(a_["n"], seed=a_["seed"])
    x = torch.as_tensor(b.pos, device=dev).contiguous()
    v = torch.as_tensor(b.vel, device=dev).contiguous()
    m = torch.as_tensor(b.mass, device=dev).contiguous()
    tgt = x + torch.as_tensor(dx, device=dev)
    lam = torch.ones_like(x)
    grads, gms = {}, {}
    for prec in ("fp32_comp", "fp64", "df64"):
        with nbody.NBody(b.n, prec, device=dev.index) as nb:
            if tuning != "none":
                tune.apply(nb, table)
            nb.forces_backward(x, m, 1.0, a_["eps"], lam)
            if prec == "fp32_comp":
                nb.profile(True)
                for _ in range(5):
                    nb.forces_backward(x, m, 1.0, a_["eps"], lam)
                vn, vms = nb.profile_read(2)
                nb.profile(False)

            def grad():
                x0 = x.clone().requires_grad_()
                v0 = v.clone().requires_grad_()
                mm = m.clone().requires_grad_()
                xT, _ = rollout(nb, x0, v0, mm, 1.0, a_["eps"], a_["dt"], a_["steps"],
                                a_["every"])
                ((xT - tgt) ** 2).sum(-1).mean().backward()
                return [g.detach().cpu().numpy() for g in (x0.grad, v0.grad, mm.grad)]

            if prec == "fp32_comp":
                grad()
            else:
                nb.forces(x, m, 1.0, a_["eps"])
            with Timer(torch, dev, stream, lambda: None) as t:
                grads[prec] = grad()
            gms[prec] = t.ms
            nb.sync()

    def gerr(p):
        return {name: float(np.linalg.norm(g - r) / np.linalg.norm(r))
                for name, g, r in zip(("x0", "v0", "m"), grads[p], grads["fp64"])}

    n = float(b.n)
    out["adjoint"] = {"vjp_value": n * n / (vms / vn / 1e3) / 1e9, "unit": UNIT,
                      "vjp_ms": vms / vn, "n": b.n,
                      "gradient_ms": gms["fp32_comp"], "gradient_ms_fp64": gms["fp64"],
                      "gradient_ms_df64": gms["df64"],
                      "fp32_speedup_over_fp64": gms["fp64"] / gms["fp32_comp"],
                      "gradient_rel_err_vs_fp64": {"fp32_comp": gerr("fp32_comp"),
                                                   "df64": gerr("df64")},
                      "gradient": f"{a_['steps']} steps, checkpoints every {a_['every']}, "
                                  "forward + recompute + reverse sweep; relative errors are "
                                  "||g - g_fp64|| / ||g_fp64|| per input"}
    out["precision"] = precision_form(torch, dev, tune, table, tuning)
    if tree_bodies is not None:  # Barnes-Hut on the same bodies (full line: --workload tree)
        t_ = TREE
        x = torch.as_tensor(tree_bodies.pos, device=dev).contiguous()
        m = torch.as_tensor(tree_bodies.mass, device=dev).contiguous()
        with nbody.NBody(tree_bodies.n, "fp32_comp", device=dev.index) as nb:
            a = nb.tree_forces(x, m, 1.0, t_["eps"], t_["theta"], t_["leaf_cap"],
                               group=t_["group"])
            nb.profile(True)
            for _ in range(5):
                nb.tree_forces(x, m, 1.0, t_["eps"], t_["theta"], t_["leaf_cap"], out=a,
                               group=t_["group"])
            wn, wms = nb.profile_read(4)
            bn, bms = nb.profile_read(5)
            nb.profile(False)
            st = nb.tree_stats()
        inter = st["cell_interactions"] + st["body_interactions"]
        walk, build = wms / max(wn, 1), bms / max(bn, 1)
        n = float(tree_bodies.n)
        out["tree"] = {"theta": t_["theta"], "leaf_cap": t_["leaf_cap"], "group": t_["group"],
                       "ms_per_eval": walk + build, "walk_ms": walk, "build_ms": build,
                       "interactions": inter, "walk_value": inter / (walk / 1e3) / 1e9,
                       "unit": UNIT,
                       "walk_frac_of_fp32_peak": FLOPS_PER_INTERACTION * inter
                       / (walk / 1e3) / 1e12 / peak_tflops,
                       "direct_sum_equivalent": n * n / ((walk + build) / 1e3) / 1e9,
                       "note": "one tree build + walk of the throughput workload's bodies; "
                               "error and parity in bench.py --workload tree"}
        f_ = FMM
        with nbody.NBody(tree_bodies.n, "fp32_comp", device=dev.index) as nb:
            a = nb.fmm_forces(x, m, 1.0, f_["eps"], f_["theta"], f_["order"], f_["leaf_cap"])
            nb.profile(True)
            for _ in range(5):
                nb.fmm_forces(x, m, 1.0, f_["eps"], f_["theta"], f_["order"], f_["leaf_cap"],
                              out=a)
            bn, bms = nb.profile_read(5)
            fn, fms = nb.profile_read(6)
            qn, qms = nb.profile_read(7)
            nb.profile(False)
            st = nb.fmm_stats()
        build, far, near = bms / max(bn, 1), fms / max(fn, 1), qms / max(qn, 1)
        out["fmm"] = {"theta": f_["theta"], "order": f_["order"], "leaf_cap": f_["leaf_cap"],
                      "ms_per_eval": build + far + near, "build_ms": build, "far_ms": far,
                      "near_ms": near, "expansions": st["expansions"],
                      "direct_pairs": st["direct_pairs"],
                      "far_frac_of_fp32_peak": st["expansions"] * m2l_flops(f_["order"])
                      / (far / 1e3) / 1e12 / peak_tflops,
                      "near_frac_of_fp32_peak": FLOPS_PER_INTERACTION * st["direct_pairs"]
                      / (near / 1e3) / 1e12 / peak_tflops,
                      "bodies_per_s": n / ((build + far + near) / 1e3) / 1e9, "unit": FMM_UNIT,
                      "note": "one tree build + fast multipole evaluation of the throughput "
                              "workload's bodies; far: flops of the expansions' contractions "
                              f"({m2l_flops(f_['order'])} each), near: 20 per pair; error and "
                              "parity in bench.py --workload fmm"}
    return out


PRECISION = {"name": "Plummer N=65536, eps 0.005, fp32 Kahan-compensated, 1 force eval + 100 KDK "
                     "steps of dt 5e-4", "n": 65536, "seed": 1, "eps": 0.005, "dt": 5e-4,
             "steps": 100}
TREE = {"name": "two-plummer N=1048576, Barnes-Hut theta 0.5, leaves <= 16 bodies, groups of 64, "
                "1 force eval + 10 KDK steps (tree rebuilt per eval), fp32 walk, f64 state",
        "seed": 2, "eps": 0.002, "dt": 1e-3, "steps": 10, "theta": 0.5, "leaf_cap": 16,
        "group": 64, "cpu_n_per": 65_536}
TREE_METRIC = "tree interactions/s (cell + body, G/s)"
FMM = {"name": "two-plummer N=1048576, fast multipole theta 0.6, order 6, leaves <= 64 bodies, "
               "one force evaluation per step (tree rebuilt), fp32 expansions and pair terms, "
               "f64 output",
       "seed": 2, "eps": 0.002, "theta": 0.6, "order": 6, "leaf_cap": 64, "cpu_n_per": 65_536}
FMM_METRIC = "FMM force evaluations: bodies/s (N per evaluation / time, G/s; an O(N) method)"
FMM_UNIT = "Gbodies/s"


def m2l_flops(order):
    """Multiply-adds of one cell-to-cell expansion's contraction, x 2: the
    sum over |n| + |k| <= p of moment x derivative (C(p+6, 6) terms)."""
    from math import comb
    return 2 * comb(order + 6, 6)
PLAIN = {"name": "Plummer N=1024, eps 0.01, fp64, 1 force eval + 10 KDK steps of dt 1e-3 "
                 "(one graph launch)", "n": 1024, "seed": 0, "eps": 0.01, "dt": 1e-3, "steps": 10}


def _line(args, ws, value, ms_step, cfg, extra, dtype="f32", scaling="weak"):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": scaling, "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded Plummer spheres)", "config": cfg}
    line.update(extra)
    print(json.dumps(line), flush=True)


def tree_oracle_rate(w, theta, leaf_cap, group):
    """The oracle's (single-threaded) tree code on the same recipe at 2 x cpu_n_per bodies."""
    import oracle
    from paper_1211_2292_gb300 import inputs
    b = inputs.two_plummer(w["cpu_n_per"], seed=w["seed"])
    t0 = time.perf_counter()
    _, st, cnt = oracle.bh_forces(b.pos, b.mass, 1.0, w["eps"], theta, leaf_cap, group,
                                   counts=True)
    el = time.perf_counter() - t0
    inter = st["cell_interactions"] + st["body_interactions"]
    sample = (f"two-plummer N={b.n} (same recipe), theta {theta}, leaves <= {leaf_cap}, groups "
              f"of {group}: one tree build + walk, {el:.1f} s")
    return inter / el / 1e9, sample, b, cnt


def tree_workload(args, ws, torch, dev, stream, T, flush, table):
    """Barnes-Hut line: value = walk interactions / time over 1 + 10 steps."""
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody
    w = TREE
    theta = w["theta"] if args.theta is None else args.theta
    lc = w["leaf_cap"] if args.leaf_cap is None else args.leaf_cap
    grp = w["group"] if args.group is None else args.group
    b = inputs.two_plummer(args.n_per, seed=w["seed"])
    x0, v0, m = T(b.pos), T(b.vel), T(b.mass)
    G, eps, dt, K = 1.0, w["eps"], w["dt"], w["steps"]
    with nbody.NBody(b.n, "fp32_comp", device=dev.index) as nb:
        nb.tree_schedule(args.tree_sched, args.tree_chunk)
        x, v = x0.clone(), v0.clone()
        a = torch.empty_like(x)

        def step():
            x.copy_(x0)
            v.copy_(v0)
            nb.tree_step(x, v, m, G, eps, theta, lc, dt, K, a, group=grp)

        # interactions of one step, eval by eval (the walk is deterministic)
        inter = []
        step_evals = []
        x.copy_(x0)
        v.copy_(v0)
        nb.tree_forces(x, m, G, eps, theta, lc, out=a, group=grp)
        st = nb.tree_stats()
        inter.append(st["cell_interactions"] + st["body_interactions"])
        step_evals.append(st)
        for _ in range(K):
            nb.tree_step(x, v, m, G, eps, theta, lc, dt, 1, a, acc_valid=True, group=grp)
            st = nb.tree_stats()
            inter.append(st["cell_interactions"] + st["body_interactions"])
        per_step = float(sum(inter))
        warm = max(args.warmup, 10)  # about a second of GPU work before timing
        for _ in range(warm):
            step()
        nb.profile(True)
        l0 = nb.launches
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = None
        clocks = ClockSampler(gpu_id)
        clocks.wait_ready()
        with Timer(torch, dev, stream, lambda: None) as t:
            for _ in range(args.steps):
                step()
                flush.fill_(1.0)
        ck = clocks.stop()
        launches = nb.launches - l0
        wn, wms = nb.profile_read(4)
        bn, bms = nb.profile_read(5)
        nb.profile(False)
        # walk time per schedule (the paper's Table VI study of loop schedules,
        # here on the tree walk): eager evaluations of the initial state
        study = []
        for sched, chunk in (("static", 1), ("dynamic", 1), ("dynamic", 4), ("dynamic", 16),
                             ("dynamic", 64), ("guided", 1), ("guided", 4)):
            nb.tree_schedule(sched, chunk)
            nb.tree_forces(x0, m, G, eps, theta, lc, out=a, group=grp)
            nb.profile(True)
            for _ in range(3):
                nb.tree_forces(x0, m, G, eps, theta, lc, out=a, group=grp)
            sn, sms = nb.profile_read(4)
            nb.profile(False)
            study.append({"sched": sched, "chunk": chunk, "walk_ms": sms / max(sn, 1)})
        nb.tree_schedule(args.tree_sched, args.tree_chunk)
        # accuracy of the first evaluation: tree vs the exact sum on sampled bodies
        rows = inputs.sample_rows(b.n, 4096, seed=1)
        ref = oracle.accel_rows(b.pos, b.mass, rows, G, eps)
        at_all, cnt_all = nb.tree_forces(x0, m, G, eps, theta, lc, group=grp, counts=True)
        at_all, cnt_all = at_all.cpu().numpy(), cnt_all.cpu().numpy().astype(np.int64)
        at = at_all[rows]
        e = np.linalg.norm(at - ref, axis=1) / np.linalg.norm(ref, axis=1)
        # parity at full size: 48 seeded groups against the oracle's tree code
        ngroups = (b.n + grp - 1) // grp
        gsel = np.sort(np.random.default_rng(5).choice(ngroups, min(48, ngroups), replace=False))
        gidx, ga, gc = oracle.bh_groups(b.pos, b.mass, G, eps, theta, lc, grp, gsel)
        gi = gidx[gidx >= 0]
        ge = np.linalg.norm(at_all[gi] - ga[gi], axis=1) / np.linalg.norm(ga[gi], axis=1)
        parity = {"sampled_groups": int(gsel.size), "bodies": int(gi.size), "n": b.n,
                  "counts_equal_oracle": bool(np.array_equal(cnt_all[gi], gc[gi])),
                  "force_rel_err_max": float(ge.max()),
                  "force_rel_err_rms": float(np.sqrt((ge ** 2).mean())),
                  "vs": "oracle tree code (oracle_bh_groups), same tree and groups"}
    value = per_step * args.steps / (t.ms / 1e3) / 1e9
    evals = K + 1
    walk_ms = wms / max(wn, 1)
    sm_max = (ck or {}).get("sm_max_mhz") or NOMINAL_SM_MAX_MHZ
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = num_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = FLOPS_PER_INTERACTION * per_step / evals / (walk_ms / 1e3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        rate, sample, bs, rcnt = tree_oracle_rate(w, theta, lc, grp)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        with nbody.NBody(bs.n, "fp32_comp", device=dev.index) as nb:
            _, gcnt = nb.tree_forces(T(bs.pos), T(bs.mass), G, eps, theta, lc, counts=True,
                                     group=grp)
            nb.sync()
        parity["counts_equal_oracle_whole_run"] = {
            "n": bs.n, "equal": bool(np.array_equal(gcnt.cpu().numpy(), rcnt))}
    n = float(b.n)
    line = {"metric": TREE_METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": warm, "ms_per_step": t.ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": w["name"] if args.n_per == WORKLOAD["n_per"] else
                       f"two-plummer N={b.n} tree", "n": b.n, "theta": theta, "leaf_cap": lc,
                       "group": grp, "schedule": f"{args.tree_sched}, chunk {args.tree_chunk}",
                       "force_evals_per_step": evals,
                       "l2": "256 MiB buffer written between steps"},
            "interactions_per_step": per_step,
            "first_eval": {"nodes": step_evals[0]["nodes"], "leaves": step_evals[0]["leaves"],
                           "cell_interactions": step_evals[0]["cell_interactions"],
                           "body_interactions": step_evals[0]["body_interactions"]},
            "ms_per_force_eval": t.ms / args.steps / evals,
            "walk_ms": walk_ms, "build_ms": bms / max(bn, 1),
            "direct_sum_equivalent": {"value": n * n * evals * args.steps / (t.ms / 1e3) / 1e9,
                                      "unit": UNIT, "note": "N^2 per evaluation / time"},
            "force_error_vs_direct_sum": {"rms": float(np.sqrt((e ** 2).mean())),
                                          "max": float(e.max()),
                                          "sample": "4096 bodies, FP64 oracle direct sum"},
            "roofline": {"bound": "alu", "kernel": "tree_walk_kernel", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": traffic_from_profile("tree_walk_two_plummer_n1048576_dram.md",
                                                         "tree.cu")
                         if (b.n, theta, lc, grp) == (1 << 20, 0.5, 16, 64) else None,
                         "note": f"{FLOPS_PER_INTERACTION} flops per cell or body interaction; "
                                 "walk kernel event-timed inside the timed region; peak = SMs x "
                                 "128 FP32 lanes x 2 x max SM clock"},
            "schedule_study": study,
            "parity": parity, "cpu_baseline": cpu, "clocks": ck, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    return 0


def fmm_workload(args, ws, torch, dev, stream, T, flush):
    """Fast multipole line: value = bodies per evaluation / time (a rate that
    does not grow with N for an O(N) method), K evaluations with the tree
    rebuilt each time; the direct-sum-equivalent N^2 rate beside it."""
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody
    w = FMM
    theta = w["theta"] if args.theta is None else args.theta
    lc = w["leaf_cap"] if args.leaf_cap is None else args.leaf_cap
    order = w["order"] if args.order is None else args.order
    b = inputs.two_plummer(args.n_per, seed=w["seed"])
    x, m = T(b.pos), T(b.mass)
    G, eps = 1.0, w["eps"]
    with nbody.NBody(b.n, "fp32_comp", device=dev.index) as nb:
        a = nb.fmm_forces(x, m, G, eps, theta, order, lc)
        st = nb.fmm_stats()
        warm = max(args.warmup, 10)  # about a tenth of a second of GPU work before timing
        for _ in range(warm):
            nb.fmm_forces(x, m, G, eps, theta, order, lc, out=a)
        nb.profile(True)
        l0 = nb.launches
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = None
        clocks = ClockSampler(gpu_id)
        clocks.wait_ready()
        with Timer(torch, dev, stream, lambda: None) as t:
            for _ in range(args.steps):
                nb.fmm_forces(x, m, G, eps, theta, order, lc, out=a)
                flush.fill_(1.0)
        ck = clocks.stop()
        launches = nb.launches - l0
        bn, bms = nb.profile_read(5)
        fn, fms = nb.profile_read(6)
        qn, qms = nb.profile_read(7)
        nb.profile(False)
        # accuracy against the exact sum on sampled bodies; every body must
        # meet every other once (through an expansion or directly)
        rows = inputs.sample_rows(b.n, 4096, seed=1)
        ref = oracle.accel_rows(b.pos, b.mass, rows, G, eps)
        af, cnt = nb.fmm_forces(x, m, G, eps, theta, order, lc, counts=True)
        af, cnt = af.cpu().numpy(), cnt.cpu().numpy().astype(np.int64)
        e = np.linalg.norm(af[rows] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        covers = bool(np.all(cnt[:, 1] + cnt[:, 2] == b.n))
    n = float(b.n)
    value = n * args.steps / (t.ms / 1e3) / 1e9
    far_ms, near_ms, build_ms = fms / max(fn, 1), qms / max(qn, 1), bms / max(bn, 1)
    sm_max = (ck or {}).get("sm_max_mhz") or NOMINAL_SM_MAX_MHZ
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = num_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    far_tf = st["expansions"] * m2l_flops(order) / (far_ms / 1e3) / 1e12
    near_tf = FLOPS_PER_INTERACTION * st["direct_pairs"] / (near_ms / 1e3) / 1e12
    phases = {
        "far": {"kernels": "fmm_p2m_kernel, fmm_m2m_kernel x 10 levels, fmm_lists_kernel x 11 "
                           "levels + 1 over the leaves, fmm_m2l_kernel, fmm_l2l_kernel x 10 "
                           "levels, fmm_items_kernel",
                "ms": far_ms, "expansions": st["expansions"], "achieved_tflops": far_tf,
                "flops_per_expansion": m2l_flops(order)},
        "near": {"kernels": "fmm_near_kernel, fmm_combine_kernel", "ms": near_ms,
                 "direct_pairs": st["direct_pairs"], "achieved_tflops": near_tf,
                 "pairs_per_s": st["direct_pairs"] / (near_ms / 1e3) / 1e9},
        "build_ms": build_ms}
    far_dominant = far_ms >= near_ms
    roof = {"bound": "alu",
            "kernel": "far phase: fmm_m2l_kernel with the upward, list and L2L passes" if far_dominant
            else "fmm_near_kernel",
            "achieved": far_tf if far_dominant else near_tf, "peak": peak, "unit": "TFLOP/s",
            "frac": (far_tf if far_dominant else near_tf) / peak,
            "traffic": traffic_from_profile(
                "fmm_far_two_plummer_n1048576_dram.md" if far_dominant
                else "fmm_near_two_plummer_n1048576_dram.md", "fmm_impl.cuh")
            if (b.n, theta, lc, order) == (1 << 20, 0.6, 64, 6) else None,
            "note": f"far: {m2l_flops(order)} flops per cell-to-cell expansion (its contraction); "
                    f"near: {FLOPS_PER_INTERACTION} per pair; phases event-timed inside the timed "
                    "region; peak = SMs x 128 FP32 lanes x 2 x max SM clock"}
    cpu, parity = None, None
    if not args.no_cpu_baseline:
        bs = inputs.two_plummer(w["cpu_n_per"], seed=w["seed"])
        t0 = time.perf_counter()
        ra, rst, rc = oracle.fmm_forces(bs.pos, bs.mass, G, eps, theta, order, lc, counts=True)
        el = time.perf_counter() - t0
        sample = (f"two-plummer N={bs.n} (same recipe), theta {theta}, order {order}, leaves <= "
                  f"{lc}: one evaluation, {el:.1f} s")
        cpu = {"value": float(bs.n) / el / 1e9, "unit": FMM_UNIT, "cores": oracle.threads(),
               "kind": "oracle", "sample": sample}
        with nbody.NBody(bs.n, "fp32_comp", device=dev.index) as nb:
            ga, gc = nb.fmm_forces(T(bs.pos), T(bs.mass), G, eps, theta, order, lc, counts=True)
            nb.sync()
            gst = nb.fmm_stats()
        ga, gc = ga.cpu().numpy(), gc.cpu().numpy().astype(np.int64)
        rms_a = np.sqrt((np.linalg.norm(ra, axis=1) ** 2).mean())
        pe = np.linalg.norm(ga - ra, axis=1) / rms_a
        parity = {"n": bs.n, "counts_equal_oracle": bool(np.array_equal(gc, rc)),
                  "stats_equal_oracle": gst == rst,
                  "force_err_max": float(pe.max()), "force_err_rms": float(np.sqrt((pe ** 2).mean())),
                  "norm": "per body |a - a_oracle| / rms |a_oracle|",
                  "vs": "oracle fast multipole method, whole run"}
    line = {"metric": FMM_METRIC, "value": value, "unit": FMM_UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": warm, "ms_per_step": t.ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": w["name"] if args.n_per == WORKLOAD["n_per"] else
                       f"two-plummer N={b.n} fmm", "n": b.n, "theta": theta, "order": order,
                       "leaf_cap": lc, "force_evals_per_step": 1,
                       "l2": "256 MiB buffer written between steps"},
            "first_eval": st, "phases": phases,
            "ms_per_force_eval": t.ms / args.steps,
            "direct_sum_equivalent": {"value": n * n * args.steps / (t.ms / 1e3) / 1e9,
                                      "unit": UNIT, "note": "N^2 per evaluation / time"},
            "force_error_vs_direct_sum": {"rms": float(np.sqrt((e ** 2).mean())),
                                          "max": float(e.max()),
                                          "sample": "4096 bodies, FP64 oracle direct sum"},
            "every_pair_met_once": covers,
            "roofline": roof, "parity": parity, "cpu_baseline": cpu, "clocks": ck,
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    return 0


def other_workload(args, ws, rank, local):
    """precision / plain / differentiation: single-GPU lines (rank 0 only)."""
    if rank != 0:
        return 0
    import numpy as np
    import torch
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody, tune
    from paper_1211_2292_gb300.autograd import rollout
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    table = None if args.tuning in ("none", "default") else args.tuning
    timer = lambda: Timer(torch, dev, stream, lambda: None)  # noqa: E731
    T = lambda a: torch.as_tensor(a, device=dev).contiguous()  # noqa: E731
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush.fill_(1.0)  # first use outside the timed region (kernel load / JIT)
    cpu = None

    if args.workload == "precision":
        w = PRECISION
        b = inputs.plummer(w["n"], seed=w["seed"])
        rows = inputs.sample_rows(b.n, 4096, seed=1)
        t0 = time.perf_counter()
        oracle.accel_rows(b.pos, b.mass, rows, 1.0, w["eps"])
        el = time.perf_counter() - t0
        cpu = {"value": rows.size * b.n / el / 1e9, "unit": UNIT, "cores": oracle.threads(),
               "kind": "oracle", "sample": f"4096 of {b.n} force rows ({el:.1f} s)"}
        with nbody.NBody(b.n, "fp32_comp", device=dev.index) as nb:
            if args.tuning != "none":
                tune.apply(nb, table)
            x, v, m = T(b.pos), T(b.vel), T(b.mass)
            a = torch.empty_like(x)
            for _ in range(args.warmup):
                xs, vs = x.clone(), v.clone()
                nb.step(xs, vs, m, 1.0, w["eps"], w["dt"], w["steps"], a)
            l0 = nb.launches
            with timer() as t:
                for _ in range(args.steps):
                    nb.step(x, v, m, 1.0, w["eps"], w["dt"], w["steps"], a)
                    flush.fill_(1.0)
            launches = nb.launches - l0
        evals = w["steps"] + 1
        value = float(b.n) ** 2 * evals * args.steps / (t.ms / 1e3) / 1e9
        pf = precision_form(torch, dev, tune, table, args.tuning)
        extra = {"force_error": dict(pf["fp32"]["force_error"],
                                     fp64_max=pf["fp64"]["force_error"]["max"],
                                     sample="4096 bodies (seeded), vs FP64 oracle"),
                 "energy": dict(pf["energy"], note="100 steps of dt 5e-4 from the initial "
                                                   "state; energies in FP64"),
                 "fp64_form": pf["fp64"], "fp32_over_fp64": pf["fp32_over_fp64"],
                 "cpu_baseline": cpu, "gpu_launches": launches}
        _line(args, ws, value, t.ms / args.steps,
              {"workload": w["name"], "n": b.n, "force_evals_per_step": evals,
               "precision": "fp32_comp", "state": "f64"}, extra)
        return 0

    if args.workload == "plain":
        w = PLAIN
        b = inputs.plummer(w["n"], seed=w["seed"])
        t0 = time.perf_counter()
        rx, rv, ra = oracle.kdk(b.pos, b.vel, b.mass, 1.0, w["eps"], w["dt"], w["steps"])
        re = oracle.energy(rx, rv, b.mass, 1.0, w["eps"])
        el = time.perf_counter() - t0
        evals = w["steps"] + 1
        cpu = {"value": float(b.n) ** 2 * evals / el / 1e9, "unit": UNIT,
               "cores": oracle.threads(), "kind": "oracle",
               "sample": f"the whole workload ({el:.3f} s incl. energy)"}
        with nbody.NBody(b.n, "fp64", device=dev.index) as nb:
            if args.tuning != "none":
                tune.apply(nb, table)
            x, v, m = T(b.pos), T(b.vel), T(b.mass)
            a = torch.empty_like(x)
            xs, vs = x.clone(), v.clone()
            for _ in range(args.warmup):
                xs.copy_(x)
                vs.copy_(v)
                nb.step(xs, vs, m, 1.0, w["eps"], w["dt"], w["steps"], a, graph=True)
            l0 = nb.launches
            with timer() as t:
                for _ in range(args.steps):
                    xs.copy_(x)
                    vs.copy_(v)
                    nb.step(xs, vs, m, 1.0, w["eps"], w["dt"], w["steps"], a, graph=True)
            launches = nb.launches - l0
            e1 = nb.energy(xs, vs, m, 1.0, w["eps"])
            ga = a.cpu().numpy()
            err = np.linalg.norm(ga - ra, axis=1) / np.linalg.norm(ra, axis=1)
            extra = {"parity": {"acc_max_rel": float(err.max()),
                                "pos_max_abs": float(np.abs(xs.cpu().numpy() - rx).max()),
                                "energy_rel": abs(e1[2] - re[2]) / abs(re[2]),
                                "vs": "FP64 oracle, same workload"},
                     "cpu_baseline": cpu, "gpu_launches": launches}
        value = float(b.n) ** 2 * evals * args.steps / (t.ms / 1e3) / 1e9
        _line(args, ws, value, t.ms / args.steps,
              {"workload": w["name"], "n": b.n, "force_evals_per_step": evals,
               "precision": "fp64", "state": "f64"}, extra, dtype="f64")
        return 0

    if args.workload == "tree":
        return tree_workload(args, ws, torch, dev, stream, T, flush, table)
    if args.workload == "fmm":
        return fmm_workload(args, ws, torch, dev, stream, T, flush)

    # differentiation
    a_ = ADJOINT
    b, dx = inputs.plummer_with_perturbation(a_["n"], seed=a_["seed"])
    with nbody.NBody(b.n, "fp32_comp", device=dev.index) as nb:
        if args.tuning != "none":
            tune.apply(nb, table)
        x, v, m = T(b.pos), T(b.vel), T(b.mass)
        tgt = T(b.pos + dx)  # stand-in target for timing; parity uses the oracle's run

        def grad():
            x0 = x.clone().requires_grad_()
            v0 = v.clone().requires_grad_()
            mm = m.clone().requires_grad_()
            xT, _ = rollout(nb, x0, v0, mm, 1.0, a_["eps"], a_["dt"], a_["steps"], a_["every"])
            loss = ((xT - tgt) ** 2).sum(-1).mean()
            loss.backward()
            return loss

        for _ in range(args.warmup):
            grad()
        l0 = nb.launches
        with timer() as t:
            for _ in range(args.steps):
                grad()
        launches = nb.launches - l0
    K = a_["steps"]
    force_evals = (K + 1) + (K + K // a_["every"])  # forward + per-segment recompute
    vjp_evals = K + 1
    pairs = float(b.n) ** 2 * (force_evals + vjp_evals)
    value = pairs * args.steps / (t.ms / 1e3) / 1e9
    _line(args, ws, value, t.ms / args.steps,
          {"workload": f"Plummer N={b.n}, eps {a_['eps']}, {K} KDK steps of dt {a_['dt']}, "
                       f"gradient w.r.t. x0, v0, m with checkpoints every {a_['every']}",
           "n": b.n, "force_evals_per_step": force_evals, "vjp_evals_per_step": vjp_evals,
           "precision": "fp32_comp (float64 adjoint accumulation)"},
          {"gradient_ms": t.ms / args.steps, "gpu_launches": launches,
           "note": "interactions counted for forward, recompute and VJP evaluations"})
    return 0


LET_W = {"name": "two-plummer N=1048576, parallel tree code (ORB domains, locally essential "
                 "trees), Barnes-Hut theta 0.5, leaves <= 16, groups of 64, one force evaluation "
                 "per step", "seed": 2, "eps": 0.002, "theta": 0.5, "leaf_cap": 16, "group": 64}


def let_workload(args, ws, rank, local):
    """Parallel tree code line (paper Sec. IV-B).  Under torchrun, one process
    per GPU over NCCL.  On one GPU, --procs processes are emulated by threads
    whose kernels run one after another on the device: the line then gives
    the single-GPU cost of the sharded evaluation (every process's ORB,
    exchange, tree, LET exports and walks), not a multi-GPU time.  value =
    cell + body interactions of all processes / the force phase's time (tree
    build, LET export and exchange, walks)."""
    import numpy as np
    import torch
    from paper_1211_2292_gb300 import inputs, let, nbody
    w = LET_W
    b = inputs.two_plummer(args.n_per, seed=w["seed"])
    N = b.n
    G, eps, th, lc, grp = 1.0, w["eps"], w["theta"], w["leaf_cap"], w["group"]
    emulated = ws == 1
    P = args.procs if emulated else ws
    if not emulated:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if not emulated else 0)
    torch.cuda.set_device(dev)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def proc(comm):
        r = comm.rank
        lo, hi = r * N // P, (r + 1) * N // P
        with nbody.NBody(N if emulated else max(2 * (hi - lo), 1), "fp32_comp",
                         device=dev.index) as nb:
            x, v, m = (torch.as_tensor(a[lo:hi], device=dev).contiguous()
                       for a in (b.pos, b.vel, b.mass))
            ids = torch.arange(lo, hi, dtype=torch.int64, device=dev)
            e0 = ev()
            part = let.orb_partition(nb, comm, x, ids)
            x, v, m, ids = let.exchange(nb, comm, part, x, v, m, ids)
            e1 = ev()
            torch.cuda.synchronize(dev)
            orb_ms = e0.elapsed_time(e1)
            for _ in range(args.warmup):
                let.let_forces(nb, comm, x, m, G, eps, th, lc, grp)
            t = []
            nb.profile(True)
            for _ in range(args.steps):
                # a collective on each side: the span covers every process's
                # kernels (on one GPU they share the device's default stream)
                comm.allreduce(np.zeros(1), "sum")
                torch.cuda.synchronize(dev)
                a0 = ev()
                let.let_forces(nb, comm, x, m, G, eps, th, lc, grp)
                comm.allreduce(np.zeros(1), "sum")
                a1 = ev()
                torch.cuda.synchronize(dev)
                t.append(a0.elapsed_time(a1))
            nb.profile(False)
            # the walk kernels alone: the processes in turn (the others wait at
            # a host barrier, so on one GPU no other work is on the device),
            # each walking its tree and its received LETs once more
            _, lets = let.let_forces(nb, comm, x, m, G, eps, th, lc, grp, return_lets=True)
            wn, wms = 0, 0.0
            for turn in range(P):
                comm.allreduce(np.zeros(1), "sum")
                if turn == comm.rank and x.shape[0]:
                    torch.cuda.synchronize(dev)
                    nb.profile(True)
                    nb.let_forces(G, eps, th, grp, lets)
                    wn, wms = nb.profile_read(4)
                    nb.profile(False)
            st = nb.tree_stats() if x.shape[0] else {"cell_interactions": 0, "body_interactions": 0}
            return {"n": int(x.shape[0]), "orb_exchange_ms": orb_ms,
                    "force_ms": float(np.mean(t)), "walk_ms": wms, "walks": wn,
                    "interactions": st["cell_interactions"] + st["body_interactions"]}

    if emulated:
        res = let.run_threads(P, proc)
    else:
        mine = proc(let.TorchComm(device=f"cuda:{local}"))
        res = [None] * ws
        torch.distributed.all_gather_object(res, mine)
    if rank == 0:
        inter = sum(r["interactions"] for r in res)
        # the evaluation's span: the slowest process (on one GPU every
        # process's span covers all processes' kernels)
        span = max(r["force_ms"] for r in res)
        # the walk kernels' roofline: 20 flops per cell or body interaction
        # over the walks' summed event time (every process's walks, one after
        # another on one GPU; the slowest process's on several)
        walk_ms = (sum if emulated else max)(r["walk_ms"] for r in res)
        props = torch.cuda.get_device_properties(dev)
        sm_max = float(load_peaks().get("sm_max_mhz", NOMINAL_SM_MAX_MHZ))
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        achieved = FLOPS_PER_INTERACTION * inter / (walk_ms / 1e3) / 1e12
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            bs = inputs.two_plummer(TREE["cpu_n_per"], seed=w["seed"])
            rk = oracle.orb(bs.pos, P)
            t0 = time.perf_counter()
            _, cst, _ = oracle.bh_sharded(bs.pos, bs.mass, G, eps, th, lc, grp, rk, P)
            el = time.perf_counter() - t0
            cpu = {"value": (cst["cell_interactions"] + cst["body_interactions"]) / el / 1e9,
                   "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the oracle's parallel tree code on two-plummer N={bs.n} (same "
                             f"recipe) over {P} ORB domains: one evaluation, {el:.1f} s"}
        line = {"metric": TREE_METRIC, "value": inter / (span / 1e3) / 1e9, "unit": UNIT,
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": span,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded Plummer spheres)",
                "config": {"workload": w["name"], "n": N, "processes": P,
                           "processes_emulated_on_one_gpu": emulated,
                           "theta": th, "leaf_cap": lc, "group": grp},
                "per_process": res,
                "roofline": {"bound": "alu", "kernel": "tree_walk_kernel (local tree and LETs)",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None,
                             "note": f"{FLOPS_PER_INTERACTION} flops per cell or body "
                                     "interaction over the walks' event time"},
                "cpu_baseline": cpu,
                "note": ("processes emulated by threads on one GPU: their kernels run one "
                         "after another, so this is the one-GPU cost of the sharded "
                         "evaluation, not a multi-GPU time" if emulated else
                         "one process per GPU over NCCL")}
        print(json.dumps(line), flush=True)
    if not emulated:
        torch.distributed.destroy_process_group()
    return 0


def _relerr(a, ref):
    import numpy as np
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _err_stats(a, ref):
    import numpy as np
    e = _relerr(a, ref)
    return {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}


def float64_forms(torch, dev, tune, table, args, b, n64, G, eps, dt, nk, err_idx, ref_rows,
                  fp32_rate):
    """The metric's comparison: the same workload in the FP64 form (one force
    evaluation, kernel event-timed) and in the double-float form (1 + nk KDK
    steps, as the float32 line), each with its per-body relative force error
    against the FP64 oracle on the float32 line's 4096 sampled bodies."""
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody
    x = torch.as_tensor(b.pos[:n64], device=dev).contiguous()
    v = torch.as_tensor(b.vel[:n64], device=dev).contiguous()
    m = torch.as_tensor(b.mass[:n64], device=dev).contiguous()
    if n64 == b.n:
        rows, ref = err_idx, ref_rows
        sample = f"{rows.size} bodies (seeded, as the float32 line), vs FP64 oracle"
    else:
        rows = inputs.sample_rows(n64, 256, seed=3)
        ref = oracle.accel_rows(b.pos[:n64], b.mass[:n64], rows, G, eps)
        sample = f"{rows.size} of the first {n64} bodies (seeded), vs FP64 oracle"
    pairs = float(n64) ** 2
    with nbody.NBody(n64, "fp64", device=dev.index) as nb64:
        if args.tuning != "none":
            tune.apply(nb64, table)
        a64 = torch.empty_like(x)
        nb64.profile(True)
        nb64.forces(x, m, G, eps, out=a64)
        k64, ms64 = nb64.profile_read(0)
        nb64.profile(False)
        nb64.sync()
    v64 = pairs / (ms64 / max(k64, 1) / 1e3) / 1e9
    err64 = _err_stats(a64.cpu().numpy()[rows], ref)
    out = {"value": v64, "unit": UNIT, "n": n64, "force_evals": 1,
           "kernel_ms": ms64 / max(k64, 1), "fp32_over_fp64": fp32_rate / v64,
           "force_error": dict(err64, sample=sample),
           "note": "one FP64 force evaluation of the whole workload, kernel event-timed"}
    with nbody.NBody(n64, "df64", device=dev.index) as nbd:
        if args.tuning != "none":
            tune.apply(nbd, table)
        ad = nbd.forces(x, m, G, eps)
        errd = _err_stats(ad.cpu().numpy()[rows], ref)
        xs, vs = x.clone(), v.clone()
        stream = torch.cuda.current_stream(dev)
        nbd.profile(True)
        with Timer(torch, dev, stream, lambda: None) as t:
            nbd.step(xs, vs, m, G, eps, dt, nk, ad)
        kd, msd = nbd.profile_read(0)
        nbd.profile(False)
        nbd.sync()
    vd = pairs / (msd / max(kd, 1) / 1e3) / 1e9
    out["df64_form"] = {
        "value": vd, "unit": UNIT, "n": n64, "force_evals": kd, "kernel_ms": msd / max(kd, 1),
        "step_value": pairs * kd / (t.ms / 1e3) / 1e9, "ms_per_step": t.ms,
        "over_fp64": vd / v64, "fp32_over_df64": fp32_rate / vd,
        "force_error": dict(errd, sample=sample),
        "note": f"double-float pair arithmetic (error-free sums and products of float32 "
                f"pairs), Morton order; one step = 1 + {nk} KDK steps as the float32 line"}
    return out


def precision_form(torch, dev, tune, table, tuning="default"):
    """The precision workload (Plummer N = 65,536, eps 0.005, 100 KDK steps of
    dt 5e-4) in the float32 compensated and FP64 forms on the GPU: force error
    against the oracle on 4096 sampled bodies, energy drift of each run and the
    float32 run's difference from the FP64 GPU run."""
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody
    w = PRECISION
    b = inputs.plummer(w["n"], seed=w["seed"])
    rows = inputs.sample_rows(b.n, 4096, seed=1)
    ref = oracle.accel_rows(b.pos, b.mass, rows, 1.0, w["eps"])
    stream = torch.cuda.current_stream(dev)
    T = lambda a: torch.as_tensor(a, device=dev).contiguous()  # noqa: E731
    res = {}
    for prec in ("fp64", "fp32_comp"):
        with nbody.NBody(b.n, prec, device=dev.index) as nb:
            if tuning != "none":
                tune.apply(nb, table)
            x, v, m = T(b.pos), T(b.vel), T(b.mass)
            a = nb.forces(x, m, 1.0, w["eps"])
            err = _err_stats(a.cpu().numpy()[rows], ref)
            e0 = nb.energy(x, v, m, 1.0, w["eps"])
            with Timer(torch, dev, stream, lambda: None) as t:
                nb.step(x, v, m, 1.0, w["eps"], w["dt"], w["steps"], a, acc_valid=True)
            e1 = nb.energy(x, v, m, 1.0, w["eps"])
            nb.sync()
            res[prec] = {"err": err, "e0": e0, "e1": e1, "x": x.cpu().numpy(), "ms": t.ms}
    r32, r64 = res["fp32_comp"], res["fp64"]
    pairs = float(b.n) ** 2 * w["steps"]
    return {
        "workload": w["name"], "n": b.n, "steps": w["steps"],
        "fp32": {"value": pairs / (r32["ms"] / 1e3) / 1e9, "unit": UNIT, "ms": r32["ms"],
                 "force_error": r32["err"]},
        "fp64": {"value": pairs / (r64["ms"] / 1e3) / 1e9, "unit": UNIT, "ms": r64["ms"],
                 "force_error": r64["err"]},
        "fp32_over_fp64": r64["ms"] / r32["ms"],
        "energy": {"E0": r64["e0"][2],
                   "drift_fp64_gpu": abs(r64["e1"][2] - r64["e0"][2]) / abs(r64["e0"][2]),
                   "drift_fp32": abs(r32["e1"][2] - r32["e0"][2]) / abs(r32["e0"][2]),
                   "fp32_vs_fp64_final": abs(r32["e1"][2] - r64["e1"][2]) / abs(r64["e0"][2]),
                   "max_position_diff": float(np.abs(r32["x"] - r64["x"]).max())},
        "note": "force error on 4096 sampled bodies vs the FP64 oracle; energies (FP64 "
                "diagnostics) before and after 100 steps from the initial state; value = "
                "N^2 x 100 / the 100-step run's time (cached first force)"}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    if args.workload == "let":
        if args.warmup < 3:
            args.warmup = 3
        return let_workload(args, ws, rank, local)
    if args.workload in ("precision", "plain", "differentiation", "tree", "fmm"):
        if args.warmup < 3:
            args.warmup = 3
        return other_workload(args, ws, rank, local)

    import numpy as np
    import torch
    import oracle
    from paper_1211_2292_gb300 import inputs, nbody, shard, tune

    if args.warmup < 3:
        print("bench: --warmup raised to 3", file=sys.stderr)
        args.warmup = 3

    # ---------------------------------------------------------------- inputs
    if args.workload == "batched":
        w = BATCHED
        bodies, off = inputs.plummer_batch(w["nsys"], w["lo"], w["hi"], seed=w["seed"])
        mine = shard.shard_systems(np.diff(off), ws, rank)
        idx, loc = shard.gather_rows(off, mine)
        b = inputs.Bodies(bodies.pos[idx], bodies.vel[idx], bodies.mass[idx])
        pairs_per_eval = float(sum(int(loc[k + 1] - loc[k]) ** 2 for k in range(len(loc) - 1)))
        G, eps, dt, nk = w["G"], w["eps"], w["dt"], w["steps"]
        wname, evals = w["name"], nk
        prec_desc = "fp32_comp (batched persistent kernel, graph)"
    else:
        w = WORKLOAD
        b = inputs.two_plummer(args.n_per, seed=w["seed"])
        G, eps, dt, nk = w["G"], w["eps"], w["dt"], w["steps"]
        wname = w["name"] if b.n == 2 * w["n_per"] else w["name"].replace("1048576", str(b.n))
        pairs_per_eval = float(b.n) ** 2
        evals = nk + 1
        prec_desc = "fp32_comp"
    n = b.n

    # CPU baseline (oracle, before any GPU work) and float32 error reference
    cpu, err_idx, ref_rows = None, None, None
    if args.workload == "throughput":
        err_idx = inputs.sample_rows(n, 4096, seed=1)
        t0 = time.perf_counter()
        ref_rows = oracle.accel_rows(b.pos, b.mass, err_idx, G, eps)
        t_err = time.perf_counter() - t0
        if rank == 0 and not args.no_cpu_baseline:
            rate, el, rows = err_idx.size * n / t_err, t_err, err_idx.size
            if t_err < 0.5 * args.cpu_seconds:
                rate, el, rows = oracle_rate(b.pos, b.mass, G, eps, args.cpu_seconds)
            cpu = {"value": rate / 1e9, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                   "sample": f"{rows} of {n} rows of one force evaluation ({el:.1f} s, FP64 C)"}
    elif rank == 0 and not args.no_cpu_baseline:
        k = int(np.argmax(np.diff(off)))
        s, e = off[k], off[k + 1]
        rate, el, rows = oracle_rate(bodies.pos[s:e], bodies.mass[s:e], G, eps, args.cpu_seconds)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{rows} force rows of the largest system (N={e - s}) ({el:.1f} s)"}

    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    barrier = (lambda: dist.barrier()) if dist is not None else (lambda: None)
    stream = torch.cuda.current_stream(dev)

    table = None if args.tuning in ("none", "default") else args.tuning
    nb = nbody.NBody(max(n, 1), "fp32_comp", device=dev.index)
    tuned = 0 if args.tuning == "none" else tune.apply(nb, table)
    if args.force_variant >= 0:
        nb.tune_set(0, 0, 1 << 40, args.force_variant, 0)
    pos = torch.as_tensor(b.pos, device=dev).contiguous()
    vel = torch.as_tensor(b.vel, device=dev).contiguous()
    mass = torch.as_tensor(b.mass, device=dev).contiguous()
    acc = torch.empty_like(pos)

    force_err = None
    if args.workload == "throughput":
        a0 = nb.forces(pos, mass, G, eps).cpu().numpy()[err_idx]
        e = np.linalg.norm(a0 - ref_rows, axis=1) / np.linalg.norm(ref_rows, axis=1)
        force_err = {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max()),
                     "sample": "4096 bodies (seeded), vs FP64 oracle"}

    if args.workload == "batched":
        nb.batch_plan(loc)
        nb.forces_batched(pos, mass, G, eps, out=acc)

        def step():
            nb.step_batched(pos, vel, mass, G, eps, dt, nk, acc, acc_valid=True, graph=True)
    else:
        def step():
            nb.step(pos, vel, mass, G, eps, dt, nk, acc)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush.fill_(1.0)  # first use outside the timed region (kernel load / JIT)
    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    clocks.wait_ready()
    nb.profile(True)
    l0 = nb.launches
    with Timer(torch, dev, stream, barrier) as t:
        for _ in range(args.steps):
            step()
            flush.fill_(1.0)
    launches = nb.launches - l0
    kind = 1 if args.workload == "batched" else 0
    nf, force_ms = nb.profile_read(kind)
    nb.profile(False)
    clk = clocks.stop()
    if nf == 0:  # kernels ran inside a captured graph: time eager launches
        nb.profile(True)
        for _ in range(3):
            nb.forces_batched(pos, mass, G, eps, out=acc)
        nf, force_ms = nb.profile_read(kind)
        nb.profile(False)
    t_max = shard.max_over_ranks(t.ms, dist)
    # every rank processes the same amount in "throughput"; in "batched" each
    # rank's share is summed
    pairs_total = pairs_per_eval * evals * args.steps
    if dist is not None:
        pt = torch.tensor([pairs_total], dtype=torch.float64, device=dev)
        dist.all_reduce(pt)
        pairs_total = float(pt.item())
    value = pairs_total / (t_max / 1e3) / 1e9

    # roofline of the dominant kernel (plain FP32 ALU work)
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(load_peaks().get("sm_max_mhz", NOMINAL_SM_MAX_MHZ))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    avg_ms = force_ms / max(nf, 1)
    achieved = FLOPS_PER_INTERACTION * pairs_per_eval / (avg_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": traffic_from_profile() if args.workload == "throughput" else None,
                "kernel": ("force_f32_batched_kernel (Kahan)" if kind else
                           "force_f32_kernel (Kahan)"),
                "launches_timed": nf, "avg_launch_ms": avg_ms,
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 "
                              f"lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz); "
                              f"{FLOPS_PER_INTERACTION} flops per interaction"}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak_tflops * clk["sm_mhz"] / sm_max)

    # float64 forms at the workload's size: one FP64 force evaluation and the
    # double-float form's 1 + 10 steps, with errors on the sampled bodies
    fp64 = None
    if args.workload == "throughput":
        n64 = n if args.fp64_n is None else min(args.fp64_n, n)
        if n64 > 0:
            fp32_rate = pairs_per_eval / (avg_ms / 1e3) / 1e9
            fp64 = float64_forms(torch, dev, tune, table, args, b, n64, G, eps, dt, nk,
                                 err_idx, ref_rows, fp32_rate)

    forms = None
    if not args.no_forms and rank == 0 and args.workload == "throughput":
        forms = measure_forms(torch, dev, tune, table, peak_tflops, tree_bodies=b,
                              tuning=args.tuning)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hp = torch.as_tensor(b.pos).pin_memory()
        hv = torch.as_tensor(b.vel).pin_memory()
        hm = torch.as_tensor(b.mass).pin_memory()
        op = torch.empty_like(hp).pin_memory()
        ov = torch.empty_like(hv).pin_memory()
        e2e_steps = max(1, min(args.steps, 3))

        def e2e_step():
            pos.copy_(hp, non_blocking=True)
            vel.copy_(hv, non_blocking=True)
            mass.copy_(hm, non_blocking=True)
            if args.workload == "batched":
                nb.step_batched(pos, vel, mass, G, eps, dt, nk, acc, graph=True)
            else:
                nb.step(pos, vel, mass, G, eps, dt, nk, acc)
            op.copy_(pos, non_blocking=True)
            ov.copy_(vel, non_blocking=True)
            flush.fill_(1.0)

        e2e_step()
        with Timer(torch, dev, stream, barrier) as te:
            for _ in range(e2e_steps):
                e2e_step()
        ems = shard.max_over_ranks(te.ms, dist)
        e_evals = evals + (1 if args.workload == "batched" else 0)
        e2e = {"value": pairs_total / (args.steps * evals) * e_evals * e2e_steps / (ems / 1e3) / 1e9,
               "unit": UNIT,
               "h2d_bytes_per_step": int(hp.numel() + hv.numel() + hm.numel()) * 8,
               "d2h_bytes_per_step": int(op.numel() + ov.numel()) * 8, "steps": e2e_steps}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak" if args.workload == "throughput" else "strong",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": wname, "n": n if ws == 1 or args.workload == "throughput"
                       else int(BATCHED["nsys"]), "G": G, "eps": eps, "dt": dt,
                       "force_evals_per_step": evals, "precision": prec_desc, "state": "f64",
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": ("single GPU" if ws == 1 else
                                       "replicas" if args.workload == "throughput" else
                                       "systems sharded across ranks (LPT), no collective"),
                       "tuning_entries": tuned, "variant": nb.tune_get(kind, n)},
            "fp32_peak_frac": roofline["frac"],
            "force_error": force_err,
            "fp64_form": fp64,
            "forms": forms,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    nb.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
