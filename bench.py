#!/usr/bin/env python
"""Throughput benchmark of the softened direct-sum n-body path on GB300.

Default workload: two Plummer spheres of 524,288 bodies each (N = 1,048,576),
centres at (+-5, 0, 0) approaching at relative velocity 0.5, lognormal
(sigma 0.5) masses normalised to 1, eps = 0.002, seed 2.  One bench step is
one force evaluation plus 10 kick-drift-kick steps (11 force evaluations) in
the float32 Kahan-compensated form with float64 state.  Metric: pairwise
interactions per second, N^2 per force evaluation.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of
the workload (the single-system path is not sharded); value is the sum over
ranks divided by the slowest rank's time.

The JSON line also carries: the float64 form's rate, the float32 force error
against the FP64 oracle on 4096 sampled bodies, the force kernel's roofline
(event-timed inside the timed region), the oracle's CPU rate, an end-to-end
rate with host buffers, the SM clocks sampled during the timed region and
the number of library kernels launched.
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
METRIC = "pairwise interactions/s (G/s)"
UNIT = "Ginteractions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-n", type=int, default=262_144,
                    help="bodies for the float64-form rate (first bodies of the workload)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-per", type=int, default=WORKLOAD["n_per"],
                    help="bodies per sphere (smaller cases for profiling)")
    ap.add_argument("--tuning", default="default",
                    help="kernel tuning table (JSON from paper_1211_2292_gb300.tune), "
                         "'default' for the packaged GB300 table, 'none' for built-in defaults")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd[1:1] = ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_from_profile():
    """DRAM bytes per force launch from the committed ncu summary, or None
    when the force kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "force_f32comp_two_plummer_n1048576.md")
    src = os.path.join(ROOT, "paper_1211_2292_gb300", "csrc", "force_f32.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("force_f32.cu sha256[:16]") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_oracle_rate(pos, mass, G, eps, target_s, rows_idx=None):
    """Oracle interactions/s on host cores over a bounded sample of rows."""
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs
    n = mass.shape[0]
    probe = inputs.sample_rows(n, 64, seed=7)
    t0 = time.perf_counter()
    oracle.accel_rows(pos, mass, probe, G, eps)
    dt0 = max(time.perf_counter() - t0, 1e-6)
    rate = probe.size * n / dt0
    rows = int(min(n, max(256, rate * target_s / n)))
    idx = inputs.sample_rows(n, rows, seed=8) if rows_idx is None else rows_idx
    t0 = time.perf_counter()
    ref = oracle.accel_rows(pos, mass, idx, G, eps)
    el = time.perf_counter() - t0
    return idx.size * n / el, el, idx, ref, oracle.threads()


def reference_arm(args, ws, rank):
    """Oracle (FP64 CPU) timed on the host cores, same metric and workload."""
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1211_2292_gb300 import inputs
    w = WORKLOAD
    b = inputs.two_plummer(w["n_per"], seed=w["seed"])
    n = b.n
    # rows per step so that one step is ~ a few seconds of CPU work
    probe = inputs.sample_rows(n, 64, seed=7)
    t0 = time.perf_counter()
    oracle.accel_rows(b.pos, b.mass, probe, w["G"], w["eps"])
    rate = probe.size * n / max(time.perf_counter() - t0, 1e-6)
    rows = int(min(n, max(128, rate * 6.0 / n)))
    idx = inputs.sample_rows(n, rows, seed=9)
    for _ in range(args.warmup):
        oracle.accel_rows(b.pos, b.mass, idx, w["G"], w["eps"])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.accel_rows(b.pos, b.mass, idx, w["G"], w["eps"])
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = rows * n * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Plummer spheres)",
        "config": {"workload": w["name"], "n": n, "eps": w["eps"],
                   "sample": f"{rows} of {n} force rows per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": f"{rows} rows x {n} bodies of one force evaluation per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, ws, rank)

    import numpy as np
    import torch
    from paper_1211_2292_gb300 import inputs, nbody

    if args.warmup < 3:
        print("bench: --warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    w = WORKLOAD
    b = inputs.two_plummer(args.n_per, seed=w["seed"])
    n = b.n
    G, eps, dt, nk = w["G"], w["eps"], w["dt"], w["steps"]
    wname = w["name"] if n == 2 * WORKLOAD["n_per"] else w["name"].replace("1048576", str(n))

    # CPU baseline (oracle) before any GPU work; its rows also give the
    # reference forces for the float32 error.
    cpu = None
    err_idx = inputs.sample_rows(n, 4096, seed=1)
    import oracle
    t0 = time.perf_counter()
    ref_rows = oracle.accel_rows(b.pos, b.mass, err_idx, G, eps)
    t_err = time.perf_counter() - t0
    if rank == 0 and not args.no_cpu_baseline:
        rate = err_idx.size * n / t_err
        el = t_err
        rows = err_idx.size
        if t_err < 0.5 * args.cpu_seconds:
            rate, el, idx2, _, _ = cpu_oracle_rate(b.pos, b.mass, G, eps, args.cpu_seconds)
            rows = idx2.size
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{rows} of {n} rows of one force evaluation ({el:.1f} s, FP64 C)"}

    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1211_2292_gb300 import tune
    table = None if args.tuning == "none" else (None if args.tuning == "default" else args.tuning)
    nb = nbody.NBody(n, "fp32_comp", device=dev.index)
    tuned = 0 if args.tuning == "none" else tune.apply(nb, table)
    pos = torch.as_tensor(b.pos, device=dev).contiguous()
    vel = torch.as_tensor(b.vel, device=dev).contiguous()
    mass = torch.as_tensor(b.mass, device=dev).contiguous()
    acc = torch.empty_like(pos)

    # float32 force error on the sampled bodies at t = 0
    a0 = nb.forces(pos, mass, G, eps).cpu().numpy()[err_idx]
    e = np.linalg.norm(a0 - ref_rows, axis=1) / np.linalg.norm(ref_rows, axis=1)
    force_err = {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max()),
                 "sample": "4096 bodies (seeded), vs FP64 oracle"}

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        nb.step(pos, vel, mass, G, eps, dt, nk, acc)
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    time.sleep(0.3)
    nb.profile(True)
    l0 = nb.launches
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        nb.step(pos, vel, mass, G, eps, dt, nk, acc)
        flush.fill_(1.0)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = nb.launches - l0
    nf, force_ms = nb.profile_read(0)
    nb.profile(False)
    clk = clocks.stop()

    evals = nk + 1
    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    inter = float(n) * n * evals * args.steps * ws
    value = inter / (t_max / 1e3) / 1e9

    # roofline of the force kernel (plain FP32 ALU work)
    props = torch.cuda.get_device_properties(dev)
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", NOMINAL_SM_MAX_MHZ))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    avg_force_ms = force_ms / max(nf, 1)
    achieved = FLOPS_PER_INTERACTION * float(n) * n / (avg_force_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic_from_profile(),
                "kernel": "force_f32_kernel (Kahan)", "launches_timed": nf,
                "avg_launch_ms": avg_force_ms,
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes"
                              f" x 2 x {sm_max:.0f} MHz (sm_max_mhz)"}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak_tflops * clk["sm_mhz"] / sm_max)

    # float64 form on the first fp64_n bodies
    fp64 = None
    n64 = min(args.fp64_n, n)
    if n64 > 0:
        nb64 = nbody.NBody(n64, "fp64", device=dev.index)
        if args.tuning != "none":
            tune.apply(nb64, table)
        p64, m64 = pos[:n64].contiguous(), mass[:n64].contiguous()
        a64 = torch.empty_like(p64)
        nb64.forces(p64, m64, G, eps, out=a64)
        nb64.profile(True)
        nb64.forces(p64, m64, G, eps, out=a64)
        k64, ms64 = nb64.profile_read(0)
        nb64.profile(False)
        fp64 = {"value": float(n64) ** 2 / (ms64 / 1e3) / 1e9, "unit": UNIT, "n": n64,
                "kernel_ms": ms64, "note": "one FP64 force evaluation of the first n bodies "
                                           "(the rate does not depend on N once the GPU is full)"}
        fp64["fp32_over_fp64"] = (float(n) * n / (avg_force_ms / 1e3) / 1e9) / fp64["value"]
        nb64.close()

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hp = torch.as_tensor(b.pos).pin_memory()
        hv = torch.as_tensor(b.vel).pin_memory()
        hm = torch.as_tensor(b.mass).pin_memory()
        op = torch.empty_like(hp).pin_memory()
        ov = torch.empty_like(hv).pin_memory()
        dp, dv, dm = torch.empty_like(pos), torch.empty_like(vel), torch.empty_like(mass)
        e2e_steps = max(1, min(args.steps, 3))

        def e2e_step():
            dp.copy_(hp, non_blocking=True)
            dv.copy_(hv, non_blocking=True)
            dm.copy_(hm, non_blocking=True)
            nb.step(dp, dv, dm, G, eps, dt, nk, acc)
            op.copy_(dp, non_blocking=True)
            ov.copy_(dv, non_blocking=True)
            flush.fill_(1.0)

        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ems = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": float(n) * n * evals * e2e_steps * ws / (ems / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(hp.numel() + hv.numel() + hm.numel()) * 8,
               "d2h_bytes_per_step": int(op.numel() + ov.numel()) * 8,
               "steps": e2e_steps}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Plummer spheres)",
            "config": {"workload": wname, "n": n, "G": G, "eps": eps, "dt": dt,
                       "force_evals_per_step": evals, "precision": "fp32_comp",
                       "state": "f64", "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "tuning_entries": tuned,
                       "variant": nb.tune_get(0, n)},
            "fp32_peak_frac": roofline["frac"],
            "force_error": force_err,
            "fp64_form": fp64,
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
