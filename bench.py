#!/usr/bin/env python3
"""Throughput benchmark of the CI-SCvx discretization/linearization hot path.

One step = one pass of the whole hot path over one batch of synthetic input:
the linearized discretization (A, B-, B+, S, defects, penalty increments) of
every interval plus the adjoint VJP of L = sum w.defect + rho.penalty, with
inputs resident in HBM.  value = intervals linearized (STM + VJP) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank processes its own batch
(instances are independent, no collective on the data path) -> weak scaling;
value = total intervals over all ranks / max rank time.

Also reported: the plain FP64 GPU path's throughput on the same workload, the
FP64-pipe roofline of the dominant kernel (CUDA events on its stream), an
end-to-end number through the public API with host buffers, the FP64 oracle
on the host cores (cpu_baseline), and SM clocks sampled during the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_09993_gb300 import synth  # noqa: E402

# FP64 peak derived from the unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
# x 2 flop x 2.07 GHz (a microbenchmark measured 1.196 TFLOP/s at 1.99 GHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

WORKLOADS = {
    # 7-link chain (HalfCheetah-shaped), N = 50, 10 RK4 substeps, one instance
    "cheetah7-n50-sub10": dict(kind="single", make=lambda: synth.cheetah_n50(seed=0)),
}
DEFAULT_WORKLOAD = "cheetah7-n50-sub10"

# Executed FP64 flops per interval of the dominant kernel (ncu SASS counters
# dfma*2 + dadd + dmul, per launch / intervals), see profiles/.
FLOPS_PER_INTERVAL = {
    ("cheetah7-n50-sub10", "discretize", "fp32_phi"): 42_900,
    ("cheetah7-n50-sub10", "discretize", "fp64"): 84_400,
    ("cheetah7-n50-sub10", "vjp", "fp32_phi"): 73_300,
}


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while active."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
class SingleWorkload:
    """One instance through ciscvx_discretize + ciscvx_discretize_vjp."""

    def __init__(self, prob, dev):
        import torch
        from paper_2604_09993_gb300 import api
        self.api, self.torch, self.p = api, torch, prob
        self.model = api.Model(prob.robot)
        t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        self.X, self.U, self.s, self.w, self.rho = (t(prob.X), t(prob.U), t(prob.s), t(prob.w), t(prob.rho))
        self.intervals = prob.N
        self.n_sub = prob.n_sub
        self.out = {}
        self.ws = torch.empty(api.workspace_size(self.model, api.OP_VJP, prob.N), dtype=torch.uint8, device=dev)

    def disc(self, precision):
        if precision not in self.out:
            self.out[precision] = self.api.discretize(self.model, self.X, self.U, self.s, self.n_sub, precision)
        else:
            self.api.discretize(self.model, self.X, self.U, self.s, self.n_sub, precision, out=self.out[precision])

    def vjp(self, precision):
        self.api.discretize_vjp(self.model, self.X, self.U, self.s, self.w, self.rho, self.n_sub, precision,
                                workspace=self.ws)

    def step(self, precision):
        self.disc(precision)
        self.vjp(precision)

    def e2e_step(self, host, precision):
        """Public API with host buffers: H2D of the inputs, compute, D2H of every output."""
        torch = self.torch
        X = host["X"].to(self.X.device, non_blocking=True)
        U = host["U"].to(self.X.device, non_blocking=True)
        s = host["s"].to(self.X.device, non_blocking=True)
        w = host["w"].to(self.X.device, non_blocking=True)
        rho = host["rho"].to(self.X.device, non_blocking=True)
        out = self.api.discretize(self.model, X, U, s, self.n_sub, precision)
        gX, gU, gs, L = self.api.discretize_vjp(self.model, X, U, s, w, rho, self.n_sub, precision, workspace=self.ws)
        res = dict(out, gX=gX, gU=gU, gs=gs, L=L)
        for k, v in res.items():
            host["out_" + k].copy_(v, non_blocking=True)
        return res

    def host_buffers(self):
        torch = self.torch
        h = {}
        for k in ("X", "U", "s", "w", "rho"):
            h[k] = getattr(self, k).cpu().pin_memory()
        return h

    def alloc_host_outputs(self, host, res):
        for k, v in res.items():
            host["out_" + k] = torch_empty_pinned(self.torch, v)

    def check_status(self):
        self.api.sync_status(self.model)


def torch_empty_pinned(torch, like):
    return torch.empty(like.shape, dtype=like.dtype, pin_memory=True)


def time_steps(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def kernel_time(torch, fn, reps, stream):
    """Average duration of one call of fn (a single kernel launch sequence) with events on its stream."""
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.mean(ts)


def cpu_baseline(name, seconds_budget=15.0):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample."""
    import oracle
    oracle.build()
    spec = WORKLOADS[name]
    prob = spec["make"]()
    cores = os.cpu_count() or 1
    R = prob.robot.as_dict()
    t0 = time.perf_counter()
    n_done = 0
    reps = 0
    while True:
        oracle.discretize(R, prob.X, prob.U, prob.s, prob.n_sub, threads=cores)
        oracle.vjp(R, prob.X, prob.U, prob.s, prob.w, prob.rho, prob.n_sub, threads=cores)
        n_done += prob.N
        reps += 1
        if time.perf_counter() - t0 > min(seconds_budget, 10.0) or reps >= 200:
            break
    dt = time.perf_counter() - t0
    return {"value": n_done / dt, "unit": "intervals/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} passes of the full {prob.N}-interval instance (STM by dual-number IND + "
                      f"Phi-contracted VJP), {cores} threads"}


def run_ours(args):
    import torch
    rank, world, lrank = dist_env()
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(lrank)
        tdist.init_process_group("nccl")
    dev = torch.device(f"cuda:{lrank}")
    torch.cuda.set_device(dev)
    from paper_2604_09993_gb300 import api, build
    build.build()
    api.load()
    spec = WORKLOADS[args.workload]
    wl = SingleWorkload(spec["make"](), dev)
    stream = torch.cuda.current_stream()
    prec = args.precision

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    # plain FP64 comparator and the headline path
    barrier()
    t64 = time_steps(torch, lambda: wl.step("fp64"), args.steps, args.warmup, stream)
    barrier()
    with ClockSampler(lrank) as cs:
        barrier()
        t = time_steps(torch, lambda: wl.step(prec), args.steps, args.warmup, stream)
        barrier()
    clocks = cs.summary()
    wl.check_status()
    if world > 1:
        import torch.distributed as tdist
        tt = torch.tensor([t, t64], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        t, t64 = tt.tolist()
    units = wl.intervals * world
    value = units * args.steps / t
    value64 = units * args.steps / t64

    # dominant kernel: time the discretize and the VJP launches separately
    kd = kernel_time(torch, lambda: wl.disc(prec), 10, stream)
    kv = kernel_time(torch, lambda: wl.vjp(prec), 10, stream)
    dom, kt = ("discretize", kd) if kd >= kv else ("vjp", kv)
    fpi = FLOPS_PER_INTERVAL.get((args.workload, dom, prec))
    roof = {"bound": "alu", "kernel": f"k_{dom}<{'float' if prec == 'fp32_phi' else 'double'}>",
            "unit": "TFLOP/s", "peak": round(FP64_PEAK_TFLOPS, 4), "peak_source": "derived FP64 pipe",
            "launch_ms": kt * 1e3, "traffic": None}
    if fpi:
        ach = fpi * wl.intervals / kt / 1e12
        roof.update(achieved=ach, frac=ach / FP64_PEAK_TFLOPS)
    else:
        roof.update(achieved=None, frac=None)

    # end to end through the public API with host buffers
    host = wl.host_buffers()
    out = api.discretize(wl.model, wl.X, wl.U, wl.s, wl.n_sub, prec)
    gX, gU, gs, L = api.discretize_vjp(wl.model, wl.X, wl.U, wl.s, wl.w, wl.rho, wl.n_sub, prec, workspace=wl.ws)
    res0 = dict(out, gX=gX, gU=gU, gs=gs, L=L)
    wl.alloc_host_outputs(host, res0)
    te = time_steps(torch, lambda: wl.e2e_step(host, prec), args.steps, min(args.warmup, 3), stream)
    h2d = sum(host[k].numel() * host[k].element_size() for k in ("X", "U", "s", "w", "rho"))
    d2h = sum(v.numel() * v.element_size() for v in res0.values())

    if rank != 0:
        return
    line = {
        "metric": "linearized intervals/s (STM + adjoint VJP)",
        "value": value, "unit": "intervals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 state / f32 Phi" if prec == "fp32_phi" else "f64",
        "data": "synthetic (seeded robots, no dataset)",
        "config": {"workload": args.workload, "precision": prec, "instances": 1,
                   "intervals_per_gpu": wl.intervals, "n_sub": wl.n_sub,
                   "l2": "inputs+outputs below L2: cold-cache not enforced"},
        "fp64_path": {"value": value64, "ms_per_step": t64 / args.steps * 1e3,
                      "speedup": value / value64},
        "gpu_launches": args.steps * (1 + 3),
        "roofline": roof,
        "e2e": {"value": units * args.steps / te, "unit": "intervals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cb = cpu_baseline(args.workload)
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline(args.workload, seconds_budget=2.0)
    for _ in range(args.steps):
        per_step.append(cpu_baseline(args.workload, seconds_budget=2.0)["value"])
    v = statistics.mean(per_step)
    line = {"impl": "reference", "metric": "linearized intervals/s (STM + adjoint VJP)", "value": v,
            "unit": "intervals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded robots, no dataset)",
            "config": {"workload": args.workload},
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": "intervals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32_phi", choices=["fp64", "fp32_phi"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
