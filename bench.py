#!/usr/bin/env python3
"""Throughput benchmark of the CI-SCvx discretization/linearization hot path.

One step = one pass of the whole hot path over one batch of synthetic input:
the linearized discretization (A, B-, B+, S, defects, penalty increments) of
every interval of every instance plus the adjoint VJP of
L = sum w.defect + rho.penalty, with inputs resident in HBM.
value = intervals linearized (STM + VJP) per second.

Default workload: 4096 instances of the 7-link chain, N = 400 intervals,
20 RK4 substeps, s ~ U[0.01, 0.05], FP32 Phi with FP64 state (batched plan,
persistent launch).  A batch step is one ciscvx_batch_discretize_and_vjp
call: both outputs from one pass, the interval's FP64 trajectory shared; the
two paths are also timed as separate calls (roofline.separate_*_ms).  The
plain FP64 GPU path runs the same workload as the comparator (`fp64_path`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank processes its own batch
(instances are independent; no collective on the data path) -> weak scaling;
value = total intervals over all ranks / max rank time.
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
METRIC = "linearized intervals/s (STM + adjoint VJP) vs plain FP64 GPU path at stated error"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_BYTES = 126 * 2 ** 20
# impulse-relaxation parameter of the node constraints in the paper-scale leg
NODE_DELTA_PAPER = 1e-3


def _measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


HBM_GBS = _measured_hbm_gbs()

# make(n_inst, seed): rank r of a multi-GPU run uses seed r (its own independent batch)
WORKLOADS = {
    "cheetah7-sweep-4096x400x20": dict(kind="batch", instances=4096,
                                       make=lambda n, seed=0: synth.cheetah_sweep(seed=seed, n_inst=n)),
    "mixed-1024": dict(kind="batch", instances=1024,
                       make=lambda n, seed=0: synth.mixed_batch(seed=seed, n_inst=n)),
    "cheetah7-n50-sub10": dict(kind="single", instances=1,
                               make=lambda n, seed=0: synth.cheetah_n50(seed=seed)),
    "hopper-n10-sub4": dict(kind="single", instances=1,
                            make=lambda n, seed=0: synth.hopper_fp64(seed=seed)),
    "cheetah7-n100-sub10": dict(kind="single", instances=1,
                                make=lambda n, seed=0: synth.cheetah_adjoint(seed=seed)),
}
DEFAULT_WORKLOAD = "cheetah7-sweep-4096x400x20"

# Executed FP64 flops per interval of the FP64 kernels (ncu SASS counters
# 2*DFMA + DADD + DMUL of one launch / intervals of that launch), recorded in
# profiles/; keyed by (robot, n_sub, kernel, precision).  These are the counts
# of the uncapped variant.  The FP32-Phi kernels are not FP64-bound any more
# (their stage values run in float-float on the FP32 pipe): their roofline is
# the instruction issue rate below.  FP64_STATE_FLOPS is the FP64 work per
# interval of the FP64-state formulation of the same fused pass (an earlier
# build of this kernel), kept as a context figure.
FLOPS_PER_INTERVAL = {
    ("cheetah7", 20, "discretize", "fp64"): 126_146,
    ("cheetah7", 20, "vjp", "fp64"): 82_621,
}
FP64_STATE_FLOPS = {("cheetah7", 20, "fused", "fp32_phi"): 30_693}
# Warp-instructions issued per interval (ncu smsp__inst_executed.sum / the
# 102 400 intervals of the capture), keyed by (robot, n_sub, kernel,
# precision, register-cap variant).  The uncapped variant's count is the
# kernel's work; a capped variant executes a few per cent more (spills and
# recomputation).  The fused step with dense outputs is two kernels: the
# fused pass staging compact values, and k_expand_dense widening them.
WARP_INSTR_PER_INTERVAL = {
    ("cheetah7", 20, "fused", "fp32_phi", 0): (1_120_225_652 + 129_843_200) / 102400,
}
# Issue peak: 152 SMs x 4 schedulers x 1 warp-instruction/clk x 2.07 GHz.
ISSUE_PEAK = 152 * 4 * 2.07e9
# DRAM bytes (read + write) per interval of each kernel from the same captures
# (256 instances x 400 intervals; traffic scales with the intervals processed),
# keyed by (robot, n_sub, kernel, precision, register-cap variant).  None when
# the variant the tuner picked was not captured.
DRAM_BYTES_PER_INTERVAL = {
    ("cheetah7", 20, "discretize", "fp64", 0): (407.3e6 + 3762.1e6) / 102400,
    ("cheetah7", 20, "vjp", "fp64", 0): (258.3e6 + 227.4e6) / 102400,
    ("cheetah7", 20, "fused", "fp32_phi", 0): (394.4e6 + 476.3e6 + 171.3e6 + 1595.8e6) / 102400,
}


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while active."""

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

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
        num = lambda v: float(v) if v.replace(".", "", 1).isdigit() else None  # noqa: E731
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
class BatchWorkload:
    """Instances packed for a batch plan; one plan per (precision, output format), autotuned.

    fmt "dense" writes the full A/B-/B+ blocks, "compact" only their structural
    nonzeros (ciscvx_model_pattern order); S, defect, penalty and the VJP are
    the same in both."""

    def __init__(self, spec, n_inst, dev, seed=0):
        import torch
        from paper_2604_09993_gb300 import api
        self.api, self.torch, self.dev = api, torch, dev
        self.batch = spec["make"](n_inst, seed)
        b = self.batch
        self.models = [api.Model(r) for r in b.robots]
        probs = [b.instance(i) for i in range(len(b))]
        self.robot_name = b.robots[0].name if len(b.robots) == 1 else "mixed"
        self.n_sub = int(b.n_subs[0]) if len(set(b.n_subs.tolist())) == 1 else None
        self.intervals = int(b.Ns.sum())
        self.plans = {}
        p0 = self.plan("fp32_phi")
        t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        self.X = t(p0.pack([p.X for p in probs], "X"))
        self.U = t(p0.pack([p.U for p in probs], "U"))
        self.s = t(p0.pack([p.s for p in probs], "s"))
        self.w = t(p0.pack([p.w for p in probs], "defect"))
        self.rho = t(p0.pack([p.rho for p in probs], "penalty"))
        del probs
        self.out, self.gout, self.ws = {}, {}, None

    def plan(self, prec, fmt="dense"):
        if (prec, fmt) not in self.plans:
            b = self.batch
            self.plans[(prec, fmt)] = self.api.BatchPlan(self.models, b.model_idx, b.Ns, b.n_subs,
                                                         precision=prec, out_format=fmt)
        return self.plans[(prec, fmt)]

    def prepare(self, prec, fmt="dense"):
        pl = self.plan(prec, fmt)
        need = pl.vjp_workspace_size()
        if self.ws is None or self.ws.numel() < need:
            self.ws = self.torch.empty(need, dtype=self.torch.uint8, device=self.dev)
        if (prec, fmt) not in self.out:
            self.out[(prec, fmt)] = pl.alloc_outputs(self.dev)
            pl.autotune(self.X, self.U, self.s, out=self.out[(prec, fmt)])
            pl.autotune_fused(self.X, self.U, self.s, self.w, self.rho, workspace=self.ws,
                              out=self.out[(prec, fmt)])

    def free(self, prec, fmt="dense"):
        self.out.pop((prec, fmt), None)
        self.gout.pop((prec, fmt), None)
        self.torch.cuda.empty_cache()

    def disc(self, prec, fmt="dense"):
        self.plan(prec, fmt).discretize(self.X, self.U, self.s, out=self.out[(prec, fmt)])

    def vjp(self, prec, fmt="dense"):
        pl = self.plan(prec, fmt)
        self.gout[(prec, fmt)] = pl.discretize_vjp(self.X, self.U, self.s, self.w, self.rho,
                                                   workspace=self.ws, out=self.gout.get((prec, fmt)))

    def step(self, prec, fmt="dense"):
        """One pass of the hot path: linearization and adjoint VJP of every interval
        (ciscvx_batch_discretize_and_vjp: one shared FP64 trajectory per interval)."""
        key = (prec, fmt)
        _, self.gout[key] = self.plan(prec, fmt).discretize_and_vjp(
            self.X, self.U, self.s, self.w, self.rho, workspace=self.ws, out=self.out[key],
            gout=self.gout.get(key))

    def check_status(self):
        for pl in self.plans.values():
            pl.sync_status()

    def tune(self, prec, fmt="dense"):
        pl = self.plan(prec, fmt)
        return {"discretize": pl.tune(), "fused": pl.tune_fused()}

    # end to end through the public API with host buffers: ciscvx_batch_run_host
    # (chunked, H2D / compute / D2H overlapped on three streams)
    E2E_CHUNKS = 8

    def e2e_setup(self, prec, fmt="dense"):
        torch = self.torch
        self.host_in = {k: getattr(self, k).cpu().pin_memory() for k in ("X", "U", "s", "w", "rho")}
        self.dev_in = {k: torch.empty_like(getattr(self, k)) for k in ("X", "U", "s", "w", "rho")}
        outs = dict(self.out[(prec, fmt)])
        outs.update({k: v for k, v in self.gout[(prec, fmt)].items() if v is not None})
        self.host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in outs.items()}
        h2d = sum(v.numel() * v.element_size() for v in self.host_in.values())
        d2h = sum(v.numel() * v.element_size() for v in self.host_out.values())
        return h2d, d2h

    def e2e_step(self, prec, fmt="dense"):
        h, d = self.host_in, self.dev_in
        ho, g = self.host_out, self.gout[(prec, fmt)]
        host_vjp = {"w": h["w"], "rho": h["rho"], "gX": ho["gX"], "gU": ho["gU"], "gs": ho["gs"], "L": ho["L"]}
        dev_vjp = {"w": d["w"], "rho": d["rho"], "gX": g["gX"], "gU": g["gU"], "gs": g["gs"], "L": g["L"]}
        self.plan(prec, fmt).run_host({k: h[k] for k in ("X", "U", "s")}, ho,
                                      {k: d[k] for k in ("X", "U", "s")}, self.out[(prec, fmt)],
                                      n_chunks=self.E2E_CHUNKS, host_vjp=host_vjp, dev_vjp=dev_vjp,
                                      workspace=self.ws)

    def e2e_free(self):
        self.host_in = self.host_out = self.dev_in = None
        self.torch.cuda.empty_cache()

    # node constraints (impact map + relaxed impulse conditions) at every node
    # of every instance: one ciscvx_node_linearize call per model over its
    # instances' nodes (pre-impact states = the node states, post-impact =
    # a seeded perturbation, impulses and multipliers seeded)
    NODE_DELTA = 1e-3

    def node_setup(self):
        torch, b = self.torch, self.batch
        p0 = self.plan("fp32_phi")
        gen = torch.Generator(device=self.dev)
        gen.manual_seed(1234)
        self.node_jobs = []
        for mi, m in enumerate(self.models):
            inst = np.nonzero(b.model_idx == mi)[0]
            if len(inst) == 0:
                continue
            # the node states of this model's instances, gathered (setup only, not timed)
            idx = np.concatenate([np.arange(p0.offsets[i]["X"], p0.offsets[i]["X"] + (int(b.Ns[i]) + 1) * m.nxt)
                                  for i in inst])
            n = len(idx) // m.nxt
            Xm = self.X[torch.from_numpy(idx).to(self.dev)].view(n, m.nxt).contiguous()
            Xp = (Xm + 0.1 * torch.randn(Xm.shape, generator=gen, device=self.dev, dtype=torch.float64)).contiguous()
            Phi = torch.randn((n, 2 * m.nc), generator=gen, device=self.dev, dtype=torch.float64)
            Gam = torch.rand((n, m.nc), generator=gen, device=self.dev, dtype=torch.float64)
            e = np.full(m.nc, 0.3)
            out = self.api.node_linearize(m, Xp, Xm, Phi, Gam, self.NODE_DELTA, e)
            self.node_jobs.append((m, Xp, Xm, Phi, Gam, e, out))
        return sum(j[1].shape[0] for j in self.node_jobs)

    # SOCP canonicalization (ciscvx_socp_fill) of every instance of the first
    # model that shares its horizon, from the plan's compact linearization
    # (structural nonzeros of A, B-, B+), the node constraints and Psi (all
    # built untimed in setup)
    def socp_setup(self, prec):
        torch, b, api = self.torch, self.batch, self.api
        m = self.models[0]
        N = int(b.Ns[0])
        inst = np.nonzero((b.model_idx == 0) & (b.Ns == N))[0]
        p = self.plan(prec, "compact")
        per = {"X": (N + 1) * m.nxt, "U": (N + 1) * m.nu, "s": N, "A": N * m.nnz_a,
               "B": N * m.nnz_b, "S": N * m.nxt, "defect": N * m.nxt}
        n = len(inst)
        if not np.array_equal(inst, np.arange(n)) or any(
                p.offsets[i][k] != i * v for i in inst for k, v in per.items()):
            return None  # the instances are not a plain concatenation in the plan
        self.prepare(prec, "compact")
        self.disc(prec, "compact")
        out = self.out[(prec, "compact")]
        gen = torch.Generator(device=self.dev)
        gen.manual_seed(99)
        nn = n * (N + 1)
        Xp = self.X[: nn * m.nxt].view(nn, m.nxt)
        Xm = (Xp + 0.05 * torch.randn(Xp.shape, generator=gen, device=self.dev, dtype=torch.float64)).contiguous()
        Phi = torch.randn((nn, 2 * m.nc), generator=gen, device=self.dev, dtype=torch.float64)
        Gam = torch.rand((nn, m.nc), generator=gen, device=self.dev, dtype=torch.float64)
        nd = api.node_linearize(m, Xp, Xm, Phi, Gam, self.NODE_DELTA, np.full(m.nc, 0.3))
        ps = api.psi_linearize(m, Xp, Xm, self.NODE_DELTA, 1e-4)
        # Psi per instance: drop the rows that straddle two instances
        pad = lambda t: torch.cat([t, t[:1]]).view(n, N + 1, *t.shape[1:])[:, :N].contiguous()  # noqa: E731
        psi, dpsi = pad(ps["psi"]), pad(ps["dpsi"])
        del ps
        self.socp = api.Socp(m, N, "node", w_px=2000.0, w_ep=50000.0, w_torque=1.0, s_min=0.005,
                             s_max=0.1, torque_max=np.full(m.nj, 50.0), x_init=np.zeros(6 * m.nb),
                             x_final=np.zeros(6 * m.nb), phi_format="compact")
        self.socp_in = {"Xp": Xp, "Xm": Xm, "U": self.U[: n * per["U"]], "s": self.s[: n * N], "Phi": Phi,
                        "Gam": Gam, "A": out["A"], "Bm": out["Bm"], "Bp": out["Bp"], "S": out["S"],
                        "defect": out["defect"], "g": nd["g"], "Gvm": nd["Gvm"], "Gth": nd["Gth"],
                        "Gphi": nd["Gphi"], "Gpx": nd["Gpx"], "theta": nd["theta"], "dtheta": nd["dtheta"],
                        "psi": psi, "dpsi": dpsi}
        self.socp_n, self.socp_prec = n, prec
        self.socp_out = self.socp.fill(n, self.socp_in, precision=prec)
        d = self.socp.dims
        # algorithmic bytes per instance: every output once, every input element the
        # assembly references once (A and B-/B+ at their structural pattern)
        el = 4 if prec == "fp32_phi" else 8
        nq, nc, nxt = 3 * m.nb, m.nc, m.nxt
        out_b = 8 * (d["nnz_A"] + d["nnz_G"] + 2 * d["n_eq"] + 2 * d["n_ineq"] + d["n_var"])
        in_b = (el * N * (m.nnz_a + 2 * m.nnz_b + nxt) + 8 * N * nxt
                + 8 * (N + 1) * (2 * nxt + m.nu + 3 * nc + nxt + nq * nq + nq * m.nb + nq * 2 * nc
                                 + 8 * nc + 8 * nc * 10)
                + 8 * N * (psi.shape[-1] * 3))
        return {"instances": n, "N": N, "dims": d, "bytes_per_instance": out_b + in_b}

    def socp_step(self):
        self.socp.fill(self.socp_n, self.socp_in, out=self.socp_out, precision=self.socp_prec)

    def socp_free(self):
        self.socp = self.socp_in = self.socp_out = None
        self.torch.cuda.empty_cache()

    def node_step(self):
        for m, Xp, Xm, Phi, Gam, e, out in self.node_jobs:
            self.api.node_linearize(m, Xp, Xm, Phi, Gam, self.NODE_DELTA, e, out=out)

    def node_free(self):
        self.node_jobs = None
        self.torch.cuda.empty_cache()


class SingleWorkload:
    """One instance.  A step is the fused linearization + VJP pass of a
    one-instance batch plan (ciscvx_batch_discretize_and_vjp: the interval's
    trajectory integrated once, one launch plus the per-instance finish); the
    single-instance entry points ciscvx_discretize and ciscvx_discretize_vjp
    are timed as the separate calls."""

    def __init__(self, spec, n_inst, dev, seed=0):
        import torch
        from paper_2604_09993_gb300 import api
        self.api, self.torch, self.dev = api, torch, dev
        prob = spec["make"](1, seed)
        self.model = api.Model(prob.robot)
        t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        self.X, self.U, self.s, self.w, self.rho = (t(prob.X), t(prob.U), t(prob.s), t(prob.w), t(prob.rho))
        self.intervals, self.n_sub, self.robot_name = prob.N, prob.n_sub, prob.robot.name
        self.out, self.gout, self.plans, self.pout, self.pgout = {}, {}, {}, {}, {}
        self.ws = torch.empty(api.workspace_size(self.model, api.OP_VJP, prob.N), dtype=torch.uint8, device=dev)

    def plan(self, prec):
        if prec not in self.plans:
            self.plans[prec] = self.api.BatchPlan([self.model], [0], [self.intervals], [self.n_sub], precision=prec)
        return self.plans[prec]

    def prepare(self, prec):
        if prec not in self.out:
            self.out[prec] = self.api.discretize(self.model, self.X, self.U, self.s, self.n_sub, prec)
            self.vjp(prec)
            pl = self.plan(prec)
            self.pws = self.torch.empty(pl.vjp_workspace_size(), dtype=self.torch.uint8, device=self.dev)
            self.pout[prec] = pl.alloc_outputs(self.dev)
            pl.autotune_fused(self.X, self.U, self.s, self.w, self.rho, workspace=self.pws, out=self.pout[prec])

    def free(self, prec):
        pass

    def disc(self, prec):
        self.api.discretize(self.model, self.X, self.U, self.s, self.n_sub, prec, out=self.out[prec])

    def vjp(self, prec):
        gX, gU, gs, L = self.api.discretize_vjp(self.model, self.X, self.U, self.s, self.w, self.rho,
                                                self.n_sub, prec, workspace=self.ws)
        self.gout[prec] = {"gX": gX, "gU": gU, "gs": gs, "L": L}

    def step(self, prec):
        _, self.pgout[prec] = self.plan(prec).discretize_and_vjp(
            self.X, self.U, self.s, self.w, self.rho, workspace=self.pws, out=self.pout[prec],
            gout=self.pgout.get(prec))

    def check_status(self):
        self.api.sync_status(self.model)
        for pl in self.plans.values():
            pl.sync_status()

    def tune(self, prec):
        return {"fused": self.plan(prec).tune_fused()} if prec in self.plans else None

    def e2e_setup(self, prec):
        torch = self.torch
        self.host_in = {k: getattr(self, k).cpu().pin_memory() for k in ("X", "U", "s", "w", "rho")}
        outs = dict(self.out[prec])
        outs.update(self.gout[prec])
        self.host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in outs.items()}
        return (sum(v.numel() * v.element_size() for v in self.host_in.values()),
                sum(v.numel() * v.element_size() for v in self.host_out.values()))

    def e2e_step(self, prec):
        d = {k: v.to(self.dev, non_blocking=True) for k, v in self.host_in.items()}
        out = self.api.discretize(self.model, d["X"], d["U"], d["s"], self.n_sub, prec)
        gX, gU, gs, L = self.api.discretize_vjp(self.model, d["X"], d["U"], d["s"], d["w"], d["rho"],
                                                self.n_sub, prec, workspace=self.ws)
        res = dict(out, gX=gX, gU=gU, gs=gs, L=L)
        for k, v in self.host_out.items():
            v.copy_(res[k], non_blocking=True)

    def e2e_free(self):
        self.host_in = self.host_out = None


# ---------------------------------------------------------------------------
# timing
# ---------------------------------------------------------------------------
# A buffer larger than L2, written between timed steps when a workload's
# inputs fit in L2 (set by run_ours; None: inputs already exceed L2).
L2_FLUSH = None


def time_steps(torch, fn, steps, warmup, stream, name="timed"):
    """Seconds for `steps` calls of fn after `warmup` calls, CUDA events on the
    launching stream.  With L2_FLUSH set, L2 is flushed before every step,
    outside the timed spans, and the spans are summed.  The whole measurement
    is an NVTX range `name` (host-side marker; profilers can filter on it)."""
    torch.cuda.nvtx.range_push(name)
    try:
        return _time_steps(torch, fn, steps, warmup, stream)
    finally:
        torch.cuda.nvtx.range_pop()


def _time_steps(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if L2_FLUSH is None:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3
    return kernel_time(torch, fn, steps, stream) * steps


def kernel_time(torch, fn, reps, stream):
    """Mean duration of fn's launches with CUDA events on the launching stream."""
    ts = []
    for _ in range(reps):
        if L2_FLUSH is not None:
            L2_FLUSH.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.mean(ts)


def cpu_baseline(name, budget_s=12.0):
    """The FP64 oracle, as it stands, on all host cores over a bounded sample of the workload."""
    import oracle
    oracle.build()
    spec = WORKLOADS[name]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    n_int, n_inst = 0, 0
    if spec["kind"] == "single":
        p = spec["make"](1)
        it = (p for _ in range(100000))
    else:
        b = spec["make"](spec["instances"])
        it = (b.instance(i) for i in range(len(b)))
    for p in it:
        R = p.robot.as_dict()
        oracle.discretize(R, p.X, p.U, p.s, p.n_sub, threads=cores)
        oracle.vjp(R, p.X, p.U, p.s, p.w, p.rho, p.n_sub, threads=cores)
        n_int += p.N
        n_inst += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n_int / dt, "unit": "intervals/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_inst} instance pass(es) of the workload ({n_int} intervals): dual-number "
                      f"IND linearization + Phi-contracted VJP, FP64, {cores} threads"}


def paper_cpu_baseline(p, budget_s=4.0):
    """The oracle on a bounded sample of the paper-dynamics workload (all host cores)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    R = p.robot.as_dict()
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < budget_s and n + 4 * cores <= p.N:
        k = n + 4 * cores
        oracle.discretize(R, p.X[n:k + 1], p.U[n:k + 1], p.s[n:k], p.n_sub, threads=cores)
        n = k
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "intervals/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {n} intervals of the workload: dual-number IND with the dense "
                      f"KKT solve of Eq. (3), FP64, {cores} threads"}


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
    stream = torch.cuda.current_stream()
    global L2_FLUSH

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(vals):
        from paper_2604_09993_gb300 import dist as pdist
        return pdist.max_over_ranks(vals, device=dev)

    def measure_paper():
        """The paper's own model on the 7-link chain (joint reaction forces
        eliminated by Eq. (3), RKF45 substeps, sinusoidal surface): the
        coupled-links path, one instance of args.paper_intervals intervals x
        10 substeps per GPU; linearization and its VJP, FP32-Phi and FP64."""
        global L2_FLUSH
        saved = L2_FLUSH
        if L2_FLUSH is None:  # its inputs fit in L2: flush it before every timed call
            L2_FLUSH = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
        torch.cuda.empty_cache()
        pp = synth.cheetah_paper_sweep(seed=rank, N=args.paper_intervals)
        mp = api.Model(pp.robot)
        t_ = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        Xp, Up, sp = t_(pp.X), t_(pp.U), t_(pp.s)
        paper = {"metric": "linearized intervals/s (STM), and of the reverse-mode adjoint VJP",
                 "unit": "intervals/s",
                 "workload": f"7-link chain, eliminated joint forces, RKF45, sinusoidal surface "
                             f"{synth.TERRAIN_SINE[0]} sin({synth.TERRAIN_SINE[1]:.4f} x), "
                             f"1 x {pp.N} intervals x {pp.n_sub} substeps per GPU",
                 }
        precs = ("fp32_phi", "fp64") if args.paper_precision == "both" else (args.paper_precision,)
        for pr in precs:
            lo, hi = api.discretize_workspace_size(mp, pp.N, pp.n_sub, pr)
            ws = torch.empty(max(lo, min(hi, api.DISCRETIZE_WS_CAP)), dtype=torch.uint8, device=dev)
            out = api.discretize(mp, Xp, Up, sp, pp.n_sub, pr, workspace=ws)
            fn = lambda: api.discretize(mp, Xp, Up, sp, pp.n_sub, pr, out=out, workspace=ws)  # noqa: E731
            barrier()
            tp = time_steps(torch, fn, args.steps, args.warmup, stream, name="paper dynamics: linearization")
            barrier()
            api.sync_status(mp)
            tp, = max_over_ranks([tp])
            paper[pr] = {"value": pp.N * world * args.steps / tp, "ms_per_call": tp / args.steps * 1e3,
                         "chunks": -(-hi // ws.numel()), "workspace_bytes": ws.numel()}
            del out, ws
            torch.cuda.empty_cache()
            # the VJP of the same workload (reverse-mode adjoint of the coupled path)
            wv = torch.randn((pp.N, mp.nxt), dtype=torch.float64, device=dev)
            rv = torch.full((pp.N, mp.nc), 10.0, dtype=torch.float64, device=dev)
            lo, hi = api.discretize_workspace_size(mp, pp.N, pp.n_sub, pr, api.OP_VJP)
            ws = torch.empty(max(lo, min(hi, api.DISCRETIZE_WS_CAP)), dtype=torch.uint8, device=dev)
            fv = lambda: api.discretize_vjp(mp, Xp, Up, sp, wv, rv, pp.n_sub, pr, workspace=ws)  # noqa: E731
            barrier()
            tv = time_steps(torch, fv, max(1, args.steps // 2), args.warmup, stream, name="paper dynamics: VJP")
            barrier()
            api.sync_status(mp)
            tv, = max_over_ranks([tv])
            paper[pr]["vjp"] = {"value": pp.N * world * max(1, args.steps // 2) / tv,
                                "ms_per_call": tv / max(1, args.steps // 2) * 1e3}
            del ws
            torch.cuda.empty_cache()
            # linearization + VJP in one call (one-instance plan): one nominal pass
            # per chunk feeds both the tangent kernel and the adjoint
            pl = api.BatchPlan([mp], [0], [pp.N], [pp.n_sub], precision=pr)
            wsb = torch.empty(max(pl.vjp_workspace_size(), api.DISCRETIZE_WS_CAP), dtype=torch.uint8, device=dev)
            ob = pl.alloc_outputs(dev)
            _, gb = pl.discretize_and_vjp(Xp.reshape(-1), Up.reshape(-1), sp, wv.reshape(-1), rv.reshape(-1),
                                          workspace=wsb, out=ob)
            fb = lambda: pl.discretize_and_vjp(Xp.reshape(-1), Up.reshape(-1), sp, wv.reshape(-1),  # noqa: E731
                                               rv.reshape(-1), workspace=wsb, out=ob, gout=gb)
            barrier()
            tb = time_steps(torch, fb, max(1, args.steps // 2), args.warmup, stream,
                            name="paper dynamics: linearization + VJP")
            barrier()
            pl.sync_status()
            tb, = max_over_ranks([tb])
            paper[pr]["linearization_and_vjp"] = {
                "value": pp.N * world * max(1, args.steps // 2) / tb, "ms_per_call": tb / max(1, args.steps // 2) * 1e3,
                "what": "ciscvx_batch_discretize_and_vjp of a one-instance plan (one nominal pass for both)"}
            if pr == "fp32_phi" and not args.no_e2e:
                # end to end through the public API: pinned host inputs copied in,
                # linearization and VJP, every output copied back
                hin = {k: v.reshape(-1).cpu().pin_memory()
                       for k, v in (("X", Xp), ("U", Up), ("s", sp), ("w", wv), ("rho", rv))}
                din = {k: torch.empty_like(v, device=dev) for k, v in hin.items()}
                res = {}

                def e2e_step():
                    for k, v in hin.items():
                        din[k].copy_(v, non_blocking=True)
                    o, g = pl.discretize_and_vjp(din["X"], din["U"], din["s"], din["w"], din["rho"], workspace=wsb,
                                                 out=ob, gout=gb)
                    if "host" not in res:
                        res["host"] = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                                       for k, v in list(o.items()) + list(g.items())}
                    for k, v in list(o.items()) + list(g.items()):
                        res["host"][k].copy_(v, non_blocking=True)

                e2e_step()
                torch.cuda.synchronize()
                te = time_steps(torch, e2e_step, max(1, args.steps // 2), 1, stream, name="paper dynamics: end to end")
                te, = max_over_ranks([te])
                h2d = sum(v.numel() * v.element_size() for v in hin.values())
                d2h = sum(v.numel() * v.element_size() for v in res["host"].values())
                paper[pr]["e2e"] = {"value": pp.N * world * max(1, args.steps // 2) / te, "unit": "intervals/s",
                                    "what": "linearization + VJP per interval, host buffers",
                                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
                del hin, din, res
            del wsb, ob, gb, pl, wv, rv
            torch.cuda.empty_cache()
        del Xp, Up, sp, mp
        if world == 1 and not args.no_cpu_baseline:
            paper["cpu_baseline"] = paper_cpu_baseline(pp)

        L2_FLUSH = saved
        return paper

    def measure_psi(robot, n_iv):
        """Psi^{delta,eps} and its Jacobian (FP64) on n_iv intervals of seeded node states."""
        rx = synth.with_cross_states(robot)
        mp = api.Model(rx)
        npsi, ny = api.psi_rows(mp), mp.ny
        gen = torch.Generator(device=dev)
        gen.manual_seed(4321)
        Xp = torch.rand((n_iv + 1, mp.nxt), generator=gen, device=dev, dtype=torch.float64)
        Xm = torch.rand((n_iv + 1, mp.nxt), generator=gen, device=dev, dtype=torch.float64)
        po = api.psi_linearize(mp, Xp, Xm, 1e-2, 1e-4)
        barrier()
        tp = time_steps(torch, lambda: api.psi_linearize(mp, Xp, Xm, 1e-2, 1e-4, out=po), args.steps,
                        args.warmup, stream, name="Psi")
        barrier()
        api.sync_status(mp)
        tp, = max_over_ranks([tp])
        # algorithmic bytes per interval: y+ and y- read, Psi and its Jacobian written
        bpi = 8 * (2 * ny + npsi * (1 + ny))
        out = {"metric": "linearized intervals/s (Psi^{delta,eps}, Eq. (12) auxiliary state, FP64)",
               "value": n_iv * world * args.steps / tp, "unit": "intervals/s",
               "intervals_per_gpu": n_iv, "robot": rx.name, "n_psi": npsi, "n_y": ny,
               "ms_per_call": tp / args.steps * 1e3, "bytes_per_interval": bpi,
               "achieved_gbs": bpi * n_iv * args.steps / tp / 1e9}
        out["hbm_frac_of_measured"] = out["achieved_gbs"] / HBM_GBS if HBM_GBS else None
        del Xp, Xm, po, mp
        torch.cuda.empty_cache()
        return out

    if args.psi_only:
        rng = np.random.default_rng(rank)
        psi = measure_psi(synth.cheetah7(rng), args.psi_intervals)
        if rank == 0:
            print(json.dumps({
                "metric": psi["metric"], "value": psi["value"], "unit": "intervals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": psi["ms_per_call"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded node states)",
                "config": {"workload": f"Psi, 7-link chain with the Eq. (12) state, {args.psi_intervals} intervals"},
                "psi": psi}))
        return

    def measure_paper_scale():
        """One SCP iteration's transcription at the sizes of the paper's monoped
        scenario (15 nodes, 10 steps per interval; joint reaction forces
        eliminated, RKF45, the full Eq. (12) state): the linearization
        (ciscvx_discretize, coupled path), the node constraints at the 15
        nodes, Psi^{delta,eps} between them and the canonicalization into
        the SOCP (ciscvx_socp_fill), each timed alone and all four as one
        step, per precision; L2 flushed before every timed call."""
        global L2_FLUSH
        if L2_FLUSH is None:
            L2_FLUSH = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
        pp = synth.monoped_paper(seed=rank)
        m = api.Model(pp.robot)
        N = pp.N
        t_ = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        X, U, s = t_(pp.X), t_(pp.U), t_(pp.s)
        gen = torch.Generator(device=dev)
        gen.manual_seed(77)
        Xm = (X + 0.05 * torch.randn(X.shape, generator=gen, device=dev, dtype=torch.float64)).contiguous()
        Phi = torch.randn((N + 1, 2 * m.nc), generator=gen, device=dev, dtype=torch.float64)
        Gam = torch.rand((N + 1, m.nc), generator=gen, device=dev, dtype=torch.float64)
        rest = np.full(m.nc, 0.3)
        socp = api.Socp(m, N, "node", w_px=2000.0, w_ep=50000.0, w_torque=1.0, s_min=0.005, s_max=0.1,
                        torque_max=np.full(m.nj, 50.0), x_init=np.zeros(6 * m.nb), x_final=np.zeros(6 * m.nb),
                        phi_format="dense")
        res = {"metric": "SCP-iteration transcription latency: linearization + node constraints + Psi + SOCP "
                         "canonicalization, one instance",
               "unit": "ms", "higher_is_better": False,
               "workload": f"2-link monoped, eliminated joint forces, RKF45, flat ground, Eq. (12) state, "
                           f"{N + 1} nodes x {pp.n_sub} substeps",
               "dims": dict(socp.dims), "paper": "about 50 ms per SCP iteration for the whole iteration "
                                                  "(transcription, canonicalization and the QOCO solve; "
                                                  "hardware not stated)"}
        for pr in ("fp64", "fp32_phi"):
            lo, hi = api.discretize_workspace_size(m, N, pp.n_sub, pr)
            ws = torch.empty(max(lo, hi), dtype=torch.uint8, device=dev)
            out = api.discretize(m, X, U, s, pp.n_sub, pr, workspace=ws)
            nd = api.node_linearize(m, X, Xm, Phi, Gam, NODE_DELTA_PAPER, rest)
            ps = api.psi_linearize(m, X, Xm, NODE_DELTA_PAPER, 1e-4)
            inp = {"Xp": X, "Xm": Xm, "U": U, "s": s, "Phi": Phi, "Gam": Gam, "A": out["A"], "Bm": out["Bm"],
                   "Bp": out["Bp"], "S": out["S"], "defect": out["defect"], "g": nd["g"], "Gvm": nd["Gvm"],
                   "Gth": nd["Gth"], "Gphi": nd["Gphi"], "Gpx": nd["Gpx"], "theta": nd["theta"],
                   "dtheta": nd["dtheta"], "psi": ps["psi"], "dpsi": ps["dpsi"]}
            so = socp.fill(1, inp, precision=pr)
            parts = {
                "linearization": lambda: api.discretize(m, X, U, s, pp.n_sub, pr, out=out, workspace=ws),
                "node_constraints": lambda: api.node_linearize(m, X, Xm, Phi, Gam, NODE_DELTA_PAPER, rest,
                                                               out=nd),
                "psi": lambda: api.psi_linearize(m, X, Xm, NODE_DELTA_PAPER, 1e-4, out=ps),
                "socp_fill": lambda: socp.fill(1, inp, out=so, precision=pr),
            }

            def whole():
                for f in parts.values():
                    f()

            r = {k: time_steps(torch, f, args.steps, args.warmup, stream, name=f"paper scale: {k}") /
                 args.steps * 1e3 for k, f in parts.items()}
            r["iteration"] = time_steps(torch, whole, args.steps, args.warmup, stream,
                                        name="paper scale: iteration") / args.steps * 1e3
            api.sync_status(m)
            res[pr] = r
        return res

    if args.paper_scale:
        ps_res = measure_paper_scale()
        if rank == 0:
            f64 = ps_res["fp64"]["iteration"]
            print(json.dumps({
                "metric": ps_res["metric"], "value": f64, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": f64, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded robot)",
                "config": {"workload": ps_res["workload"], "l2": "L2 flushed before every timed call"},
                "paper_scale": ps_res}))
        return

    if args.paper_only:
        paper = measure_paper()
        if rank == 0:
            f32 = paper.get("fp32_phi") or paper["fp64"]
            print(json.dumps({
                "metric": paper["metric"], "value": f32["value"], "unit": "intervals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": f32["ms_per_call"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 state + f32 Phi", "data": "synthetic (seeded robot)",
                "config": {"workload": paper["workload"], "l2": "L2 flushed before every timed call"},
                "paper_dynamics": paper}))
        return

    spec = WORKLOADS[args.workload]
    n_inst = args.instances or spec["instances"]
    wl = (BatchWorkload if spec["kind"] == "batch" else SingleWorkload)(spec, n_inst, dev, seed=rank)
    prec = args.precision
    in_bytes = sum(getattr(wl, k).numel() * 8 for k in ("X", "U", "s", "w", "rho"))
    if in_bytes <= L2_BYTES:
        L2_FLUSH = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    # headline path
    wl.prepare(prec)
    wl.step(prec)
    barrier()
    with ClockSampler(lrank) as cs:
        barrier()
        t = time_steps(torch, lambda: wl.step(prec), args.steps, args.warmup, stream, name="headline step")
        barrier()
    clocks = cs.summary()
    # the linearization and the VJP as separate calls (each path on its own)
    kd = kernel_time(torch, lambda: wl.disc(prec), 5, stream)
    kv = kernel_time(torch, lambda: wl.vjp(prec), 5, stream)
    # batch step: one fused launch (+ the per-instance finish) does both
    kf = kernel_time(torch, lambda: wl.step(prec), 5, stream)
    wl.check_status()
    t, kd, kv = max_over_ranks([t, kd, kv])
    if kf is not None:
        kf, = max_over_ranks([kf])
    units = wl.intervals * world
    value = units * args.steps / t

    if kf is not None:
        dom, kt, kname = "fused", kf, "k_batch_disc_vjp"
    else:
        dom, kt = ("discretize", kd) if kd >= kv else ("vjp", kv)
        kname = {"discretize": "k_discretize", "vjp": "k_vjp"}[dom]
    tune = wl.tune(prec)
    occ = tune[dom]["occupancy"] if tune and dom in tune else 0
    bpi = DRAM_BYTES_PER_INTERVAL.get((wl.robot_name, wl.n_sub, dom, prec, occ))
    kprec = "float" if prec == "fp32_phi" else "double"
    wpi = WARP_INSTR_PER_INTERVAL.get((wl.robot_name, wl.n_sub, dom, prec, 0))
    fpi = FLOPS_PER_INTERVAL.get((wl.robot_name, wl.n_sub, dom, prec))
    if wpi:
        # instruction issue bound: the FP32-Phi kernels run their stage values in
        # float-float on the FP32 pipe; FP64 pipe, FP32 pipe and DRAM all below it
        ach = wpi * wl.intervals / kt
        kdesc = f"{kname}<{kprec}>"
        if dom == "fused" and spec["kind"] == "batch":
            kdesc += f" (compact values staged) + k_expand_dense<{kprec}>"
        roof = {"bound": "alu", "kernel": kdesc, "unit": "G warp-instructions/s",
                "peak": round(ISSUE_PEAK / 1e9, 1),
                "peak_source": "derived issue rate: 152 SMs x 4 schedulers x 1 instr/clk x 2.07 GHz",
                "achieved": ach / 1e9, "frac": ach / ISSUE_PEAK,
                "work_per_interval": round(wpi),
                "work_source": "ncu smsp__inst_executed.sum of the step's kernels, uncapped variant"}
        f64 = FP64_STATE_FLOPS.get((wl.robot_name, wl.n_sub, dom, prec))
        if f64:
            roof["fp64_equivalent"] = {
                "flops_per_interval": f64, "tflops": f64 * wl.intervals / kt / 1e12,
                "frac_of_fp64_peak": f64 * wl.intervals / kt / 1e12 / FP64_PEAK_TFLOPS,
                "note": "FP64 work of the FP64-state formulation of this pass, per second of this kernel"}
    elif fpi:
        ach = fpi * wl.intervals / kt / 1e12
        roof = {"bound": "alu", "kernel": f"{kname}<{kprec}>", "unit": "TFLOP/s",
                "peak": round(FP64_PEAK_TFLOPS, 4), "peak_source": "derived FP64 pipe",
                "achieved": ach, "frac": ach / FP64_PEAK_TFLOPS}
    else:
        roof = {"bound": "alu", "kernel": f"{kname}<{kprec}>", "unit": None, "peak": None,
                "achieved": None, "frac": None}
    roof.update({"launch_ms": kt * 1e3, "separate_discretize_ms": kd * 1e3, "separate_vjp_ms": kv * 1e3,
                 "occupancy_variant": occ,
                 "traffic": None if bpi is None else bpi * wl.intervals,
                 "traffic_source": None if bpi is None else "ncu dram bytes of a 102400-interval launch, scaled"})

    # end to end through the public API with host (pinned) buffers
    def measure_e2e(fmt):
        h2d, d2h = wl.e2e_setup(prec, fmt) if fmt != "dense" else wl.e2e_setup(prec)
        ke = max(1, args.steps // 2)
        step = (lambda: wl.e2e_step(prec, fmt)) if fmt != "dense" else (lambda: wl.e2e_step(prec))
        te = time_steps(torch, step, ke, 1, stream, name="end to end")
        te, = max_over_ranks([te])
        wl.e2e_free()
        return {"value": units * ke / te, "unit": "intervals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h}

    e2e = None if args.no_e2e else measure_e2e("dense")

    # the same step with compact outputs (structural nonzeros of A, B-, B+ only)
    compact = None
    if spec["kind"] == "batch" and not args.no_compact:
        wl.free(prec)
        wl.prepare(prec, "compact")
        wl.step(prec, "compact")
        barrier()
        tc = time_steps(torch, lambda: wl.step(prec, "compact"), args.steps, args.warmup, stream, name="compact outputs")
        barrier()
        kdc = kernel_time(torch, lambda: wl.disc(prec, "compact"), 5, stream)
        wl.check_status()
        tc, kdc = max_over_ranks([tc, kdc])
        pc = wl.plan(prec, "compact")
        compact = {"value": units * args.steps / tc, "ms_per_step": tc / args.steps * 1e3,
                   "discretize_ms": kdc * 1e3,
                   "output_bytes_per_interval": sum(
                       v.numel() * v.element_size() for v in wl.out[(prec, "compact")].values()) / wl.intervals,
                   "tune": pc.tune(),
                   "e2e": None if args.no_e2e else measure_e2e("compact")}
        wl.free(prec, "compact")

    # plain FP64 GPU path (comparator); after the headline, its end-to-end run
    # and the compact-output leg, so that those see the device as a process
    # running only the FP32-Phi path does (the FP64 leg's tens of GB of
    # allocations, once freed, left the end-to-end copies ~20 % slower)
    t64 = kd64 = None
    if not args.no_fp64 and prec != "fp64":
        wl.prepare("fp64")
        barrier()
        t64 = time_steps(torch, lambda: wl.step("fp64"), args.steps, args.warmup, stream, name="FP64 comparator step")
        barrier()
        kd64 = kernel_time(torch, lambda: wl.disc("fp64"), 3, stream)
        t64, kd64 = max_over_ranks([t64, kd64])
        wl.free("fp64")

    # node constraints: every node of every instance, one call per model
    nodes = None
    if spec["kind"] == "batch" and not args.no_nodes:
        wl.free(prec)
        n_nodes = wl.node_setup()
        barrier()
        tn = time_steps(torch, wl.node_step, args.steps, args.warmup, stream, name="node constraints")
        barrier()
        wl.check_status()
        tn, = max_over_ranks([tn])
        nodes = {"metric": "linearized nodes/s (impact map + relaxed impulse conditions, FP64)",
                 "value": n_nodes * world * args.steps / tn, "unit": "nodes/s",
                 "nodes_per_gpu": n_nodes, "ms_per_call": tn / args.steps * 1e3}
        wl.node_free()

    # Psi^{delta,eps} (Eq. (17c)) with the Eq. (12) auxiliary state on as many
    # intervals as the batch holds, as one trajectory of seeded node states
    psi = None
    if spec["kind"] == "batch" and not args.no_nodes:
        wl.free(prec)
        psi = measure_psi(wl.batch.robots[0], wl.intervals)

    # the SOCP canonicalization of the batch's instances (one shape)
    socp = None
    if spec["kind"] == "batch" and not args.no_socp:
        wl.free(prec)
        info = wl.socp_setup(prec)
        if info is not None:
            barrier()
            tq = time_steps(torch, wl.socp_step, args.steps, args.warmup, stream, name="SOCP canonicalization")
            barrier()
            wl.check_status()
            tq, = max_over_ranks([tq])
            n_iv = info["instances"] * info["N"]
            gbs = info["bytes_per_instance"] * info["instances"] * args.steps / tq / 1e9
            socp = {"metric": "canonicalized intervals/s (SCP subproblem as a CSC SOCP, FP64 values)",
                    "value": n_iv * world * args.steps / tq, "unit": "intervals/s",
                    "instances_per_gpu": info["instances"], "N": info["N"],
                    "ms_per_call": tq / args.steps * 1e3, "dims": info["dims"],
                    "bytes_per_instance": info["bytes_per_instance"], "achieved_gbs": gbs,
                    "hbm_frac_of_measured": gbs / HBM_GBS if HBM_GBS else None,
                    "phi_inputs": prec + ", compact (structural nonzeros)"}
        wl.socp_free()
        wl.free(prec, "compact")

    # the linearization of the same batch with the full Eq. (12) auxiliary state
    # (four cross-complementarity states + one path-penalty state per contact)
    cross = None
    if spec["kind"] == "batch" and args.cross:
        import dataclasses
        wl.free(prec)
        b = wl.batch
        bx = dataclasses.replace(b, robots=[synth.with_cross_states(r) for r in b.robots])
        mx = [api.Model(r) for r in bx.robots]
        px = api.BatchPlan(mx, bx.model_idx, bx.Ns, bx.n_subs, precision=prec)
        probs = (bx.instance(i) for i in range(len(bx)))
        Xs, Us, ss, ws_, rs_ = [], [], [], [], []
        for pr in probs:
            Xs.append(pr.X); Us.append(pr.U); ss.append(pr.s); ws_.append(pr.w); rs_.append(pr.rho)
        t_ = lambda a: torch.tensor(a, device=dev)  # noqa: E731
        Xx, Ux, sx = t_(px.pack(Xs, "X")), t_(px.pack(Us, "U")), t_(px.pack(ss, "s"))
        wx, rx = t_(px.pack(ws_, "defect")), t_(px.pack(rs_, "penalty"))
        del Xs, Us, ss, ws_, rs_
        ox = px.alloc_outputs(dev)
        px.autotune(Xx, Ux, sx, out=ox)
        barrier()
        tx = time_steps(torch, lambda: px.discretize(Xx, Ux, sx, out=ox), args.steps, args.warmup, stream, name="Eq. (12) model")
        barrier()
        px.sync_status()
        tx, = max_over_ranks([tx])
        cross = {"metric": "linearized intervals/s (STM), and of the reverse-mode adjoint VJP",
                 "value": units * args.steps / tx, "unit": "intervals/s",
                 "ms_per_step": tx / args.steps * 1e3, "n_y": mx[0].ny, "tune": px.tune()}
        del ox
        # the adjoint VJP of the same batch (per-link kernel with the CROSS foot links)
        wsx = torch.empty(px.vjp_workspace_size(), dtype=torch.uint8, device=dev)
        gx = px.discretize_vjp(Xx, Ux, sx, wx, rx, workspace=wsx)
        barrier()
        tv = time_steps(torch, lambda: px.discretize_vjp(Xx, Ux, sx, wx, rx, workspace=wsx, out=gx),
                        args.steps, args.warmup, stream, name="Eq. (12) model, VJP")
        barrier()
        px.sync_status()
        tv, = max_over_ranks([tv])
        cross["vjp"] = {"value": units * args.steps / tv, "ms_per_step": tv / args.steps * 1e3,
                        "workspace_bytes": px.vjp_workspace_size()}
        # both in one pass (ciscvx_batch_discretize_and_vjp: one trajectory per interval)
        ox = px.alloc_outputs(dev)
        px.autotune_fused(Xx, Ux, sx, wx, rx, workspace=wsx, out=ox)
        _, gx = px.discretize_and_vjp(Xx, Ux, sx, wx, rx, workspace=wsx, out=ox, gout=gx)
        barrier()
        tb = time_steps(torch, lambda: px.discretize_and_vjp(Xx, Ux, sx, wx, rx, workspace=wsx, out=ox, gout=gx),
                        args.steps, args.warmup, stream, name="Eq. (12) model, linearization + VJP")
        barrier()
        px.sync_status()
        tb, = max_over_ranks([tb])
        cross["linearization_and_vjp"] = {"value": units * args.steps / tb, "ms_per_step": tb / args.steps * 1e3,
                                          "tune": px.tune_fused()}
        del gx, wsx, wx, rx, ox, px
        torch.cuda.empty_cache()
        # the same with compact outputs (the packing of X, U, s does not depend on the format)
        pxc = api.BatchPlan(mx, bx.model_idx, bx.Ns, bx.n_subs, precision=prec, out_format="compact")
        oxc = pxc.alloc_outputs(dev)
        pxc.autotune(Xx, Ux, sx, out=oxc)
        barrier()
        txc = time_steps(torch, lambda: pxc.discretize(Xx, Ux, sx, out=oxc), args.steps, args.warmup, stream,
                         name="Eq. (12) model, compact")
        barrier()
        pxc.sync_status()
        txc, = max_over_ranks([txc])
        cross["compact"] = {"value": units * args.steps / txc, "unit": "intervals/s",
                            "ms_per_step": txc / args.steps * 1e3, "tune": pxc.tune()}
        del oxc, Xx, Ux, sx, pxc
        torch.cuda.empty_cache()


    # the paper's own model on the 7-link chain (joint reaction forces
    # eliminated by Eq. (3), RKF45, sinusoidal surface): the coupled-links path
    paper = None
    if not args.no_paper:
        if spec["kind"] == "batch":
            wl.free(prec)
        paper = measure_paper()

    if rank != 0:
        return
    fp64 = None if t64 is None else {
        "value": units * args.steps / t64, "unit": "intervals/s", "ms_per_step": t64 / args.steps * 1e3,
        "discretize_ms": kd64 * 1e3, "headline_speedup": t64 / t,
        "stated_error": "FP64 path: every block rel <= 1e-10; headline: Phi blocks rel <= 1e-4, "
                        "defect/penalty/state rel <= 1e-10 (block-normwise, vs the FP64 oracle)"}
    line = {
        "metric": METRIC,
        "value": value, "unit": "intervals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 state + f32 Phi/adjoint" if prec == "fp32_phi" else "f64",
        "data": "synthetic (seeded robots; no dataset)",
        "config": {"workload": args.workload, "precision": prec, "instances_per_gpu": n_inst,
                   "intervals_per_gpu": wl.intervals, "n_sub": wl.n_sub,
                   "l2": ("inputs larger than L2" if L2_FLUSH is None
                          else "L2 flushed before every timed step (buffer of twice the L2 written)"),
                   "tune": wl.tune(prec)},
        # launches of this library per timed step: the fused discretize+VJP pass + the finish
        "gpu_launches": args.steps * 2,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        # secondary legs (other rows of the hot path on the same box)
        "compact_outputs": compact,
        "node_constraints": nodes,
        "psi": psi,
        "socp": socp,
        "aux_cross_model": cross,
        "paper_dynamics": paper,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    # last, so that it stays in any tail of this line: the metric's comparator,
    # the plain FP64 GPU path on the same workload and GPU
    line["fp64_path"] = fp64
    print(json.dumps(line))


def run_reference(args):
    """The oracle as the reference arm, timed on the host cores (bounded sample per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(args.workload, budget_s=1.0)
    vals = [cpu_baseline(args.workload, budget_s=3.0) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "intervals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded robots; no dataset)", "config": {"workload": args.workload},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "intervals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--instances", type=int, default=0, help="override the workload's instance count")
    ap.add_argument("--precision", default="fp32_phi", choices=["fp64", "fp32_phi"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparator")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compact", action="store_true", help="skip the compact-output measurement")
    ap.add_argument("--no-nodes", action="store_true", help="skip the node-constraint measurement")
    ap.add_argument("--no-socp", action="store_true", help="skip the SOCP canonicalization measurement")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the paper-dynamics (coupled links) measurement")
    ap.add_argument("--paper-only", action="store_true",
                    help="run only the paper-dynamics measurement (its own JSON line)")
    ap.add_argument("--paper-intervals", type=int, default=65536,
                    help="intervals of the paper-dynamics instance")
    ap.add_argument("--paper-precision", default="both", choices=["both", "fp32_phi", "fp64"])
    ap.add_argument("--paper-scale", action="store_true",
                    help="run only the per-SCP-iteration latency at the paper's monoped scale (own JSON line)")
    ap.add_argument("--psi-only", action="store_true",
                    help="run only the Psi^{delta,eps} measurement (its own JSON line)")
    ap.add_argument("--psi-intervals", type=int, default=1 << 20, help="intervals of the Psi-only measurement")
    ap.add_argument("--cross", action="store_true",
                    help="also time the linearization with the full Eq. (12) auxiliary state")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
