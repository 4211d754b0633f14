#!/usr/bin/env python3
"""Time-to-solution and SpMV HBM bandwidth of the reachability solver on one GB300.

Workload: the paper-style dense random chain -- n = 32768 states, each entry present
with probability 10% (about 107M stored transitions), U(0,1] weights normalised per
row, 1% goal states.  Without absorbing sinks every state reaches GS almost surely,
so the S=0/S=1 partition leaves nothing to solve (x = 1).  The step therefore solves
the system of §2.3 as the paper writes it, with S=1 = GS (PROB0_ONLY): 32440 unknowns,
about 105M entries, exact solution x* = 1 (certified by the S=0/S=1 partition).

One step = ingest + validate P (a copy from HBM-resident inputs), the partition and
extraction (§2.2-2.3), a certified bound of ||(I - A)^-1|| (a BiCGStab solve of
(I - A) tau = 1), then FP64 Jacobi, mixed-precision Jacobi (FP32 sweeps, FP64
refinement every 16 sweeps) and FP64 BiCGStab, each run until its max error against
x* is at most 1e-9; each reports its certified error bound.  The matrix is 1.3 GB, far larger than the 129 MB L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle instead.
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

METRIC = "time-to-solution @1e-6/1e-9 err & SpMV HBM GB/s vs FP64 plain Jacobi"
WORKLOAD = ("dense random chain n=32768, 10% density (~107M nnz), U(0,1] normalised, 1% goals; "
            "system of Sec. 2.3 with S=1=GS (32440 unknowns); FP64 Jacobi + mixed Jacobi + "
            "BiCGStab, each to max error <= 1e-9")
TARGET_ERR = 1e-9
# stopping thresholds that give max error <= 1e-9 on this system (contraction ~0.99)
EPS = {"jacobi": 5e-12, "mixed": 5e-12, "bicgstab": 5e-12}
K_REFINE = 16
# DRAM bytes (read + write) per launch of the current kernels on this workload, from one
# ncu capture each; set back to None whenever the kernel changes, until it is captured again.
NCU_TRAFFIC_BYTES = 1271578368 + 3304448
NCU_TRAFFIC_SWEEP32_BYTES = 633112320 + 2868224
# FP64 peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA per clock (ncu's
# roofline reports 4 FP64 flop/clk/SM) x 2 flop x 2.07 GHz; matches the 1.25 TFLOP/s nominal.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_KIND = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def make_chain():
    from paper_1210_6412_gb300 import synth
    return synth.dense_random_chain(n=32768, density=0.10, goal_frac=0.01, sink_frac=0.0)


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def cpu_info():
    """Host cores and CPU model (for the CPU baseline's record)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().startswith("Model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


class CpuOracleStep:
    """One time-to-solution of the oracle on the host cores, split into `pieces` parts.

    The oracle's partition (PROB0_ONLY) and extraction of the full matrix (numpy, as it
    stands), then its FP64 Jacobi and BiCGStab loops in their C build on `threads` cores,
    each to the benchmark's stopping rule.  The oracle has no mixed-precision form, so its
    step is precompute + Jacobi + BiCGStab.  Piece 0 also runs the precompute; pieces
    0..pieces-2 run `chunk` Jacobi sweeps each (resuming from the previous iterate); the
    last piece finishes Jacobi and runs BiCGStab.  Every part is measured, nothing is
    extrapolated: the pieces' times add up to one full time-to-solution.
    """

    def __init__(self, chain, threads=0, pieces=1, expect_sweeps=2150):
        from oracle import c_oracle
        self.co = c_oracle
        self.chain = chain
        self.threads = c_oracle.set_threads(threads)
        self.pieces = max(1, int(pieces))
        self.chunk = -(-int(expect_sweeps) // self.pieces)
        self.t = {"precompute": 0.0, "jacobi": 0.0, "bicgstab": 0.0}
        self.sweeps = 0
        self.done = False
        self.x = None

    def piece(self, i):
        import oracle as O
        c = self.chain
        if i == 0:
            t0 = time.perf_counter()
            cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, O.PROB0_ONLY)
            q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
            self.m, self.b = O.system_matrix(a), b
            self.t["precompute"] += time.perf_counter() - t0
        last = i == self.pieces - 1
        if not self.done:
            t0 = time.perf_counter()
            budget = 10_000_000 if last else self.chunk
            self.x, it, d, ok = self.co.jacobi(self.m, self.b, EPS["jacobi"], budget, x0=self.x)
            self.t["jacobi"] += time.perf_counter() - t0
            self.sweeps += it
            self.done = ok
        if last:
            t0 = time.perf_counter()
            self.xb, self.bi_iters, _, st = self.co.bicgstab(self.m, self.b, EPS["bicgstab"], 200)
            self.t["bicgstab"] += time.perf_counter() - t0

    def run(self):
        for i in range(self.pieces):
            self.piece(i)
        return self

    def total_ms(self):
        return 1e3 * sum(self.t.values())

    def record(self):
        return {"value": self.total_ms(), "unit": "ms", "cores": self.threads, "kind": "oracle",
                **cpu_info(),
                "parts_ms": {k: 1e3 * v for k, v in self.t.items()},
                "jacobi_sweeps": self.sweeps,
                "bicgstab_iters": self.bi_iters,
                "max_err": {"jacobi": float(np.max(np.abs(self.x - 1.0))),
                            "bicgstab": float(np.max(np.abs(self.xb - 1.0)))},
                "sample": ("the whole workload, measured: the oracle's partition + extraction (numpy), "
                           f"then its FP64 Jacobi ({self.sweeps} sweeps) and BiCGStab ({self.bi_iters} "
                           f"iterations) loops in C on {self.threads} host threads, each to eps = "
                           f"{EPS['jacobi']:g}; the oracle has no mixed-precision form")}


def cpu_single_core_estimate(chain_m, b, sweeps_total, sweeps=5):
    """The paper's sequential-C analogue: a few Jacobi sweeps of the C loops on one thread,
    scaled by the full sweep count (an extrapolation, labelled as such)."""
    from oracle import c_oracle
    c_oracle.set_threads(1)
    t0 = time.perf_counter()
    c_oracle.jacobi(chain_m, b, 0.0, sweeps)
    per = (time.perf_counter() - t0) / sweeps
    c_oracle.set_threads(0)
    return {"value": per * sweeps_total * 1e3, "unit": "ms", "cores": 1, "kind": "extrapolated",
            "sample": f"{sweeps} Jacobi sweeps of the C loops on one thread ({per * 1e3:.1f} ms each) "
                      f"x {sweeps_total} sweeps; Jacobi leg only"}


def run_reference(args):
    """The reference arm: the oracle on the host cores.  The K timed steps together run one
    full time-to-solution (CpuOracleStep split into K pieces); `value` is their total and
    ms_per_step their mean.  The W warm-up steps page in the inputs and the code (the
    partition of the matrix and a few sweeps), untimed."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    chain = make_chain()
    for _ in range(max(1, min(args.warmup, 1))):
        w = CpuOracleStep(chain, pieces=2, expect_sweeps=6)
        w.piece(0)
    step = CpuOracleStep(chain, pieces=args.steps)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step.piece(i)
    wall_ms = (time.perf_counter() - t0) * 1e3
    rec = step.record()
    v = rec["value"]
    rec["sample"] = (f"the {args.steps} timed steps together run one full time-to-solution "
                     f"(wall {wall_ms:.0f} ms): " + rec["sample"])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": rec,
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def kernel_times(R, n, d_in, stream, launches=20):
    """Per-launch device time of the four solver kernels on the bench system."""
    out = {}
    ctx = R.reach_create(n, *d_in, stream=stream.cuda_stream)
    try:
        R.reach_precompute(ctx, R.REACH_PROB0_ONLY)
        for meth in ("jacobi", "mixed", "bicgstab"):
            R.reach_autotune(ctx, meth)        # the mappings the timed solves used
        for k in ("jacobi64", "sweep32", "resid_mixed", "bicgstab_spmv"):
            out[k] = R.reach_time_kernel(ctx, k, launches)
    finally:
        R.reach_destroy(ctx)
    return out


def launches_per_step(infos, k, tau_iters=0):
    """Kernels of this library launched in one step (counted from the loop structure)."""
    j, mx, b = infos["jacobi"], infos["mixed"], infos["bicgstab"]
    create = 1
    # search start, its bottom-up levels (no reversed graph on this dense chain), classes,
    # scan, row counts, scan, rows, Jacobi form (with Varah's margin)
    precompute = 1 + j.get("bfs_levels", 3) + 1 + 3 + 1 + 3 + 1 + 1
    jac = j["iters"] + 2 * (j["iters"] // k) + 3
    mix = mx["refinements"] * (2 + (k - 1) + 2) + 3 + 1
    bic = 1 + 5 * b["iters"] + 3
    tau = 1 + (1 + 5 * tau_iters + 3) + 1       # right-hand side, BiCGStab, (I - A) tau' check
    return create + precompute + jac + mix + bic + tau


def finite_or_none(v):
    """JSON has no infinity: an unavailable bound is written as null."""
    return float(v) if v is not None and np.isfinite(v) else None


def run_ours(args):
    import torch
    import paper_1210_6412_gb300 as R
    from paper_1210_6412_gb300 import replicas

    ws, rank, local = dist_init()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    chain = make_chain()
    n, m = chain.n, chain.m
    d_in = [torch.from_numpy(a).to(dev) for a in (chain.rowptr, chain.col, chain.val, chain.goal)]
    h_in = [torch.from_numpy(a).pin_memory() for a in (chain.rowptr, chain.col, chain.val, chain.goal)]
    outs = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in EPS}
    h_outs = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in EPS}
    stream = torch.cuda.current_stream(dev)

    lanes = {}
    bound = {}

    def step(inputs, outputs, parts=None):
        """One step; `parts` (a dict) gets the wall time of each call, in ms."""
        infos = {}
        t = [time.perf_counter()]

        def mark(name):
            if parts is not None:
                t.append(time.perf_counter())
                parts[name] = (t[-1] - t[-2]) * 1e3

        ctx = R.reach_create(n, *inputs, stream=stream.cuda_stream)
        mark("create")
        try:
            R.reach_precompute(ctx, R.REACH_PROB0_ONLY)
            mark("precompute")
            # certified ||(I - A)^-1|| from tau = (I - A)^-1 1, for every solve's error bound
            bound["kinv"], bound["info"] = R.reach_norm_bound(ctx, "bicgstab", eps=1e-8)
            mark("norm_bound")
            for meth in ("jacobi", "mixed", "bicgstab"):
                # row mapping from the autotuner (measured once per system shape, then cached)
                lanes[meth] = R.reach_autotune(ctx, meth)["lanes"]
                _, infos[meth] = R.reach_solve(ctx, n, meth, eps=EPS[meth], max_iter=200_000,
                                               refine_k=K_REFINE, out=outputs[meth])
                mark(meth)
        finally:
            R.reach_destroy(ctx)
            mark("destroy")
        return infos

    for _ in range(args.warmup):
        infos = step(d_in, outs)

    # end to end through the public API: host (pinned) inputs copied in, x copied out.  Run
    # right after the warm-up, like the timed region below, so both see the same thermal and
    # power state (after seconds of FP64 load the Jacobi sweeps run a few % slower)
    e_ms, e_parts = [], []
    with Clocks(local) as e2e_clk:
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize(dev)
            parts = {}
            t0 = time.perf_counter()
            step(h_in, h_outs, parts)
            e_ms.append((time.perf_counter() - t0) * 1e3)
            e_parts.append(parts)
    e2e_clocks = e2e_clk.summary()
    h2d = sum(int(a.numel() * a.element_size()) for a in h_in)
    d2h = 3 * n * 8

    barrier = replicas.barrier
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    all_infos = []
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            all_infos.append(step(d_in, outs))
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.summary()
    ms = replicas.max_over_ranks(ms, dev)
    infos = all_infos[-1]
    errs = {k: float(torch.max(torch.abs(outs[k] - 1.0)).item()) for k in outs}

    jac = infos["jacobi"]
    nq, mq = jac["n_q"], jac["m_q"]
    sweep_ms = jac["ms_solve"] / max(jac["iters"], 1)
    alg_bytes = mq * 12 + nq * 32
    peak_hbm, peak_kind = peaks()
    # per-kernel device times, measured live on the context stream with CUDA events
    kern = kernel_times(R, n, d_in, stream)
    kbytes = {"jacobi64": mq * 12 + nq * 32, "sweep32": mq * (6 if nq <= 65536 else 8) + nq * 16,
              "resid_mixed": mq * (10 if nq <= 65536 else 12) + nq * 32, "bicgstab_spmv": mq * 12 + nq * 40}
    kernels = {}
    for k, t in kern.items():
        gbs = kbytes[k] / (t * 1e-3) / 1e9
        kernels[k] = {"ms": t, "alg_bytes": kbytes[k], "alg_GBps": gbs, "hbm_frac": gbs / peak_hbm}
        if k != "sweep32":
            tf = 2.0 * mq / (t * 1e-3) / 1e12
            kernels[k].update({"fp64_TFLOPs": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS})
    methods = {}
    for k, inf in infos.items():
        methods[k] = {"ms": inf["ms_solve"], "iters": inf["iters"], "max_err": errs[k],
                      "err_bound": finite_or_none(inf["err_bound"]),
                      "resid_inf": inf["resid_inf"], "alg_GBps": inf["bytes_moved"] / (inf["ms_solve"] * 1e6),
                      "refinements": inf["refinements"], "lanes": lanes.get(k)}
    fp64_tf = 2.0 * mq / (sweep_ms * 1e-3) / 1e12
    hbm_gbs = alg_bytes / (sweep_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": m, "n_q": nq, "nnz_q": mq,
                   "refine_k": K_REFINE, "l2": "inputs (1.3 GB) larger than L2; no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "methods": methods,
        "precompute_ms": jac["ms_precompute"],
        "max_err_all": max(errs.values()),
        "err_bound_all": finite_or_none(max(inf["err_bound"] for inf in infos.values())),
        "norm_bound": {"kinv": finite_or_none(bound["kinv"]), "ms": bound["info"]["ms_solve"],
                       "iters": bound["info"]["iters"], "method": "bicgstab on (I - A) tau = 1"},
        # the dominant kernel (FP64 Jacobi sweep) is bound by the FP64 pipe, not HBM
        "roofline": {"bound": "alu", "kernel": "k_jacobi64 (FP64 Jacobi sweep)",
                     "achieved": fp64_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": fp64_tf / FP64_PEAK_TFLOPS, "peak_kind": FP64_PEAK_KIND,
                     "traffic": NCU_TRAFFIC_BYTES, "alg_flops_per_launch": 2 * mq,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": sweep_ms,
                     "hbm_GBps": hbm_gbs, "hbm_frac": hbm_gbs / peak_hbm,
                     "hbm_peak": peak_hbm, "hbm_peak_kind": f"{peak_kind} copy bandwidth"},
        "spmv_hbm": {"kernel": "k_sweep32 (FP32 sweep of the mixed method)",
                     "achieved": kernels.get("sweep32", {}).get("alg_GBps"), "peak": peak_hbm,
                     "unit": "GB/s", "frac": kernels.get("sweep32", {}).get("hbm_frac"),
                     "traffic": NCU_TRAFFIC_SWEEP32_BYTES},
        "kernels": kernels,
        "e2e": {"value": statistics.median(e_ms), "unit": "ms", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": len(e_ms),
                "when": "after the warm-up, before the timed region", "clocks": e2e_clocks,
                "samples_ms": [round(v, 2) for v in e_ms],
                "parts_ms": {k: round(statistics.median(p[k] for p in e_parts), 2) for k in e_parts[0]}},
        "gpu_launches": launches_per_step(infos, K_REFINE, bound["info"]["iters"]) * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        st = CpuOracleStep(chain).run()          # one full, measured run on every host core
        line["cpu_baseline"] = st.record()
        line["cpu_baseline"]["single_core"] = cpu_single_core_estimate(st.m, st.b, st.sweeps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _timed_solves(R, torch, n, d_in, mode, eps, methods, stream):
    """One context: create + precompute + each method; device times from the library."""
    out = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    ctx = R.reach_create(n, *d_in, stream=stream.cuda_stream)
    try:
        R.reach_precompute(ctx, mode)
        xo = torch.empty(n, dtype=torch.float64, device="cuda")
        for meth in methods:
            extra = {}
            if meth in ("jacobi", "mixed", "bicgstab"):
                extra["lanes"] = R.reach_autotune(ctx, meth)["lanes"]
            if meth == "scc_jacobi":   # the decomposition, timed on its own, then the level sweeps
                _, _, si = R.reach_scc(ctx, labels=False)
                extra = {"decompose_ms": si["ms"], "n_scc": si["n_scc"], "n_levels": si["n_levels"],
                         "largest_scc": si["largest"], "exact": si["exact"], "rounds": si["rounds"],
                         "passes": si["passes"]}
            _, info = R.reach_solve(ctx, n, meth, eps=eps[meth], max_iter=2_000_000, refine_k=K_REFINE,
                                    out=xo)
            out[meth] = {"ms": info["ms_solve"] + extra.get("decompose_ms", 0.0), "iters": info["iters"],
                         "resid_inf": info["resid_inf"],
                         "alg_GBps": info["bytes_moved"] / max(info["ms_solve"], 1e-9) / 1e6,
                         "n_q": info["n_q"], "m_q": info["m_q"], "precompute_ms": info["ms_precompute"]}
            if extra:
                out[meth].update(extra, sweeps_ms=info["ms_solve"])
    finally:
        R.reach_destroy(ctx)
    ev1.record(stream)
    torch.cuda.synchronize()
    return out, ev0.elapsed_time(ev1)


def run_workload(args):
    """The other workloads of the method, one JSON line each (not the headline metric).

    random4096: 4096 states, 16 successors, 2% goals, 2% sinks, solved to max|dx| < 1e-10.
    layered: 2000 x 4000 layered model-checker-like chain (8M states).
    table1: random chains with the state and transition counts of the paper's Table 1,
            GPU time-to-solution next to the oracle's on one host core.
    batched: independent chains with 8 goal sets each (`--chains`, default 64; 256 is the
             full batch), 2% sinks, FP32 + FP64 refinement to 1e-6.
    parametric: 4M-state softmax chain, forward solve plus the adjoint gradient in theta.
    """
    import torch
    import paper_1210_6412_gb300 as R
    from paper_1210_6412_gb300 import synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    dev = lambda *a: [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]
    line = {"workload": args.workload, "unit": "ms"}
    if args.workload in ("random4096", "layered", "layered_dag", "cascade", "skewed"):
        if args.workload == "random4096":
            c = synth.random_chain()
            eps = {"jacobi": 1e-10, "mixed": 1e-10, "bicgstab": 1e-10, "scc_jacobi": 1e-10}
        elif args.workload == "layered":
            c = synth.layered_chain()
            eps = {"jacobi": 1e-12, "mixed": 1e-10, "bicgstab": 1e-12, "scc_jacobi": 1e-12}
        elif args.workload == "layered_dag":   # the layered chain without back-edges
            c = synth.layered_chain(p_forward=1.0)
            eps = {"jacobi": 1e-12, "mixed": 1e-10, "bicgstab": 1e-12, "scc_jacobi": 1e-12}
        elif args.workload == "cascade":       # 64 strongly connected stages in a row
            c = synth.cascade_chain(blocks=64, width=65536)
            eps = {"jacobi": 1e-12, "mixed": 1e-10, "bicgstab": 1e-12, "scc_jacobi": 1e-12}
        else:   # row-wise vs entry-balanced sweeps on a few very long rows
            c = synth.skewed_chain(n=1_000_000, hubs=16, hub_deg=200_000)
            eps = {"jacobi": 1e-11, "jacobi_seg": 1e-11, "mixed": 1e-10, "bicgstab": 1e-11,
                   "scc_jacobi": 1e-11}
        d_in = dev(c.rowptr, c.col, c.val, c.goal)
        for _ in range(max(1, args.warmup)):
            _timed_solves(R, torch, c.n, d_in, R.REACH_PROB01, eps, list(eps), stream)
        res, total = _timed_solves(R, torch, c.n, d_in, R.REACH_PROB01, eps, list(eps), stream)
        line.update({"n": c.n, "nnz": c.m, "eps": eps, "methods": res, "step_ms": total})
    elif args.workload == "table1":
        # the chain sizes of the paper's Table 1 (random quicksort and biased die state
        # spaces) as random chains: time-to-solution on the GPU (precompute + solve, device
        # time, inside one context) next to the oracle's on one host core (partition,
        # extraction and its solve), each to max|dx| < 1e-10.  Launch-latency bound.
        import oracle as O
        eps = {"jacobi": 1e-10, "mixed": 1e-10, "bicgstab": 1e-10}
        shapes = []
        for fam, sizes in (("quicksort", synth.TABLE1_QUICKSORT), ("biased_die", synth.TABLE1_BIASED_DIE)):
            for (n_, m_) in sizes:
                c = synth.table1_chain(n_, m_)
                d_in = dev(c.rowptr, c.col, c.val, c.goal)
                _timed_solves(R, torch, c.n, d_in, R.REACH_PROB01, eps, list(eps), stream)
                res, total = _timed_solves(R, torch, c.n, d_in, R.REACH_PROB01, eps, list(eps), stream)
                row = {"family": fam, "n": n_, "m": m_, "precompute_ms": res["jacobi"]["precompute_ms"]}
                for meth, r_ in res.items():
                    row[meth] = {"ms": r_["ms"], "iters": r_["iters"]}
                for meth in ("jacobi", "bicgstab"):
                    t0 = time.perf_counter()
                    _, _, oi = O.reach_probabilities(c.n, c.rowptr, c.col, c.val, c.goal, method=meth, eps=1e-10)
                    row["oracle_" + meth] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": oi["iters"]}
                shapes.append(row)
        line.update({"shapes": shapes, "oracle_cores": 1})
    elif args.workload == "batched":
        if args.chain_states:   # every chain of this many states (the L2 study of the sweep)
            bt = synth.batched_chains(n_chains=args.chains, n_min=args.chain_states,
                                      n_max=args.chain_states + 1, sink_frac=0.02)
        else:
            bt = synth.batched_chains(n_chains=args.chains, sink_frac=0.02)
        n, rowptr, col, val, goals, offs = bt.concat()
        d_in = dev(rowptr, col, val, goals)
        # each chain stops on its own unless --global-stop (one rule over the whole union)
        chains = None if args.global_stop else offs
        for rep in range(max(1, args.warmup) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with R.BatchSolver(n, *d_in, chains=chains) as bs:
                tune = bs.autotune() if args.batch_autotune else {}
                x, info = bs.solve(eps=1e-8, out=torch.empty((goals.shape[0], n), dtype=torch.float64,
                                                              device="cuda"))
                citers, _ = bs.chain_info()
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
        line.update({"chains": args.chains, "n": n, "nnz": int(rowptr[-1]), "k": int(goals.shape[0]),
                     "stopping": "global" if args.global_stop else "per chain",
                     "precompute_ms": info["ms_precompute"], "solve_ms": info["ms_solve"],
                     "iters": info["iters"], "refinements": info["refinements"],
                     "chain_sweeps": {"min": int(citers.min()), "median": float(np.median(citers)),
                                      "max": int(citers.max()),
                                      "row_weighted_mean": float(np.sum(citers * np.diff(offs)) / n)}
                     if chains is not None else None,
                     "resid_inf": info["resid_inf"], "err_bound": finite_or_none(info["err_bound"]),
                     "autotune": tune,
                     "alg_GBps": info["bytes_moved"] / info["ms_solve"] / 1e6, "wall_ms": wall})
        # the same answers from plain FP64 Jacobi, one (chain, goal set) at a time, same eps
        if args.plain:
            plain_ms, plain_pre, plain_iters, worst = 0.0, 0.0, 0, 0.0
            for ci_, ch in enumerate(bt.chains):
                a_, b_ = int(offs[ci_]), int(offs[ci_ + 1])
                d_ch = dev(ch.rowptr, ch.col, ch.val)
                for j in range(goals.shape[0]):
                    g_ = torch.from_numpy(np.ascontiguousarray(bt.goals[ci_][j])).cuda()
                    with R.Solver(ch.n, *d_ch, g_, stream=stream.cuda_stream) as sv:
                        xj, ij = sv.solve("jacobi", eps=1e-8, max_iter=2_000_000)
                    plain_ms += ij["ms_solve"]
                    plain_pre += ij["ms_precompute"]
                    plain_iters += ij["iters"]
                    worst = max(worst, float(torch.max(torch.abs(torch.as_tensor(xj, device="cuda")
                                                                 - x[j, a_:b_])).item()))
            line.update({"plain_fp64_jacobi": {"solve_ms": plain_ms, "precompute_ms": plain_pre,
                                               "sweeps": plain_iters, "solves": len(bt.chains) * goals.shape[0],
                                               "max_abs_diff_vs_batched": worst},
                         "batched_speedup_vs_plain_fp64": (plain_ms + plain_pre) /
                                                          (info["ms_solve"] + info["ms_precompute"])})
    elif args.workload == "parametric":
        from paper_1210_6412_gb300.autograd import reach_prob
        pc = synth.parametric_chain()
        args_d = dev(pc.rowptr, pc.col, pc.cls, pc.offset, pc.goal)
        # forward and adjoint by FP64 Jacobi (the defaults), then both by BiCGStab
        per_method = {}
        for meth in ("jacobi", "bicgstab"):
            for rep in range(max(1, args.warmup) + 1):
                theta = torch.from_numpy(pc.theta).cuda().requires_grad_(True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                y = reach_prob(theta, *args_d, pc.init, eps=1e-13, method=meth, adj_method=meth)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                y.backward()
                torch.cuda.synchronize()
                t2 = time.perf_counter()
            per_method[meth] = {"x_init": float(y), "forward_ms": (t1 - t0) * 1e3,
                                "backward_ms": (t2 - t1) * 1e3, "grad": theta.grad.detach().clone()}
        gj, gb = per_method["jacobi"].pop("grad"), per_method["bicgstab"].pop("grad")
        line.update({"n": pc.n, "nnz": pc.m, "classes": int(pc.theta.size),
                     "x_init": per_method["jacobi"]["x_init"],
                     "forward_ms": per_method["jacobi"]["forward_ms"],
                     "backward_ms": per_method["jacobi"]["backward_ms"],
                     "grad_norm": float(gj.norm()), "bicgstab": per_method["bicgstab"],
                     "max_grad_diff_bicgstab_vs_jacobi": float((gj - gb).abs().max())})
    print(json.dumps(line), flush=True)
    return 0


def run_profile(args):
    """Small fixed run for ncu: the bench workload (or `--workload layered`, the
    model-checker-like chain), one context, `--profile-iters` iterations of one method
    (no stopping test can end it early)."""
    import torch
    import paper_1210_6412_gb300 as R
    from paper_1210_6412_gb300 import synth
    if args.workload == "layered":
        chain, mode = synth.layered_chain(), R.REACH_PROB01
    else:
        chain, mode = make_chain(), R.REACH_PROB0_ONLY
    dev = torch.device("cuda", 0)
    d_in = [torch.from_numpy(a).to(dev) for a in (chain.rowptr, chain.col, chain.val, chain.goal)]
    out = torch.empty(chain.n, dtype=torch.float64, device=dev)
    with R.Solver(chain.n, *d_in, mode=mode) as s:
        del d_in                    # the context holds its own copy; keep the footprint small
        torch.cuda.empty_cache()
        _, info = s.solve(args.profile, eps=1e-300, max_iter=args.profile_iters, refine_k=K_REFINE,
                          out=out, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "iters": info["iters"], "ms": info["ms_solve"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", choices=["jacobi", "mixed", "bicgstab"], default=None,
                    help="run a short fixed-length solve for ncu and exit")
    ap.add_argument("--profile-iters", type=int, default=32)
    ap.add_argument("--workload", choices=["dense", "random4096", "layered", "layered_dag", "cascade", "skewed",
                                           "table1", "batched", "parametric"],
                    default="dense", help="dense = the benchmark; the others print their own line")
    ap.add_argument("--chains", type=int, default=64, help="--workload batched: number of chains")
    ap.add_argument("--chain-states", type=int, default=0,
                    help="--workload batched: every chain with this many states (default: sizes log-uniform in [1e3, 2e6])")
    ap.add_argument("--global-stop", action="store_true",
                    help="--workload batched: one stopping rule over the whole union instead of one per chain")
    ap.add_argument("--batch-autotune", type=int, default=1,
                    help="--workload batched: pick the sweep variant and refinement period by timing")
    ap.add_argument("--plain", type=int, default=1,
                    help="--workload batched: also solve every (chain, goal set) with plain FP64 Jacobi")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.workload != "dense":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
