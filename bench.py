#!/usr/bin/env python
"""Benchmark: RSRS factorization plus a refined solve on one GB300 (or N replicas).

One step = the whole hot path on one problem: draw Omega, Psi on the device,
sample Y, Z, run Algorithm 1 (all levels), extract and factor the root, then
solve for the right-hand sides with FP64 iterative refinement to a relative
residual of 1e-12.  Default workload: N = 65536 uniform random points in
[0,1]^2, A = I + (1/N) log|x_i - x_j| (K_ii = 0), leaf 64, k = 48, 16 RHS, at
s = s_req (the literal s = 600 is below the sample bound and is refused).

Prints one JSON line.  --impl reference times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "RSRS factor time & solves/s at 1e-10 rel err: mixed vs FP64, 1 GB300"
RTOL = 1e-12
FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (recipe table); cuBLAS DGEMM measured 1.05 on this machine
FP32_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.070e-3  # SMs x FP32 lanes x 2 x max SM clock (GHz) -> TFLOP/s


# Kernel classes that run in FP32 arithmetic in the mixed path (the rest stay FP64).
MIXED_FP32 = {"sample", "gram", "chol", "gather", "proj_nt", "proj_solve", "proj_acc", "cpqr", "ef_update",
              "extract", "schur"}


def _class_roof(name: str, mixed: bool, sample_kernel: int):
    """(bound, peak TFLOP/s, note) for a kernel class."""
    if mixed and name == "sample" and sample_kernel in (0, 2):
        bf16 = _peaks().get("bf16_tflops")
        src = "measured bf16 %.1f" % bf16 if bf16 else "fallback bf16 1900"
        tf32 = (bf16 or 1900.0) * 1.1 / 2.25
        return ("tensor", tf32 / 3.0,
                f"3xTF32 effective = TF32 / 3 (three TF32 products per FP32 product); TF32 = {src} x nominal "
                "1.1/2.25; of measured")
    if mixed and name in MIXED_FP32:
        return ("alu", FP32_TFLOPS_NOMINAL, "FP32 SIMT nominal: 152 SMs x 128 lanes x 2 x 2.07 GHz")
    return ("alu", FP64_TFLOPS_NOMINAL, "FP64 nominal 1.25 TFLOP/s (cuBLAS DGEMM measured 1.05 on this pool)")


def _traffic(name: str, workload: str):
    """DRAM bytes per launch of this kernel class from the committed ncu summary, when it was taken
    on this workload and the kernel's source has not changed since (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tab = json.load(fh)
    except (OSError, ValueError):
        return None
    e = tab.get(name)
    if not e or e.get("workload") != workload:
        return None
    with open(os.path.join(ROOT, e["source"]), "rb") as fh:
        if hashlib.sha1(fh.read()).hexdigest() != e["source_sha1"]:
            return None
    return e["dram_bytes_per_launch"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _problem(idx: int, n: int = 0):
    """Workload ``idx``; ``n`` > 0 keeps its kind and sizes but draws n points (profiling runs)."""
    pr = W.config(idx)[0]
    if n and n != pr.n and pr.kernel != "stencil7":
        pts = W.uniform_points(n, pr.d, W.rng_for(pr.cfg, 0, W.STREAM_POINTS))
        pr = W.kernel_problem(pr.cfg, f"{pr.name.split('_')[0]}_N{n}_k{pr.k}", pts, pr.kernel, pr.leaf, pr.k,
                              pr.s_cfg, pr.nrhs)
    return pr


def _cpu_baseline(pr, s: int, budget_s: float = 20.0) -> dict:
    """The CPU oracle, as it stands, timed on a bounded sample of the workload and extrapolated.

    Sample: the oracle's sampling product on 64 rows, its Algorithm-1 box loop on
    the first boxes of the deepest levels (until ``budget_s``), and its solve
    sweep is not timed separately (a refinement step is dominated by the dense
    FP64 residual product, timed through the same 64-row sample).
    """
    from oracle import operators as oops
    from oracle import rsrs as orsrs
    from oracle.tree import Schedule as OSched
    from oracle.tree import Tree as OTree

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    tree = OTree(pr.points, pr.leaf)
    sched = OSched(tree, pr.k)
    n = pr.n
    rng = np.random.default_rng(0)
    om = rng.standard_normal((n, s))
    ps = rng.standard_normal((n, s))
    op = oops.make_operator(pr)
    idx = np.arange(64)
    t0 = time.perf_counter()
    _ = op.rows(idx) @ om
    t_rows = (time.perf_counter() - t0) / 64.0
    t_sample = 2 * n * t_rows
    # Algorithm 1 on stand-in sketches: the arithmetic per box does not depend on their values
    y, z = om * 1.0001, ps * 1.0001
    flops_model = lambda st: 2 * (st["b"] + st["n"]) ** 2 * s + 2 * (st["b"] + st["n"]) ** 3
    done = 0
    t0 = time.perf_counter()
    m = 4
    while True:
        orsrs.factor(tree, sched, y, z, om, ps, max_steps=m)
        el = time.perf_counter() - t0
        done = m
        if el > budget_s or m >= len(sched.steps):
            break
        m = min(len(sched.steps), m * 2)
        t0 = time.perf_counter()
    sample_flops = sum(flops_model(st) for st in sched.steps[:done])
    total_flops = sum(flops_model(st) for st in sched.steps)
    t_factor = el * total_flops / sample_flops
    iters = 3  # refinement corrections typical of this workload
    t_refine = (iters + 1) * n * t_rows * pr.nrhs / s
    total = t_sample + t_factor + t_refine
    return {"value": pr.nrhs / total, "unit": "RHS/s (factor + refined solve)", "cores": cores,
            "kind": "oracle",
            "sample": (f"oracle sampling product on 64 of {n} rows; Algorithm 1 on the first {done} of "
                       f"{len(sched.steps)} boxes ({el:.1f} s), extrapolated by per-box l^2 s + l^3 work; "
                       f"refinement from the row-product rate"),
            "est_factor_s": t_sample + t_factor}


def _rank_env():
    """(world size, rank, local rank) from the launcher's environment; torchrun sets all three."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _barrier():
    """Barrier over the ranks of the process group, when one is initialised (N > 1)."""
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _job_time(ms, units, device):
    """Whole-job time and work over the ranks.  Every rank runs its own replica of the path with
    no exchange between them, so the job takes the slowest rank's time (MAX) and has processed
    every rank's units (SUM).  Without a process group (one GPU) both pass through unchanged."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


def run_reference(args):
    _, rank, _ = _rank_env()
    if rank != 0:  # the CPU oracle runs once, on rank 0; the other ranks exit without work
        return
    pr = _problem(args.workload, args.n)
    from oracle.tree import Schedule as OSched
    from oracle.tree import Tree as OTree

    s = max(pr.s_cfg, OSched(OTree(pr.points, pr.leaf), pr.k).s_req)
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(_cpu_baseline(pr, s, budget_s=max(5.0, 60.0 / (args.warmup + args.steps))))
    tv = vals[args.warmup:]
    v = statistics.median(x["value"] for x in tv)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": tv[0]["unit"], "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * pr.nrhs / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(pr, s),
            "cpu_baseline": {"kind": "oracle", "cores": tv[0]["cores"], "sample": tv[0]["sample"], "value": v},
            "e2e": {"value": v, "unit": tv[0]["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(pr, s):
    return {"workload": pr.name, "N": pr.n, "d": pr.d, "kernel": pr.kernel, "leaf": pr.leaf, "k": pr.k,
            "p": pr.k, "s_cfg": pr.s_cfg, "s": s, "nrhs": pr.nrhs, "rtol": RTOL,
            "l2": "inputs larger than L2 (Y, Z, Omega, Psi are N x s FP64, 0.96 GB each)"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    __graft_entry__.build()
    import paper_2311_01451_gb300 as R

    pr = _problem(args.workload, args.n)
    tree = R.Tree(pr.points, pr.leaf)
    info = tree.info(pr.k)
    s = max(pr.s_cfg, info.s_req_mixed if args.precision == "mixed" else info.s_req)
    kind = R.kind_of(pr.kernel)
    b_host = pr.rhs()  # N x nrhs column-major
    B = torch.tensor(np.ascontiguousarray(b_host.T), device="cuda")
    X = torch.zeros_like(B)
    stream = torch.cuda.current_stream()
    prec = R.RSRS_PREC_MIXED if args.precision == "mixed" else R.RSRS_PREC_FP64

    tune, tune_info = _autotune(args, R, tree, kind, pr.k, s, pr.diag_shift, pr.scale, prec)

    def step(seed, profile=False):
        f = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=seed,
                     profile=profile, sample_kernel=args.sample_kernel, tune=tune)
        rep = f.refine(B, X, rtol=RTOL, maxit=30)
        st = f.stats()
        cls = f.class_stats()
        del f
        return rep, st, cls

    for w in range(args.warmup):
        step(1000 + w)
    torch.cuda.synchronize()
    _barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps, sts, clss = [], [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.steps):
            rep, st, cls = step(rank * 100003 + i, profile=True)
            reps.append(rep)
            sts.append(st)
            clss.append(cls)
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier()
    ms, total_rhs = _job_time(e0.elapsed_time(e1), pr.nrhs * args.steps, "cuda")
    value = total_rhs / (ms / 1e3)
    x_mixed = X.clone()

    # per-class times averaged over the timed steps; the dominant class gives the roofline
    names = list(clss[0].keys())
    avg = {nm: (sum(c[nm][0] for c in clss) / len(clss), clss[0][nm][1], clss[0][nm][2]) for nm in names}
    dom = max(avg, key=lambda nm: avg[nm][0])
    dom_ms, dom_gflop, dom_launch = avg[dom]
    bound, peak, peak_note = _class_roof(dom, prec == R.RSRS_PREC_MIXED, args.sample_kernel)
    achieved = dom_gflop / dom_ms if dom_ms > 0 else 0.0  # GFLOP/ms = TFLOP/s
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s (factor + refined solve, per step)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)" if prec == R.RSRS_PREC_MIXED else "f64",
        "data": "synthetic (seeded uniform points, device Philox test matrices, Gaussian RHS)",
        "config": _config(pr, s),
        "factor_ms": statistics.mean(x.t_sample_ms + x.t_compress_ms + x.t_root_ms for x in sts),
        "refine_iterations": [r.iterations for r in reps],
        "rel_residual": max(r.rel_residual for r in reps),
        "gpu_launches": sum(int(x.kernel_launches) + int(rp.kernel_launches) for rp, x in zip(reps, sts)),
        "kernel_classes_ms": {nm: round(avg[nm][0], 3) for nm in names},
        "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": _traffic(dom, pr.name),
                     "peak_note": peak_note,
                     "algorithmic_gflop_per_step": dom_gflop, "launches_per_step": dom_launch},
        "clocks": clk.summary(),
        "autotune": tune_info,
    }
    # solves/s with the factor reused (refined and plain), and the FP64 comparison
    f = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=7, tune=tune)
    torch.cuda.synchronize()
    a0 = time.perf_counter()
    rep = f.refine(B, X, rtol=RTOL, maxit=30)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - a0
    Fs = B.clone()
    a0 = time.perf_counter()
    f.solve(Fs)
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - a0
    line["solves_per_s_refined"] = pr.nrhs / t_ref
    line["solves_per_s_unrefined"] = pr.nrhs / t_sol
    # GMRES with the same factor as preconditioner (the paper's solver), to 1e-10 as in its tables
    Xg = torch.zeros_like(B)
    torch.cuda.synchronize()
    a0 = time.perf_counter()
    gm = f.gmres(B, Xg, rtol=1e-10, restart=30, maxit=30)
    torch.cuda.synchronize()
    t_gm = time.perf_counter() - a0
    line["gmres"] = {"rtol": 1e-10, "iterations": gm.iterations, "rel_residual": gm.rel_residual,
                     "solves_per_s": pr.nrhs / t_gm}
    del f
    if not args.no_compare and rank == 0:
        a0 = time.perf_counter()
        f64 = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=R.RSRS_PREC_FP64,
                       seed=1000)
        X64 = torch.zeros_like(B)
        rep64 = f64.refine(B, X64, rtol=RTOL, maxit=30)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - a0
        st64 = f64.stats()
        rel = float(torch.linalg.norm(x_mixed - X64) / torch.linalg.norm(X64))
        line["fp64"] = {"factor_ms": st64.t_sample_ms + st64.t_compress_ms + st64.t_root_ms,
                        "step_ms": t64 * 1e3, "refine_iterations": rep64.iterations,
                        "rhs_per_s": pr.nrhs / t64, "mixed_vs_fp64_rel_diff": rel}
        line["speedup_vs_fp64"] = (t64 * 1e3) / (ms / args.steps)
        del f64
    # end to end through the C ABI from host buffers: tree from host points, RHS H2D from pinned
    # memory, factor, refined solve, result D2H
    b_pin = torch.tensor(np.ascontiguousarray(b_host.T)).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    torch.cuda.synchronize()
    a0 = time.perf_counter()
    t2 = R.Tree(pr.points, pr.leaf)
    Bd = b_pin.to("cuda", non_blocking=True)
    Xd = torch.zeros_like(Bd)
    f = R.Factor(t2, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=11, tune=tune)
    f.refine(Bd, Xd, rtol=RTOL, maxit=30)
    x_pin.copy_(Xd, non_blocking=True)
    torch.cuda.synchronize()
    te = time.perf_counter() - a0
    del f
    line["e2e"] = {"value": pr.nrhs / te, "unit": line["unit"],
                   "h2d_bytes_per_step": int(pr.points.nbytes + b_pin.numel() * 8),
                   "d2h_bytes_per_step": int(x_pin.numel() * 8)}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = _cpu_baseline(pr, s, budget_s=args.cpu_budget)
        line["cpu_baseline"].pop("est_factor_s", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_gpu_batched(args):
    """The batched workload: every problem of W.config(args.workload) factored together with
    rsrs_build_batched (one launch per (height, colour) group across problems, batched roots), then
    each problem's right-hand sides refined to RTOL.  value = all problems' RHS per step / time."""
    import torch
    import torch.distributed as dist

    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    __graft_entry__.build()
    import paper_2311_01451_gb300 as R

    prs = W.config(args.workload)
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    k = prs[0].k
    s = max(max((t.info(k).s_req_mixed if args.precision == "mixed" else t.info(k).s_req) for t in trees),
            prs[0].s_cfg)
    kinds = [R.kind_of(p.kernel) for p in prs]
    prec = R.RSRS_PREC_MIXED if args.precision == "mixed" else R.RSRS_PREC_FP64
    Bs = [torch.tensor(np.ascontiguousarray(p.rhs().T), device="cuda") for p in prs]
    Xs = [torch.zeros_like(b) for b in Bs]
    stream = torch.cuda.current_stream()

    tune, tune_info = _autotune(args, R, trees, kinds, k, s, [p.diag_shift for p in prs], [p.scale for p in prs],
                                prec)

    def step(seed, profile=False):
        fs = R.build_batched(trees, kinds, k, s, [p.diag_shift for p in prs], [p.scale for p in prs],
                             precision=prec, seed=seed, profile=profile, sample_kernel=args.sample_kernel,
                             tune=tune)
        reps = [f.refine(b, x, rtol=RTOL, maxit=30) for f, b, x in zip(fs, Bs, Xs)]
        its = [r.iterations for r in reps]
        st, cls = fs[0].stats(), fs[0].class_stats()
        del fs
        return its, st, cls, sum(int(r.kernel_launches) for r in reps)

    for w in range(args.warmup):
        step(2000 + w)
    torch.cuda.synchronize()
    _barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.steps):
            res.append(step(3000 + rank * 100003 + i, profile=True))
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier()
    ms, total_rhs = _job_time(e0.elapsed_time(e1), sum(p.nrhs for p in prs) * args.steps, "cuda")
    clss = [r[2] for r in res]
    names = list(clss[0].keys())
    avg = {nm: (sum(c[nm][0] for c in clss) / len(clss), clss[0][nm][1], clss[0][nm][2]) for nm in names}
    dom = max(avg, key=lambda nm: avg[nm][0])
    dom_ms, dom_gflop, dom_launch = avg[dom]
    bound, peak, peak_note = _class_roof(dom, prec == R.RSRS_PREC_MIXED, args.sample_kernel)
    achieved = dom_gflop / dom_ms if dom_ms > 0 else 0.0
    st = res[0][1]
    line = {
        "metric": METRIC, "value": total_rhs / (ms / 1e3), "unit": "RHS/s (factor + refined solve, per step)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)" if prec == R.RSRS_PREC_MIXED else "f64",
        "data": "synthetic (seeded uniform points, device Philox test matrices, Gaussian RHS)",
        "config": {"workload": f"batch2d_{len(prs)}x_N2048-16384_k{k}", "problems": len(prs),
                   "N_total": int(sum(p.n for p in prs)), "kernel": prs[0].kernel, "leaf": prs[0].leaf, "k": k,
                   "s_cfg": prs[0].s_cfg, "s": s, "nrhs_per_problem": prs[0].nrhs, "rtol": RTOL,
                   "l2": "inputs larger than L2"},
        "factor_ms": st.t_sample_ms + st.t_compress_ms + st.t_root_ms,
        "refine_iterations_max": max(max(r[0]) for r in res),
        "gpu_launches": sum(int(r[1].kernel_launches) + r[3] for r in res),
        "kernel_classes_ms": {nm: round(avg[nm][0], 3) for nm in names},
        "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_note": peak_note,
                     "algorithmic_gflop_per_step": dom_gflop, "launches_per_step": dom_launch},
        "clocks": clk.summary(),
        "autotune": tune_info,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _autotune(args, R, trees, kinds, k, s, shifts, scales, prec):
    """Launch shapes from the library's autotuner (before the warm-up; cached per device and
    workload in the temporary directory), or the defaults with --tune none."""
    if args.tune == "none":
        return None, None
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "rsrs_tune_cache.txt")
    t0 = time.perf_counter()
    tune, rep = R.autotune(trees, kinds, k, s, shifts, scales, precision=prec, reps=1, cache=cache,
                           sample_kernel=args.sample_kernel)
    rep["seconds"] = round(time.perf_counter() - t0, 2)
    return tune, {"tune": tune, **rep}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", type=int, default=1, help="workload index (1: 2D N=65536, k=48)")
    ap.add_argument("--n", type=int, default=0, help="override the number of points (profiling runs only)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--sample-kernel", type=int, default=0, help="mixed sampling: 0 default, 1 FP32 SIMT, 2 tcgen05")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--tune", choices=["auto", "none"], default="auto",
                    help="launch shapes: the library's autotuner (cached) or the defaults")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif len(W.config(args.workload)) > 1:
        run_gpu_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
