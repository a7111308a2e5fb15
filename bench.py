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
UNIT = "RHS/s (factor + refined solve, per step)"
RTOL = 1e-12
FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (recipe table); cuBLAS DGEMM measured 1.05 on this machine
FP32_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.070e-3  # SMs x FP32 lanes x 2 x max SM clock (GHz) -> TFLOP/s


# Kernel classes of the mixed path: products on the tensor cores (3xTF32) and FP32 SIMT arithmetic;
# the rest (LU, its solves, the root's LU and inverse) stay FP64.
MIXED_TENSOR = {"sample", "gram", "chol", "proj_nt", "proj_solve", "proj_acc", "lu_rhs", "schur"}
MIXED_FP32 = {"cpqr", "ef_update", "extract", "id_finish", "lu"}
# Classes whose time is data movement (gathers, list copies): no FLOP roof.
MOVE = {"lists", "gather"}


def _class_roof(name: str, mixed: bool, sample_kernel: int):
    """(bound, peak TFLOP/s, note) for a kernel class, or None for data-movement classes."""
    if name in MOVE:
        return None
    if mixed and name in MIXED_TENSOR and not (name == "sample" and sample_kernel == 1):
        bf16 = _peaks().get("bf16_tflops")
        src = "measured bf16 %.1f" % bf16 if bf16 else "fallback bf16 1900"
        tf32 = (bf16 or 1900.0) * 1.1 / 2.25
        return ("tensor", tf32 / 3.0,
                f"3xTF32 effective = TF32 / 3 (three TF32 products per FP32 product); TF32 = {src} x nominal "
                "1.1/2.25; of measured")
    if mixed and (name in MIXED_FP32 or name in MIXED_TENSOR):
        return ("alu", FP32_TFLOPS_NOMINAL, "FP32 SIMT nominal: 152 SMs x 128 lanes x 2 x 2.07 GHz")
    return ("alu", FP64_TFLOPS_NOMINAL, "FP64 nominal 1.25 TFLOP/s (cuBLAS DGEMM measured 1.05 on this pool)")


def _class_table(avg, mixed: bool, sample_kernel: int) -> dict:
    """Per kernel class: device ms per step (CUDA events on the launching stream), algorithmic GFLOP
    per step (counted by the library from the box sizes), launches, achieved TFLOP/s and the
    fraction of the class's roof."""
    out = {}
    for nm, (ms, gflop, nl) in avg.items():
        e = {"ms": round(ms, 3), "gflop": round(gflop, 3), "launches": int(nl)}
        roof = _class_roof(nm, mixed, sample_kernel)
        if roof is not None and ms > 0 and gflop > 0:
            bound, peak, _ = roof
            ach = gflop / ms  # GFLOP/ms = TFLOP/s
            e.update(bound=bound, achieved_tflops=round(ach, 3), peak_tflops=round(peak, 1),
                     frac=round(ach / peak, 4))
        out[nm] = e
    return out


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


def _reduced(pr, n: int):
    """The workload's kind of problem (geometry, kernel, leaf, k, p, right-hand sides) at n points."""
    if n >= pr.n:
        return pr
    pts = W.uniform_points(n, pr.d, W.rng_for(pr.cfg, 0, W.STREAM_POINTS))
    return W.kernel_problem(pr.cfg, f"{pr.name.split('_')[0]}_N{n}_k{pr.k}", pts, pr.kernel, pr.leaf, pr.k,
                            pr.s_cfg, pr.nrhs)


def _oracle_run(pr) -> dict:
    """One whole step of the CPU oracle, as it stands, on problem pr: tree and schedule, test
    matrices, the dense sampling product, Algorithm 1 and the root, then every right-hand side
    refined with the factor to RTOL with the dense FP64 residual.  Seconds per phase."""
    from oracle import operators as oops
    from oracle import refine as oref
    from oracle import rsrs as orsrs
    from oracle.tree import Schedule as OSched
    from oracle.tree import Tree as OTree

    t = [time.perf_counter()]
    tree = OTree(pr.points, pr.leaf)
    sched = OSched(tree, pr.k)
    s = max(pr.s_cfg, sched.s_req)
    om, ps = pr.omega(s), pr.psi(s)
    op = oops.make_operator(pr)
    y, z = oops.sample(op, om, ps)
    t.append(time.perf_counter())
    fac = orsrs.factor(tree, sched, y, z, om, ps)
    t.append(time.perf_counter())
    b = pr.rhs()
    its = []
    for c in range(b.shape[1]):
        _, hist = oref.refine(fac, op, b[:, c], rtol=RTOL, maxit=30)
        its.append(len(hist) - 1)
    t.append(time.perf_counter())
    return {"n": pr.n, "s": s, "boxes": len(sched.steps), "t_sample": t[1] - t[0], "t_factor": t[2] - t[1],
            "t_refine": t[3] - t[2], "total": t[3] - t[0], "refine_iterations": max(its)}


def _calibrate_oracle_n(pr, budget_s: float) -> int:
    """Largest N (a power of two, at least 1024, at most the workload's) whose whole oracle step is
    expected to fit the budget, judged from the step time at the smaller sizes (one run each)."""
    n, last = 1024, None
    while True:
        r = _oracle_run(_reduced(pr, n))
        last = (n, r["total"])
        if 2 * n > pr.n or r["total"] * 3.0 > budget_s:
            return last[0]
        n *= 2


def _cpu_baseline(pr, budget_s: float = 20.0) -> dict:
    """The CPU oracle as it stands, on the machine's host cores, run whole on a reduced instance of the
    workload (same kind of problem at a smaller N, chosen so that the run takes about budget_s),
    with a separately labelled model extrapolation to the workload's size."""
    from oracle.tree import Schedule as OSched
    from oracle.tree import Tree as OTree

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    n = _calibrate_oracle_n(pr, budget_s)
    r = _oracle_run(_reduced(pr, n))
    full = OSched(OTree(pr.points, pr.leaf), pr.k)
    s_full = max(pr.s_cfg, full.s_req)
    # model: sampling ~ N^2 s, box loop ~ boxes (same leaf, k and near-field sizes), refinement ~ N^2
    est = (r["t_sample"] * (pr.n / n) ** 2 * (s_full / r["s"]) + r["t_factor"] * len(full.steps) / r["boxes"]
           + r["t_refine"] * (pr.n / n) ** 2)
    return {"value": pr.nrhs / r["total"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"whole oracle step (sampling, Algorithm 1, root, {pr.nrhs} RHS refined to {RTOL:g}) on "
                       f"the same kind of problem reduced to N = {n} (s = {r['s']}, {r['boxes']} boxes): "
                       f"{r['total']:.1f} s; numpy/LAPACK on all {cores} host cores"),
            "reduced_n": n, "seconds": round(r["total"], 2),
            "phases_s": {k: round(r[k], 2) for k in ("t_sample", "t_factor", "t_refine")},
            "extrapolated_to_workload": {"value": pr.nrhs / est, "unit": UNIT, "step_s": round(est, 1),
                                         "model": "sampling x (N/n)^2 (s/s_n), box loop x boxes/boxes_n, "
                                                  "refinement x (N/n)^2; a model, not a measurement"}}


def _rank_env():
    """(world size, rank, local rank) from the launcher's environment; torchrun sets all three."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _barrier():
    """Barrier over the ranks of the process group, when one is initialised (N > 1)."""
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _shard(items, world: int, rank: int) -> list:
    """Rank r's share of independent problems: items r, r + world, r + 2 world, ...  The shares are
    disjoint, their union is the whole list, and no rank's share needs another rank's data."""
    return list(items)[rank::world]


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
    """The reference arm: the CPU oracle as it stands, each step one whole oracle step on the
    workload's kind of problem at a reduced N (calibrated once so that the K + W steps end within a
    few minutes).  Rank 0 only; the other ranks exit without work."""
    _, rank, _ = _rank_env()
    if rank != 0:
        return
    pr = _problem(args.workload, args.n)
    budget = max(5.0, 150.0 / (args.warmup + args.steps))
    n = _calibrate_oracle_n(pr, budget)
    prr = _reduced(pr, n)
    runs = [_oracle_run(prr) for _ in range(args.warmup + args.steps)]
    tv = runs[args.warmup:]
    ms = 1e3 * statistics.mean(r["total"] for r in tv)
    v = pr.nrhs / (ms / 1e3)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"whole oracle step (sampling, Algorithm 1, root, {pr.nrhs} RHS refined to {RTOL:g}) on the same "
              f"kind of problem reduced to N = {n} (s = {tv[0]['s']}, {tv[0]['boxes']} boxes); numpy/LAPACK on "
              f"all {cores} host cores")
    from oracle.tree import Schedule as OSched
    from oracle.tree import Tree as OTree

    cfg = _config(pr, max(pr.s_cfg, OSched(OTree(pr.points, pr.leaf), pr.k).s_req))
    cfg["oracle_reduced_n"] = n
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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

    if args.profile_step:  # ncu runs: W + K plain steps (build + refined solve) and nothing else
        for i in range(args.warmup + args.steps):
            f = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=500 + i,
                         sample_kernel=args.sample_kernel, tune=tune)
            rep = f.refine(B, X, rtol=RTOL, maxit=30)
            del f
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "workload": pr.name, "refine_iterations": rep.iterations,
                          "residual_kind": rep.residual_kind}), flush=True)
        return

    def step(seed, profile=False):
        f = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=seed,
                     profile=profile, sample_kernel=args.sample_kernel, tune=tune)
        rep = f.refine(B, X, rtol=RTOL, maxit=30)
        st = f.stats()
        cls = f.class_stats()
        del f
        return rep, st, cls

    # (1) the measured path: the build captured once as a CUDA graph, each step replaying it with new
    # test matrices (rsrs_refactor, a new Philox key per step) and refining the right-hand sides
    fg = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=999,
                  sample_kernel=args.sample_kernel, tune=tune, use_graph=True)
    graph_launches = int(fg.stats().kernel_launches)

    def gstep(seed):
        fg.refactor(seed)
        return fg.refine(B, X, rtol=RTOL, maxit=30)

    for w in range(args.warmup):
        gstep(1000 + w)
    torch.cuda.synchronize()
    _barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.steps):
            reps.append(gstep(rank * 100003 + i))
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier()
    ms, total_rhs = _job_time(e0.elapsed_time(e1), pr.nrhs * args.steps, "cuda")
    value = total_rhs / (ms / 1e3)
    x_mixed = X.clone()
    del fg

    # (2) beside it, plain (uncaptured) builds with per-class CUDA events, timed the same way: the
    # per-class device times and roofline fractions come from these steps
    for w in range(min(args.warmup, 1)):
        step(2000 + w)
    torch.cuda.synchronize()
    _barrier()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    preps, sts, clss = [], [], []
    torch.cuda.synchronize()
    p0.record(stream)
    for i in range(args.steps):
        rep, st, cls = step(rank * 100003 + 50 + i, profile=True)
        preps.append(rep)
        sts.append(st)
        clss.append(cls)
    p1.record(stream)
    torch.cuda.synchronize()
    _barrier()
    pms, _ = _job_time(p0.elapsed_time(p1), pr.nrhs * args.steps, "cuda")

    # per-class times averaged over the plain steps; the dominant class gives the headline roofline
    names = list(clss[0].keys())
    avg = {nm: (sum(c[nm][0] for c in clss) / len(clss), clss[0][nm][1], clss[0][nm][2]) for nm in names}
    mixed = prec == R.RSRS_PREC_MIXED
    dom = max((nm for nm in avg if _class_roof(nm, mixed, args.sample_kernel)), key=lambda nm: avg[nm][0])
    dom_ms, dom_gflop, dom_launch = avg[dom]
    bound, peak, peak_note = _class_roof(dom, mixed, args.sample_kernel)
    achieved = dom_gflop / dom_ms if dom_ms > 0 else 0.0  # GFLOP/ms = TFLOP/s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)" if mixed else "f64",
        "data": "synthetic (seeded uniform points, device Philox test matrices, Gaussian RHS)",
        "config": _config(pr, s),
        "step": "graph replay of the captured build with new test matrices (rsrs_refactor) + refined solve",
        "factor_ms": statistics.mean(x.t_sample_ms + x.t_compress_ms + x.t_root_ms for x in sts),
        "refine_iterations": [r.iterations for r in reps],
        "rel_residual": max(r.rel_residual for r in reps),
        "gpu_launches": graph_launches * args.steps + sum(int(rp.kernel_launches) for rp in reps),
        "plain_build": {"ms_per_step": pms / args.steps, "value": total_rhs / (pms / 1e3),
                        "launches_per_step": statistics.mean(int(x.kernel_launches) for x in sts),
                        "note": "uncaptured builds with per-class CUDA events (source of kernel_classes)"},
        "kernel_classes": _class_table(avg, mixed, args.sample_kernel),
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
    # the factor's first refinement also makes the residual's store of K's digits (once per factor)
    a0 = time.perf_counter()
    f.refine(B, X, rtol=RTOL, maxit=30)
    torch.cuda.synchronize()
    t_first = time.perf_counter() - a0
    X.zero_()
    a0 = time.perf_counter()
    rep = f.refine(B, X, rtol=RTOL, maxit=30)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - a0
    Fs = B.clone()
    f.solve(Fs)  # warm-up (first use of the stream-ordered scratch pool)
    torch.cuda.synchronize()
    nsol = 5
    a0 = time.perf_counter()
    for _ in range(nsol):
        f.solve(Fs)
    torch.cuda.synchronize()
    t_sol = (time.perf_counter() - a0) / nsol
    line["solves_per_s_refined"] = pr.nrhs / t_ref
    line["first_refine_ms"] = t_first * 1e3  # includes making the residual's digit store
    line["solves_per_s_unrefined"] = pr.nrhs / t_sol
    # the solve's sweeps read each factor block in the solve's arithmetic (the library's count)
    hbm = _peaks().get("hbm_gbs")
    sb = int(f.stats().solve_bytes)
    line["solve_sweeps"] = {"bytes_per_solve": sb, "ms_per_solve": t_sol * 1e3, "achieved_gbs": sb / t_sol / 1e9,
                            "peak_gbs": hbm, "frac": (sb / t_sol / 1e9 / hbm) if hbm else None,
                            "note": "one solve of 16 right-hand sides (mean of 5 after a warm-up), host clock "
                                    "around the call with a device synchronisation; of measured HBM copy peak"}
    if rep.residual_kind == R.RSRS_RESIDUAL_OZAKI:
        # the refinement's residual product (Ozaki scheme): per product it streams the factor's store of
        # K's digits once, 20 bytes per matrix entry and group of 16 right-hand sides (HBM-bound);
        # CUDA events on the launching stream around single rsrs_residual calls (store already made)
        Rr = torch.empty_like(B)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        tms = []
        for _ in range(3):
            ev[0].record(stream)
            f.residual(B, X, Rr)
            ev[1].record(stream)
            torch.cuda.synchronize()
            tms.append(ev[0].elapsed_time(ev[1]))
        gb = 20.0 * pr.n * pr.n * ((pr.nrhs + 15) // 16) / 1e9
        hbm = _peaks().get("hbm_gbs")
        ach = gb / (min(tms) / 1e3)
        line["kernel_classes"]["residual_ozaki"] = {
            "ms": round(min(tms), 3), "gbytes": round(gb, 3), "launches": 4 * ((pr.nrhs + 15) // 16),
            "bound": "hbm", "achieved_gbs": round(ach, 1), "peak_gbs": hbm,
            "frac": round(ach / hbm, 4) if hbm else None, "traffic": _traffic("residual_ozaki", pr.name),
            "note": "one rsrs_residual call (B - A X, 16 columns, including its host-side allocations), digits "
                    "streamed once; of measured HBM copy peak"}
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
        # FP64 path: FP64 throughout, its sampling product FP64-accurate by the Ozaki scheme on the
        # bf16 tensor cores (sample_kernel 3; the FP64 SIMT product where the digit store does not fit)
        f64 = R.Factor(tree, kind, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=R.RSRS_PREC_FP64,
                       seed=1000, sample_kernel=3)
        X64 = torch.zeros_like(B)
        rep64 = f64.refine(B, X64, rtol=RTOL, maxit=30)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - a0
        st64 = f64.stats()
        rel = float(torch.linalg.norm(x_mixed - X64) / torch.linalg.norm(X64))
        line["fp64"] = {"sampling": "Ozaki scheme (FP64-accurate) where the digit store fits, else FP64 SIMT",
                        "sample_ms": st64.t_sample_ms,
                        "factor_ms": st64.t_sample_ms + st64.t_compress_ms + st64.t_root_ms,
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
        line["cpu_baseline"] = _cpu_baseline(pr, budget_s=args.cpu_budget)
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

    allp = W.config(args.workload)
    k = allp[0].k
    # the sample count is common to the whole batch (all ranks), so every rank's share is built with the
    # same s as the unsharded batch
    s = max(max((t.info(k).s_req_mixed if args.precision == "mixed" else t.info(k).s_req)
                for t in (R.Tree(p.points, p.leaf) for p in allp)), allp[0].s_cfg)
    prs = _shard(allp, world, rank)  # independent problems split across ranks, no exchange
    trees = [R.Tree(p.points, p.leaf) for p in prs]
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
    assert world > 1 or total_rhs == sum(p.nrhs for p in allp) * args.steps
    clss = [r[2] for r in res]
    names = list(clss[0].keys())
    avg = {nm: (sum(c[nm][0] for c in clss) / len(clss), clss[0][nm][1], clss[0][nm][2]) for nm in names}
    dom = max((nm for nm in avg if _class_roof(nm, prec == R.RSRS_PREC_MIXED, args.sample_kernel)),
              key=lambda nm: avg[nm][0])
    dom_ms, dom_gflop, dom_launch = avg[dom]
    bound, peak, peak_note = _class_roof(dom, prec == R.RSRS_PREC_MIXED, args.sample_kernel)
    achieved = dom_gflop / dom_ms if dom_ms > 0 else 0.0
    st = res[0][1]
    line = {
        "metric": METRIC, "value": total_rhs / (ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)" if prec == R.RSRS_PREC_MIXED else "f64",
        "data": "synthetic (seeded uniform points, device Philox test matrices, Gaussian RHS)",
        "config": {"workload": f"batch2d_{len(allp)}x_N2048-16384_k{k}", "problems": len(allp),
                   "problems_per_rank": len(prs), "sharding": "problem i on rank i mod N, no exchange",
                   "N_total": int(sum(p.n for p in allp)), "kernel": prs[0].kernel, "leaf": prs[0].leaf, "k": k,
                   "s_cfg": prs[0].s_cfg, "s": s, "nrhs_per_problem": prs[0].nrhs, "rtol": RTOL,
                   "l2": "inputs larger than L2"},
        "factor_ms": st.t_sample_ms + st.t_compress_ms + st.t_root_ms,
        "refine_iterations_max": max(max(r[0]) for r in res),
        "gpu_launches": sum(int(r[1].kernel_launches) + r[3] for r in res),
        "kernel_classes": _class_table(avg, prec == R.RSRS_PREC_MIXED, args.sample_kernel),
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
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling runs only: W + K plain build-and-refine steps, no timing or extra legs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif len(W.config(args.workload)) > 1:
        run_gpu_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
