#!/usr/bin/env python
"""Time-to-tolerance of the DeepONet-BiCGStab meta-solver on one GB300.

Workload (scenes.BENCH_WORKLOADS["submarine3d-128"], the mixed-precision
configuration): 3D Helmholtz on 128^3 nodes, k = 32, 8-cell absorbing layer,
seeded-rotation submarine scatterer, scattered-field solve for a seeded plane
wave; seeded trunk [3,256,256,256], natural-order trunk basis (p = 256,
tau = 1e-6); BiCGStab right-preconditioned by the hybrid cycle (3 red-black GS
sweeps, then the trunk-basis Galerkin correction) to 1e-6 on the FP64 true
residual.  The timed form is the mixed-precision handle (complex64 Krylov
vectors, operator and cycle, BF16 basis, FP64 iterate and reliable updates);
the FP64 handle solves the same inputs for comparison (`extra`), and the 64^3
FP64 workload (cube3d-64, to 1e-8) is a second entry.

One step = one complete solve from x0 = 0 (inputs resident on the device, setup
of the trunk basis done once before the timed region).  `e2e` repeats the step
through helm_solve_host with pinned host buffers.  Under torchrun every rank
solves the same problem on its own GPU (replicas: the path has no exchange).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "time-to-1e-6 rel. residual (s) & iterations; stencil GB/s vs HBM peak, 1×GB300"
WORKLOAD = "submarine3d-128"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-iters", type=int, default=4, help="oracle iterations in the CPU sample")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def reference_iterations(name):
    try:
        return json.load(open(os.path.join(ROOT, "oracle", "reference_counts.json")))[name]["iterations"]
    except Exception:
        return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: the system temporary
        # directory); the JSON line carries their summary
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(float(r[2]) for r in rows if len(r) >= 9)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for i, nm in enumerate(names):
            if any(len(r) >= 9 and "Active" in r[5 + i] and "Not" not in r[5 + i] for r in rows):
                out["reasons"].append(nm)
        out["samples"] = len(rows)
        return out


# ------------------------------------------------------------- CPU oracle
def oracle_sample(w, sc, n_iter):
    """Time the oracle's own hybrid-preconditioned BiCGStab for n_iter iterations."""
    from oracle import assemble, krylov, tb  # test/bench infrastructure only
    A, b, _ = assemble.problem(sc)
    t0 = time.perf_counter()
    X = scenes.node_coords(sc.dim, sc.n)
    s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=w["tau"])
    M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(sc.dim, sc.n))
    t1 = time.perf_counter()
    x0 = np.zeros_like(b)
    t2 = time.perf_counter()
    krylov.bicgstab(A, b, x0, M, 1e-300, n_iter)
    t3 = time.perf_counter()
    return {"setup_s": t1 - t0, "per_iter_s": (t3 - t2) / n_iter, "kept": len(s.kept)}


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = scenes.BENCH_WORKLOADS[args.workload]
    iters = reference_iterations(args.workload)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle's own iteration count for "
                          f"{args.workload} is not stored (python -m oracle.reference_data {args.workload})"}),
              flush=True)
        return
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    from oracle import assemble, krylov, tb
    A, b, _ = assemble.problem(sc)
    X = scenes.node_coords(sc.dim, sc.n)
    t0 = time.perf_counter()
    s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=w["tau"])
    M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(sc.dim, sc.n))
    setup_s = time.perf_counter() - t0
    per = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        krylov.bicgstab(A, b, np.zeros_like(b), M, 1e-300, 1)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            per.append(dt)
    per_iter = statistics.mean(per)
    value = per_iter * iters if iters else None
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene, seeded trunk weights)",
        "config": workload_config(args.workload, w, sc, len(s.kept)),
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"oracle FP64 DeepONet-BiCGStab on the same workload, one iteration per step "
                                   f"timed ({per_iter:.3f} s/iteration), scaled by the oracle's own {iters} "
                                   f"iterations to tol={w['tol']:g} (oracle/reference_counts.json); oracle setup "
                                   f"({setup_s:.1f} s) excluded; scipy.sparse matvecs single-threaded"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SCENE_TEXT = {
    "cube3d": ("centred 16^3-node cube", "Gaussian sigma=0.04 at a seeded point", "[3,128,128,128] seeded"),
    "submarine3d": ("submarine: ellipsoid hull 0.35/0.06/0.06, sail, four fins, seeded rotation",
                    "plane wave in a seeded direction (scattered-field solve)", "[3,256,256,256] seeded"),
}


def workload_config(name, w, sc, kept):
    scat, src, trunk = SCENE_TEXT[w["scene"]]
    cfg = {"workload": name, "grid": f"{sc.n}^{sc.dim}", "k0": sc.k0, "layer_cells": sc.layer_cells,
           "scatterer": scat, "source": src, "trunk": trunk,
           "p": sc.p, "kept": kept, "tau": w["tau"], "method": w["method"], "relax": w["relax"],
           "n_r": w["n_r"], "correction": w["correction"], "tol": w["tol"],
           "precision": w.get("precision", "fp64"),
           "l2": "256 MiB buffer written between steps (L2 is 129 MB)"}
    if w["method"] == "bicgstab" and w.get("precision") == "mixed":
        cfg["outer_method_note"] = ("BiCGStab with 3 red-black sweeps per cycle: restarted FGMRES(50) stagnates "
                                    "near 1e-5 on this cavity with a seeded trunk")
    return cfg


# ------------------------------------------------------------------ GPU arm
def source_hash(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_for(workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of the
    workload, if the kernel's source file is unchanged since the capture (else None)."""
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", f"traffic_{workload}.json")))
        e = prof["kernels"][kernel]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2405_12380_gb300", "csrc", e["source"])
    if e.get("sha256_16") != source_hash(src):
        return None
    return e.get("dram_bytes_per_launch")


def stencil_bench(hm, torch, n=256, reps=20):
    """Achieved HBM bandwidth of the operator kernel y = A x on an n^3 grid (vectors
    larger than L2, inputs rotated over three buffers), complex64 and complex128.
    Algorithmic bytes per node: read x once, write y, read one mask byte
    (17 B complex64, 33 B complex128)."""
    sc = scenes.cube3d(0, n=n, width=n // 4, p=8, trunk_widths=(3, 8, 8, 8))
    P = hm.Problem(3, n, 16.0, sc.mask, layer_cells=8, layer_strength=0.5)
    out = {"grid": f"{n}^3"}
    for dt, nbytes in ((torch.complex64, 17), (torch.complex128, 33)):
        xs = [torch.randn(P.N, dtype=dt, device="cuda") for _ in range(3)]
        y = torch.empty_like(xs[0])
        for q in range(3):
            P.apply(xs[q], out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in range(reps):
            P.apply(xs[q % 3], out=y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes * P.N / (ms * 1e-3) / 1e9
        key = "c64" if dt == torch.complex64 else "c128"
        out[key] = {"us_per_apply": ms * 1e3, "GBps": gbs, "bytes_per_node": nbytes}
        del xs, y
    # complex64 sweeps: per full sweep read x and f, write x, two table bytes (26 B per node)
    f = torch.randn(P.N, dtype=torch.complex64, device="cuda")
    x = torch.randn(P.N, dtype=torch.complex64, device="cuda")
    for kind, sweeps in (("jacobi", 2), ("rbgs", 1)):
        P.relax(kind, f, x, sweeps=sweeps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in range(reps):
            P.relax(kind, f, x, sweeps=sweeps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps / sweeps
        out[f"{kind}_c64"] = {"us_per_sweep": ms * 1e3, "GBps": 26 * P.N / (ms * 1e-3) / 1e9, "bytes_per_node": 26}
    del f, x
    hbm = peaks().get("hbm_gbs") or 6800.0
    out["hbm_peak_GBps"] = hbm
    out["jacobi_c64_frac_of_hbm"] = out["jacobi_c64"]["GBps"] / hbm
    out["rbgs_c64_frac_of_hbm"] = out["rbgs_c64"]["GBps"] / hbm
    out["c64_frac_of_hbm"] = out["c64"]["GBps"] / hbm
    out["c128_frac_of_hbm"] = out["c128"]["GBps"] / hbm
    out["note"] = "c128 is bound by GB300's FP64 rate (~18 FP64 operations per node), not by HBM"
    P.close()
    torch.cuda.empty_cache()
    return out


def max_over_ranks(value, world, device="cuda"):
    """The largest value over the ranks of the job (the timing rule of multi-GPU
    runs: the slowest replica sets the time); the value itself on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_entries(w, st_prof, N, k, hbm, hbm_src, workload):
    """Per-kernel achieved HBM bandwidth of the profiled solve: algorithmic bytes
    per launch over the mean CUDA-event duration.  Mixed handles, per node:
    restriction k + 26 B (red-row residual: v and z in, 2 table bytes, the red
    residual out and in again; BF16 Q_red k B), prolongation 2k + 16 B (BF16 Q,
    z in and out), fused red-black sweep 26 B from x (x and f in, x out, 2 table
    bytes) and 18 B from zero, operator with the fused BiCGStab reduction 26 B (x and
    the dot operand in, y out, 2 table bytes).  FP64 handles: FP32-pair basis 8k B
    per row."""
    mixed = w.get("precision") == "mixed"
    out = []

    def add(name, kernel, n_key, ms_key, bytes_per_launch, what):
        n = st_prof[n_key]
        ms = st_prof[ms_key]
        if not n:
            return
        avg = ms / 1e3 / n
        out.append({"bound": "hbm", "kernel": kernel, "what": what, "achieved": bytes_per_launch / avg / 1e9,
                    "peak": hbm, "unit": "GB/s", "frac": bytes_per_launch / avg / 1e9 / hbm,
                    "peak_source": hbm_src, "traffic": traffic_for(workload, kernel),
                    "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_us": avg * 1e6,
                    "launches": n, "share_of_solve": ms / st_prof["ms"],
                    "timing": "CUDA events around every launch, one profiled solve after the timed solves"})

    if mixed:
        add("restrict", "k_march_c64<2> + k_restrict32_rr", "n_restrict", "restrict_ms", (k + 26.0) * N,
            "c = Q_red^T (v - A z) on the red rows: red residual, then BF16 tall-skinny product")
        add("prolong", "k_prolong32v", "n_prolong", "prolong_ms", (2.0 * k + 16.0) * N, "z += Q y, BF16 Q")
        nr = max(1, w["n_r"])
        add("sweep", "k_sweep_c64", "n_sweep", "sweep_ms", (18.0 + 26.0 * (nr - 1)) / nr * N,
            "complex64 red-black full sweep (one launch), the first of each cycle from zero")
        add("apply", "k_march_c64<0,DOT>", "n_apply", "apply_ms", 26.0 * N,
            "complex64 y = A x with the BiCGStab reduction (alpha or omega) in its epilogue")
    else:
        M = (N + 1) // 2
        add("restrict", "k_project_df", "n_restrict", "restrict_ms", (8.0 * k + 16.0) * M,
            "c = Q^T r on the red rows, FP32-pair Q")
        add("prolong", "k_prolong_df", "n_prolong", "prolong_ms", (8.0 * k + 32.0) * N, "z += Q y, FP32-pair Q")
        # the cooperative double-float cycle: BiCGStab input update (56 B), first
        # red half-sweep, 2 n_r - 1 half-sweeps (24.5 B each over all nodes: f,
        # x in/out of one colour, neighbour reads, two table bytes) and the
        # red-row residual (40 B)
        add("sweep", "k_cycle_df", "n_sweep", "sweep_ms", (56.0 + (2 * w["n_r"]) * 24.5 + 40.0) * N,
            "double-float red-black cycle, one cooperative launch")
        add("apply", "k_apply_bicg_df", "n_apply", "apply_ms", 50.0 * N,
            "A x from FP32 pairs (16 B), y FP64 (16 B), dot operand (16 B), two table bytes")
    return out


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2405_12380_gb300 as hm

    w = scenes.BENCH_WORKLOADS[args.workload]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    prec = w.get("precision", "fp64")

    def make_problem(precision):
        P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells,
                       layer_strength=sc.layer_strength, precision=precision)
        # right-hand side built on the device by the library (helm_rhs), from seeded data
        f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = P.don_load(sc.trunk, sc.p, tau=w["tau"])
        torch.cuda.synchronize()
        return P, f, k, time.perf_counter() - t0

    P, f, k, setup_s = make_problem(prec)
    o = hm.opts(w["method"], w["relax"], w["n_r"], correction=w["correction"], tol=w["tol"],
                restart=w["restart"], maxit=w["maxit"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        x, st = P.solve(f, None, o)
    stats = []
    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            x, st = P.solve(f, None, o)
            stats.append(st)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    # per-kernel durations: one more solve of the same workload with an event pair
    # around every launch of the kernels of interest (kept out of the timed solves,
    # whose time the event records would lengthen)
    flush.fill_(1.0)
    P.set_profiling(True)
    _, st_prof = P.solve(f, None, o)
    P.set_profiling(False)
    solve_ms = [s["ms"] for s in stats]
    mean_ms = max_over_ranks(statistics.mean(solve_ms), world)
    # e2e: the same solve through helm_solve_host with pinned host buffers
    fh = f.cpu().pin_memory()
    f_np = fh.numpy()
    xh = torch.zeros(P.N, dtype=torch.complex128).pin_memory()
    x_np = xh.numpy()
    e2e = []
    for step in range(args.warmup + args.steps):
        x_np[:] = 0
        flush.fill_(1.0)
        barrier()
        t1 = time.perf_counter()
        P.solve_host(f_np, x_np, o)
        dt = time.perf_counter() - t1
        if step >= args.warmup:
            e2e.append(dt)
    e2e_s = max_over_ranks(statistics.mean(e2e), world)
    # the converged solution: FP64 residual (library op) and error on the oracle's
    # stored reference sample
    r, nrm = P.residual(f, x)
    rel_res = float(nrm.sqrt().item() / torch.linalg.vector_norm(f).item())
    err = solution_error(args.workload, x)
    extra = {}
    if prec == "mixed":
        # the same inputs on an FP64 handle (the comparison of the mixed form)
        x64 = None
        P64, f64, k64, setup64 = make_problem("fp64")
        x64, _ = P64.solve(f64, None, o)
        t64 = []
        for _ in range(max(1, min(2, args.steps))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            x64, st64 = P64.solve(f64, None, o)
            t64.append(st64)
        extra["fp64_same_inputs"] = {
            "value": statistics.mean(s["ms"] for s in t64) / 1e3, "unit": "s",
            "iterations": statistics.mean(s["iters"] for s in t64), "status": t64[-1]["status_name"],
            "rel_res": t64[-1]["rel_res"], "setup_s": setup64, "kept": k64,
            "error_vs_oracle": solution_error(args.workload, x64),
            "speedup_of_mixed": statistics.mean(s["ms"] for s in t64) / mean_ms,
            "mixed_vs_fp64_rel_l2": float(torch.linalg.vector_norm(x - x64).item()
                                          / torch.linalg.vector_norm(x64).item())}
        P64.close()
        del P64, f64, x64
        torch.cuda.empty_cache()
    if args.workload != "cube3d-64":
        extra["cube3d-64"] = second_entry(hm, torch, flush)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    st0 = stats[-1]
    iters = statistics.mean(s["iters"] for s in stats)
    N = P.N
    hbm = peaks().get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if peaks().get("hbm_gbs") else "fallback"
    kernels = kernel_entries(w, st_prof, N, k, hbm, hbm_src, args.workload)
    roofline = max(kernels, key=lambda e: e["share_of_solve"]) if kernels else None
    cpu = None
    if world == 1 or args.gpus == 1:
        iters_ref = reference_iterations(args.workload)
        smp = oracle_sample(w, sc, args.cpu_iters)
        cpu_value = smp["per_iter_s"] * (iters_ref or iters)
        cpu = {"value": cpu_value, "unit": "s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"oracle FP64 DeepONet-BiCGStab (scipy CSR, numpy Q) on the same workload, "
                         f"{args.cpu_iters} iterations timed ({smp['per_iter_s']:.3f} s/iteration), scaled by "
                         + (f"the oracle's own {iters_ref} iterations to tol (oracle/reference_counts.json)"
                            if iters_ref else f"the GPU solve's {iters} iterations")
                         + f"; oracle setup {smp['setup_s']:.1f} s excluded; scipy.sparse single-threaded",
               "oracle_kept": smp["kept"]}
    clocks = clk.summary()
    stencil = stencil_bench(hm, torch)
    cfg = workload_config(args.workload, w, sc, k)
    cfg.update({"iterations": iters, "rel_res": rel_res, "setup_s": setup_s, "replicas": world,
                "solve_ms_each": solve_ms, "reliable_updates": "delta 0.1" if prec == "mixed" else None})
    line = {
        "metric": METRIC, "value": mean_ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/bf16 (FP64 iterate)" if prec == "mixed" else "f64",
        "data": "synthetic (seeded scene, seeded trunk weights)",
        "config": cfg, "iterations": iters, "status": st0["status_name"],
        "error_vs_oracle": err,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 2 * N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "roofline": roofline, "kernels": kernels, "extra": extra, "stencil": stencil, "cpu_baseline": cpu,
        "clocks": clocks, "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def solution_error(workload, x):
    """Relative L2 error of x on the oracle's stored reference sample (nodes drawn
    by oracle/reference_data.py), or None if the sample is missing."""
    try:
        gold = np.load(os.path.join(ROOT, "tests", "golden", f"solution_{workload}.npz"))
    except Exception:
        return None
    import torch
    idx = torch.from_numpy(gold["idx"]).to(x.device)
    xs = x[idx].cpu().numpy()
    ref = gold["x"]
    return {"rel_l2_on_sample": float(np.linalg.norm(xs - ref) / np.linalg.norm(ref)),
            "sample_nodes": int(len(ref)), "oracle_rel_res": float(gold["rel_res"])}


def second_entry(hm, torch, flush):
    """The 64^3 FP64 workload (cube3d-64: DeepONet-BiCGStab, 3 red-black sweeps, tol
    1e-8): mean of three solves after one warm-up."""
    w = scenes.BENCH_WORKLOADS["cube3d-64"]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
    k = P.don_load(sc.trunk, sc.p, tau=w["tau"])
    o = hm.opts(w["method"], w["relax"], w["n_r"], correction=w["correction"], tol=w["tol"],
                restart=w["restart"], maxit=w["maxit"])
    P.solve(f, None, o)
    sts = []
    for _ in range(3):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        x, st = P.solve(f, None, o)
        sts.append(st)
    out = {"value": statistics.mean(s["ms"] for s in sts) / 1e3, "unit": "s", "tol": w["tol"],
           "precision": "fp64", "iterations": statistics.mean(s["iters"] for s in sts), "kept": k,
           "status": sts[-1]["status_name"], "rel_res": sts[-1]["rel_res"],
           "error_vs_oracle": solution_error("cube3d-64", x), "config": workload_config("cube3d-64", w, sc, k)}
    P.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
