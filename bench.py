#!/usr/bin/env python
"""Time-to-tolerance of the DeepONet-BiCGStab meta-solver on one GB300.

Workload (scenes.BENCH_WORKLOADS["cube3d-64"]): 3D FP64 Helmholtz on 64^3 nodes,
k = 16, 8-cell absorbing layer, centred 16^3 sound-soft cube, Gaussian source;
trunk [3,128,128,128] (seeded), natural-order trunk basis (tau = 1e-6);
BiCGStab right-preconditioned by the hybrid cycle (3 red-black GS sweeps, then
the trunk-basis Galerkin correction), tolerance 1e-8 on the true residual.

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
WORKLOAD = "cube3d-64"


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
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    iters = reference_iterations(args.workload)
    from oracle import assemble, krylov, tb
    A, b, _ = assemble.problem(sc)
    X = scenes.node_coords(sc.dim, sc.n)
    s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=w["tau"])
    M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(sc.dim, sc.n))
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
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, w, sc, None),
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"oracle DeepONet-BiCGStab, 1 iteration per step timed, scaled by the "
                                   f"oracle's own {iters} iterations to 1e-8 (oracle/reference_counts.json); "
                                   f"setup excluded; scipy.sparse matvecs single-threaded"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(name, w, sc, kept):
    return {"workload": name, "grid": f"{sc.n}^{sc.dim}", "k0": sc.k0, "layer_cells": sc.layer_cells,
            "scatterer": "centred 16^3 cube", "source": "Gaussian sigma=0.04", "trunk": "[3,128,128,128] seeded",
            "p": sc.p, "kept": kept, "tau": w["tau"], "method": w["method"], "relax": w["relax"],
            "n_r": w["n_r"], "correction": w["correction"], "tol": w["tol"],
            "l2": "256 MiB buffer written between steps (L2 is 129 MB)"}


# ------------------------------------------------------------------ GPU arm
# the trunk-basis projection after red-black Gauss-Seidel reads the red rows only
RED_ONLY_PROJECTION = True


def source_hash(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_for(kernel, k):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's source
    file is unchanged since the capture (else None)."""
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "traffic_cube3d-64.json")))
        e = prof["kernels"][kernel]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2405_12380_gb300", "csrc", e["source"])
    if e.get("sha256_16") != source_hash(src) or prof.get("k") != k:
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
    from paper_2405_12380_gb300 import _lib as L

    w = scenes.BENCH_WORKLOADS[args.workload]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    # right-hand side built on the device by the library (helm_rhs), from seeded data
    P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = P.don_load(sc.trunk, sc.p, tau=w["tau"])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
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
    # check the converged solution with an independent FP64 residual (device, library op)
    r, nrm = P.residual(f, x)
    rel_res = float(nrm.sqrt().item() / torch.linalg.vector_norm(f).item())
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    st0 = stats[-1]
    iters = statistics.mean(s["iters"] for s in stats)
    N = P.N
    M = (N + 1) // 2
    fluid = int(N - int(sc.mask.astype(bool).sum()))
    hbm = peaks().get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks().get("hbm_gbs") else "fallback"
    # FP64 issue peak: 2 FP64 instructions per clock per SM (DADD, DMUL or DFMA), 152 SMs,
    # at the maximum SM clock seen by the clock sampler
    sm_mhz = (clk.summary().get("sm_max_mhz") or 2070.0)
    fp64_peak = 2 * 152 * sm_mhz * 1e6 / 1e12
    red_only = RED_ONLY_PROJECTION and w["relax"] == "rbgs" and w["n_r"] > 0

    def phase(n_key, ms_key):
        n = st_prof[n_key]
        ms = st_prof[ms_key]
        return n, ms, (ms / 1e3 / n if n else None)

    kernels = []
    df_sweep = w["relax"] == "rbgs" and w["n_r"] > 0 and w["correction"] == "tb"
    # trunk-basis projection c = Q^T r: Q as FP32 pairs (8 B per entry), r as 16 B
    # per entry (complex128, or FP32 pairs after the double-float sweeps)
    n_, ms_, avg = phase("n_restrict", "restrict_ms")
    rows = M if red_only else N
    if avg:
        b = 8.0 * k * rows + 16.0 * rows
        kernels.append({"bound": "hbm", "kernel": "k_project_df (Q^T r%s, FP32-pair arithmetic)" % (
                            ", red rows" if red_only else ""),
                        "achieved": b / avg / 1e9, "peak": hbm, "unit": "GB/s", "frac": b / avg / 1e9 / hbm,
                        "peak_source": hbm_src, "traffic": traffic_for("k_project_df", k),
                        "algorithmic_bytes_per_launch": b, "avg_launch_us": avg * 1e6, "launches": n_,
                        "share_of_solve": ms_ / st_prof["ms"]})
    # prolongation z += Q y: all of Q, z read and written
    n_, ms_, avg = phase("n_prolong", "prolong_ms")
    if avg:
        b = 8.0 * k * N + 32.0 * N
        kernels.append({"bound": "hbm", "kernel": "k_prolong_df (z += Q y, FP32-pair arithmetic)",
                        "achieved": b / avg / 1e9, "peak": hbm, "unit": "GB/s", "frac": b / avg / 1e9 / hbm,
                        "peak_source": hbm_src, "traffic": traffic_for("k_prolong_df", k),
                        "algorithmic_bytes_per_launch": b, "avg_launch_us": avg * 1e6, "launches": n_,
                        "share_of_solve": ms_ / st_prof["ms"]})
    # relaxation.  FP64 kernels: per updated fluid node 10 DADD (neighbour sum), 2
    # DFMA (f - h^-2 s), a complex multiply (2 DMUL + 2 DFMA) = 16 FP64 instructions
    # per half-sweep.  The double-float cycle of the trunk-basis correction (one
    # cooperative launch per preconditioner application): per red/black node pair a
    # first red update (complex pair product, 50 FP32 instructions), 2 n_r - 1
    # half-sweeps of 196 (10 pair additions of 11 instructions, 2 pair products of 7
    # for h^-2 s, 2 pair additions for f - h^-2 s, a complex pair product of 50) and
    # the red residual (218)
    n_, ms_, avg = phase("n_sweep", "sweep_ms")
    fp32_peak = 128 * 152 * sm_mhz * 1e6 / 1e12
    if avg and df_sweep:
        ops = (50.0 + (2 * w["n_r"] - 1) * 196.0 + 218.0) * fluid / 2
        kernels.append({"bound": "alu", "kernel": "k_cycle_df (double-float red-black cycle, one cooperative launch)",
                        "achieved": ops / avg / 1e12, "peak": fp32_peak, "unit": "T FP32 inst/s",
                        "frac": ops / avg / 1e12 / fp32_peak,
                        "peak_source": "128 FP32 instructions/clk/SM x 152 SMs x max SM clock",
                        "traffic": traffic_for("k_cycle_df", k), "algorithmic_fp32_inst_per_launch": ops,
                        "avg_launch_us": avg * 1e6,
                        "launches": n_, "share_of_solve": ms_ / st_prof["ms"]})
    elif avg:
        ops = 16.0 * fluid / 2
        kernels.append({"bound": "alu", "kernel": "k_%s (FP64 half-sweep)" % w["relax"],
                        "achieved": ops / avg / 1e12, "peak": fp64_peak, "unit": "T FP64 inst/s",
                        "frac": ops / avg / 1e12 / fp64_peak,
                        "peak_source": "2 FP64 instructions/clk/SM x 152 SMs x max SM clock",
                        "traffic": None, "algorithmic_fp64_inst_per_launch": ops, "avg_launch_us": avg * 1e6,
                        "launches": n_, "share_of_solve": ms_ / st_prof["ms"]})
    # BiCGStab operator with its fused reduction: 16 FP64 instructions for A x per
    # fluid node plus 4 (<rhat, v>) or 6 (<t, s>, <t, t>): 21 on average; on the
    # double-float input (trunk-basis red-black cycle) A x runs on the FP32 pipes and
    # the FP64 part is the conversion of y (4 F2F + 2 DADD) and the dots: 11
    n_, ms_, avg = phase("n_apply", "apply_ms")
    if avg:
        ops = (11.0 if df_sweep else 21.0) * fluid
        kernels.append({"bound": "alu", "kernel": "k_apply_bicg_df (A x in double-float, FP64 y and fused dots)" if df_sweep
                        else "k_apply_bicg (FP64 A x + fused dots)",
                        "achieved": ops / avg / 1e12, "peak": fp64_peak, "unit": "T FP64 inst/s",
                        "frac": ops / avg / 1e12 / fp64_peak,
                        "peak_source": "2 FP64 instructions/clk/SM x 152 SMs x max SM clock",
                        "traffic": traffic_for("k_apply_bicg_df" if df_sweep else "k_apply_bicg", k), "algorithmic_fp64_inst_per_launch": ops, "avg_launch_us": avg * 1e6,
                        "launches": n_, "share_of_solve": ms_ / st_prof["ms"]})
    for e in kernels:
        e["timing"] = "CUDA events around every launch, one profiled solve after the timed solves"
    roofline = max(kernels, key=lambda e: e["share_of_solve"]) if kernels else None
    cpu = None
    if world == 1 or args.gpus == 1:
        iters_ref = reference_iterations(args.workload)
        smp = oracle_sample(w, sc, args.cpu_iters)
        cpu_value = smp["per_iter_s"] * (iters_ref or iters)
        cpu = {"value": cpu_value, "unit": "s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"oracle DeepONet-BiCGStab (scipy CSR, numpy Q), {args.cpu_iters} iterations timed "
                         f"({smp['per_iter_s']:.3f} s/iter), scaled by "
                         + (f"the oracle's own {iters_ref} iterations to tol (oracle/reference_counts.json)"
                            if iters_ref else f"the GPU solve's {iters} iterations")
                         + f"; oracle setup {smp['setup_s']:.1f} s excluded; scipy.sparse single-threaded",
               "oracle_kept": smp["kept"]}
    clocks = clk.summary()
    stencil = stencil_bench(hm, torch)
    cfg = workload_config(args.workload, w, sc, k)
    cfg.update({"iterations": iters, "rel_res": rel_res, "setup_s": setup_s, "replicas": world,
                "solve_ms_each": solve_ms})
    line = {
        "metric": METRIC, "value": mean_ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene, seeded trunk weights)",
        "config": cfg, "iterations": iters, "status": st0["status_name"],
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 2 * N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "roofline": roofline, "kernels": kernels, "stencil": stencil, "cpu_baseline": cpu, "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
