"""Iteration counts of the oracle's own full solves of the timed workloads.

Test/bench infrastructure: writes oracle/reference_counts.json, which the CPU
baseline of bench.py uses to scale the oracle's measured time per iteration to
a time-to-tolerance (the full oracle solve takes minutes).  Calls only the
oracle and the input generators.

    python -m oracle.reference_counts [workload ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import scenes  # noqa: E402
from oracle import assemble, krylov, tb  # noqa: E402

OUT = os.path.join(HERE, "reference_counts.json")


def oracle_solver(w, sc, A):
    X = scenes.node_coords(sc.dim, sc.n)
    s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=w["tau"]) if w["correction"] == "tb" else None
    M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(sc.dim, sc.n))
    return M, s


def run(name: str) -> dict:
    w = scenes.BENCH_WORKLOADS[name]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    A, b, _ = assemble.problem(sc)
    t0 = time.perf_counter()
    M, s = oracle_solver(w, sc, A)
    t1 = time.perf_counter()
    x0 = np.zeros_like(b)
    if w["method"] == "bicgstab":
        x, info = krylov.bicgstab(A, b, x0, M, w["tol"], w["maxit"])
    else:
        x, info = krylov.fgmres(A, b, x0, M, w["tol"], w["restart"], w["maxit"])
    t2 = time.perf_counter()
    res = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    return {"iterations": int(info["iters"]), "status": info["status"], "rel_res": res,
            "kept": len(s.kept) if s is not None else 0, "setup_s": t1 - t0, "solve_s": t2 - t1}


if __name__ == "__main__":
    names = sys.argv[1:] or list(scenes.BENCH_WORKLOADS)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for nm in names:
        data[nm] = run(nm)
        print(nm, data[nm], flush=True)
        json.dump(data, open(OUT, "w"), indent=1)
