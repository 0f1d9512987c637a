"""Reference data of the timed workloads from the oracle alone.

For each workload of scenes.BENCH_WORKLOADS this runs the oracle's own
meta-solver (same method, relaxation, n_r and trunk-basis correction, FP64
throughout, x0 = 0) to the workload's tolerance and records its iteration count
(oracle/reference_counts.json: the CPU baseline of bench.py scales the oracle's
measured time per iteration by it), then continues the solve from that iterate
to a relative residual of 1e-10 and stores the solution on a seeded sample of
65536 nodes (tests/golden/solution_<workload>.npz: indices, values, residual),
the reference for the error of the GPU solutions, together with the oracle's
own iterate at the workload's tolerance on the same nodes (the error a correct
solve to that tolerance makes).  Test/bench infrastructure:
calls only the oracle and the input generators.

    python -m oracle.reference_data [workload ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from oracle import assemble, krylov, tb  # noqa: E402

OUT = os.path.join(HERE, "reference_counts.json")
GOLDEN = os.path.join(ROOT, "tests", "golden")
SAMPLE = 65536
SAMPLE_SEED = 12345
REF_TOL = 1e-10


def sample_indices(N: int) -> np.ndarray:
    """The seeded node sample of the stored solutions (sorted flat indices)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(N, size=min(SAMPLE, N), replace=False)).astype(np.int64)


def oracle_solver(w, sc, A):
    X = scenes.node_coords(sc.dim, sc.n)
    s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=w["tau"]) if w["correction"] == "tb" else None
    M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(sc.dim, sc.n))
    return M, s


def _solve(w, A, b, x0, M, tol):
    if w["method"] == "bicgstab":
        return krylov.bicgstab(A, b, x0, M, tol, w["maxit"])
    return krylov.fgmres(A, b, x0, M, tol, w["restart"], w["maxit"])


def run(name: str) -> dict:
    w = scenes.BENCH_WORKLOADS[name]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    A, b, _ = assemble.problem(sc)
    t0 = time.perf_counter()
    M, s = oracle_solver(w, sc, A)
    t1 = time.perf_counter()
    x, info = _solve(w, A, b, np.zeros_like(b), M, w["tol"])
    t2 = time.perf_counter()
    res = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    out = {"iterations": int(info["iters"]), "status": info["status"], "rel_res": res, "tol": w["tol"],
           "kept": len(s.kept) if s is not None else 0, "setup_s": t1 - t0, "solve_s": t2 - t1}
    # continue to the reference tolerance for the stored solution
    xr, info2 = _solve(w, A, b, x, M, REF_TOL)
    res2 = float(np.linalg.norm(b - A @ xr) / np.linalg.norm(b))
    idx = sample_indices(sc.N)
    os.makedirs(GOLDEN, exist_ok=True)
    np.savez_compressed(os.path.join(GOLDEN, f"solution_{name}.npz"), idx=idx, x=xr[idx], rel_res=res2,
                        x_norm=np.linalg.norm(xr), iterations_ref=int(info2["iters"]),
                        x_tol=x[idx], tol=w["tol"], rel_res_tol=res)
    out.update({"ref_tol": REF_TOL, "ref_rel_res": res2, "ref_extra_iterations": int(info2["iters"])})
    return out


if __name__ == "__main__":
    names = sys.argv[1:] or list(scenes.BENCH_WORKLOADS)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for nm in names:
        data[nm] = run(nm)
        print(nm, data[nm], flush=True)
        json.dump(data, open(OUT, "w"), indent=1)
