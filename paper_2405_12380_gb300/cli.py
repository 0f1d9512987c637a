"""Command-line runner: set up a named workload and solve it on cuda:0.

    python -m paper_2405_12380_gb300.cli --workload cube3d-64 [--maxit M] [--solves S]

Prints one JSON line per solve with the library's statistics.  Used to drive
profiler captures of a bounded number of iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube3d-64")
    ap.add_argument("--maxit", type=int, default=None)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--stencil", type=int, default=0, help="time y = A x on an n^3 grid instead of solving")
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    if a.stencil:
        return stencil(a.stencil, a.reps)
    w = dict(scenes.BENCH_WORKLOADS[a.workload])
    if a.maxit is not None:
        w["maxit"] = a.maxit
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    torch.cuda.set_device(0)
    P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
    k = P.don_load(sc.trunk, sc.p, tau=w["tau"]) if w["correction"] == "tb" else 0
    o = hm.opts(w["method"], w["relax"], w["n_r"], correction=w["correction"], tol=w["tol"],
                restart=w["restart"], maxit=w["maxit"])
    for _ in range(a.solves):
        x, st = P.solve(f, None, o)
        st.pop("hist", None)
        st["kept"] = k
        print(json.dumps(st), flush=True)


def stencil(n, reps):
    """Operator throughput: y = A x on n^3 (complex64 and complex128), one JSON line each."""
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm
    torch.cuda.set_device(0)
    mask = (scenes.ring_mask(3, n) | scenes.box_mask(3, n, *scenes.centred_box_nodes(n, n // 4)))
    P = hm.Problem(3, n, 16.0, mask.reshape(-1).astype("uint8"), layer_cells=8, layer_strength=0.5)
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
        print(json.dumps({"dtype": str(dt), "n": n, "us": ms * 1e3, "GBps": nbytes * P.N / (ms * 1e-3) / 1e9}))


if __name__ == "__main__":
    main()
