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
    a = ap.parse_args(argv)
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


if __name__ == "__main__":
    main()
