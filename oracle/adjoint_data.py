"""Receiver data d for the adjoint workload, from the oracle alone.

d = S u0, where u0 solves the unperturbed problem (k^2 from the layer formula,
no bumps) of scenes.bump_cube3d, computed by the oracle's BiCGStab with three
red-black Gauss-Seidel sweeps per iteration to a relative residual of 1e-10,
and S samples the 256 receivers trilinearly.  Writes
tests/golden/adjoint_d_<name>.npz.  Test/bench infrastructure: calls only the oracle
and the input generators.

    python -m oracle.adjoint_data [n]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import scenes  # noqa: E402
from oracle import adjoint, assemble, krylov, tb  # noqa: E402


def make(n: int = 96, seed: int = 0, tol: float = 1e-10):
    sc = scenes.bump_cube3d(seed, n=n)
    k2 = assemble.k2_field(3, n, sc.k0, sc.layer_cells, sc.layer_strength)      # unperturbed
    A = assemble.assemble(3, n, k2, sc.mask)
    b = assemble.rhs(3, n, sc.mask, sc.src, sc.g)
    M = tb.hybrid_preconditioner(A, None, "rbgs", 3, colours=assemble.colour(3, n))
    t0 = time.perf_counter()
    u0, info = krylov.bicgstab(A, b, np.zeros_like(b), M, tol, 20000)
    S = adjoint.trilinear(n, sc.extra["receivers"])
    d = S @ u0
    out = os.path.join(os.path.dirname(HERE), "tests", "golden", f"adjoint_d_bump_cube3d-{n}.npz")
    np.savez(out, d=d, iters=info["iters"], status=info["status"], rel_res=info["res"][-1],
             seconds=time.perf_counter() - t0)
    print(out, info["status"], info["iters"], info["res"][-1], flush=True)
    return d


if __name__ == "__main__":
    make(int(sys.argv[1]) if len(sys.argv) > 1 else 96)
