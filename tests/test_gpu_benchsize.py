"""Parity at the sizes of the workloads, in the launch configurations the bench
times, against the oracle:

* cube3d-64 (64^3 FP64, DeepONet-BiCGStab with 3 red-black sweeps and the trunk
  basis, tol 1e-8): the path is the cooperative double-float cycle with the
  BiCGStab updates fused into its first phase (152 blocks of 1024 threads over
  262,144 nodes, so every grid-stride loop takes a second trip), the operator on
  the cycle's FP32-pair output and the red-row projection.  Iterates 1 and 2
  agree element by element with the oracle's BiCGStab to 1e-10 with a trunk basis
  selected at tau = 1e-3; at the workload's tau = 1e-6 the kept columns are so
  nearly dependent that the orthonormal basis itself is determined only to ~1e-9
  by FP64 data (two correct orthonormalisations differ by that much), so there the
  iterates are held to 1e-8 and the kept columns must be identical; the converged
  solution is compared with the oracle's solution to 1e-10 on its stored node
  sample (tests/golden/solution_cube3d-64.npz, written by
  oracle/reference_data.py): its error must be within ten times the error of the
  oracle's own iterate at the same tolerance.
* square2d-64 (64^2 FP64, k = 10, the 2D configuration): DeepONet-Jacobi with 20
  damped-Jacobi sweeps per trunk-basis correction (two cycles: the seeded trunk
  does not make this relaxation converge, in the oracle either) and
  DeepONet-FGMRES(30) after 5 and 20 Arnoldi steps, to 1e-10 (trunk basis at
  tau = 1e-3, for the reason above); FGMRES with the configuration's basis
  (tau = 1e-6) solved to 1e-8 against the direct LU solution, within ten times
  the oracle FGMRES's own error at that tolerance.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, krylov, tb
from tests.gpu_common import need_gpu, rel, to_dev, torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _workload(name):
    w = scenes.BENCH_WORKLOADS[name]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    return w, sc


def _device_problem(sc, w, precision="fp64", tau=None):
    import paper_2405_12380_gb300 as hm
    P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength,
                   precision=precision)
    f = P.rhs(to_dev(sc.src), to_dev(sc.g))
    P.don_load(sc.trunk, sc.p, tau=w["tau"] if tau is None else tau)
    return P, f


def test_cube64_bench_path_iterates_and_solution():
    import paper_2405_12380_gb300 as hm
    w, sc = _workload("cube3d-64")
    A, b, _ = assemble.problem(sc)
    X = scenes.node_coords(3, sc.n)
    for tau, tol_it in ((1e-3, 1e-10), (w["tau"], 1e-8)):
        P, f = _device_problem(sc, w, tau=tau)
        assert np.allclose(f.cpu().numpy(), b, rtol=0, atol=1e-12 * np.abs(b).max())
        s = tb.tb_setup(A, sc.trunk, X, sc.mask, sc.p, tau=tau)
        assert P.kept == s.kept
        M = tb.hybrid_preconditioner(A, s, w["relax"], w["n_r"], colours=assemble.colour(3, sc.n))
        for it in (1, 2):
            x, st = P.solve(f, None, hm.opts(w["method"], w["relax"], w["n_r"], correction="tb", tol=1e-300,
                                              maxit=it))
            assert st["iters"] == it
            xo, io = krylov.bicgstab(A, b, np.zeros_like(b), M, 1e-300, it)
            assert rel(x.cpu().numpy(), xo) < tol_it, (tau, it, rel(x.cpu().numpy(), xo))
    x, st = P.solve(f, None, hm.opts(w["method"], w["relax"], w["n_r"], correction="tb", tol=w["tol"],
                                      maxit=w["maxit"]))
    assert st["status"] == 0, st["status_name"]
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) <= 1.0001 * w["tol"] * np.linalg.norm(b)
    gold = np.load(os.path.join(HERE, "golden", "solution_cube3d-64.npz"))
    idx = gold["idx"]
    err = rel(xh[idx], gold["x"])
    err_oracle = rel(gold["x_tol"], gold["x"])
    assert err <= 10 * err_oracle, (err, err_oracle)


def test_square64_config1_relaxation_and_fgmres():
    import paper_2405_12380_gb300 as hm
    sc = scenes.square2d(0)
    A, b, _ = assemble.problem(sc)
    P = hm.Problem(2, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    f = P.rhs(to_dev(sc.src), to_dev(sc.g))
    assert np.allclose(f.cpu().numpy(), b, rtol=0, atol=1e-12 * np.abs(b).max())
    P.don_load(sc.trunk, sc.p, tau=1e-3)
    s = tb.tb_setup(A, sc.trunk, scenes.node_coords(2, sc.n), sc.mask, sc.p, tau=1e-3)
    assert P.kept == s.kept
    # DeepONet-Jacobi: 20 damped-Jacobi sweeps (omega = 0.6) per trunk-basis correction
    x, st = P.solve(f, None, hm.opts("relax", "jacobi", 20, omega=0.6, correction="tb", tol=1e-300, maxit=2))
    xo, io = krylov.relaxation_metasolver(A, b, np.zeros_like(b), "jacobi", 20, lambda r: tb.tb_correct(s, r),
                                          omega=0.6, tol=1e-300, max_cycles=2)
    assert st["iters"] == io["iters"] == 2
    assert rel(x.cpu().numpy(), xo) < 1e-10
    # DeepONet-FGMRES(30): one damped-Jacobi sweep + correction per preconditioner application
    M = tb.hybrid_preconditioner(A, s, "jacobi", 1)
    for it in (5, 20):
        x, st = P.solve(f, None, hm.opts("fgmres", "jacobi", 1, correction="tb", tol=1e-300, restart=30, maxit=it))
        xo, io = krylov.fgmres(A, b, np.zeros_like(b), M, 1e-300, 30, it)
        assert rel(x.cpu().numpy(), xo) < 1e-10, (it, rel(x.cpu().numpy(), xo))
    # the configuration's basis for the converged solve
    P.don_load(sc.trunk, sc.p, tau=1e-6)
    s = tb.tb_setup(A, sc.trunk, scenes.node_coords(2, sc.n), sc.mask, sc.p, tau=1e-6)
    assert P.kept == s.kept
    M = tb.hybrid_preconditioner(A, s, "jacobi", 1)
    x, st = P.solve(f, None, hm.opts("fgmres", "jacobi", 1, correction="tb", tol=1e-8, restart=30, maxit=20000))
    assert st["status"] == 0, st["status_name"]
    u = spla.spsolve(A.tocsc(), b)
    xo, io = krylov.fgmres(A, b, np.zeros_like(b), M, 1e-8, 30, 20000)
    assert io["status"] == "converged"
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) <= 1.0001e-8 * np.linalg.norm(b)
    assert rel(xh, u) <= 10 * rel(xo, u), (rel(xh, u), rel(xo, u))
    assert abs(st["iters"] - io["iters"]) <= max(5, 0.15 * io["iters"])
