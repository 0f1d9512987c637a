"""SOR / SSOR relaxations and the DeepONet-MG preconditioner (Sec. 3.1.1, Sec. 4.3)
on the GPU against the oracle (oracle/relax.py, oracle/mg.py):

* helm_relax with HELM_SOR and HELM_SSOR (omega = 1.3), complex128 to 1e-12 and
  complex64 to 2e-5, on 2D and on odd and even 3D grids (both complex64 kernel
  families).
* The SOR hybrid cycle as BiCGStab's preconditioner, same iterate as the oracle.
* The V-cycle with and without the trunk-basis step of the 2-1-2 smoother against
  the oracle's V-cycle to 1e-10 (3D 33^3 with three levels, 2D 65^2 with four).
* MG- and DeepONet-MG-preconditioned FGMRES and BiCGStab reach the direct LU
  solution; the iteration counts are reported.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, krylov, mg, relax, tb
from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dim,n", [(2, 45), (3, 37), (3, 36)])
@pytest.mark.parametrize("kind", ["sor", "ssor"])
def test_sor_ssor_sweeps_match_oracle(dim, n, kind):
    s = small_scene(dim, n)
    P = problem_for(s)
    col = assemble.colour(dim, n)
    x0 = s["rng"].standard_normal(n ** dim) + 1j * s["rng"].standard_normal(n ** dim)
    f = s["b"]
    ref = (relax.sor if kind == "sor" else relax.ssor)(s["A"], f, x0, col, 1.3, 2)
    x = P.relax(kind, to_dev(f), to_dev(x0), sweeps=2, omega=1.3).cpu().numpy()
    assert rel(x, ref) < 1e-12, rel(x, ref)
    x32 = P.relax(kind, to_dev(f, torch.complex64), to_dev(x0, torch.complex64), sweeps=2, omega=1.3)
    assert rel(x32.cpu().numpy(), ref) < 2e-5, rel(x32.cpu().numpy(), ref)


def _tb_problem(s, widths, tau=1e-3, seed=3):
    layers = scenes.glorot_mlp(np.random.default_rng(seed), list(widths))
    P = problem_for(s)
    p = widths[-1]
    P.don_load(layers, p, tau=tau)
    so = tb.tb_setup(s["A"], layers, scenes.node_coords(s["dim"], s["n"]), s["mask"], p, tau=tau)
    assert P.kept == so.kept
    return P, so


def test_sor_cycle_bicgstab_same_iterate():
    import paper_2405_12380_gb300 as hm
    s = small_scene(3, 21)
    P, so = _tb_problem(s, [3, 32, 32, 16])
    M = tb.hybrid_preconditioner(s["A"], None, "none", 0)
    col = assemble.colour(3, 21)

    def Msor(r):
        z = relax.sor(s["A"], r, np.zeros_like(r), col, 1.2, 2)
        return z + tb.tb_correct(so, r - s["A"] @ z)
    for it in (1, 3):
        x, st = P.solve(to_dev(s["b"]), None, hm.opts("bicgstab", "sor", 2, omega=1.2, tol=1e-300, maxit=it))
        xo, _ = krylov.bicgstab(s["A"], s["b"], np.zeros_like(s["b"]), Msor, 1e-300, it)
        assert rel(x.cpu().numpy(), xo) < 1e-10, (it, rel(x.cpu().numpy(), xo))


@pytest.mark.parametrize("dim,n,levels,with_tb", [(3, 33, 3, False), (3, 33, 3, True), (2, 65, 4, False),
                                                  (2, 65, 4, True)])
def test_vcycle_matches_oracle(dim, n, levels, with_tb):
    import paper_2405_12380_gb300 as hm
    s = small_scene(dim, n, k0=6.0)
    if with_tb:
        P, so = _tb_problem(s, [dim, 32, 32, 16])
    else:
        P, so = problem_for(s), None
    P.mg_setup(levels)
    k2 = assemble.k2_field(dim, n, s["k0"], s["cells"], 0.5)
    lv = mg.hierarchy(dim, n, k2, s["mask"], levels)
    r = s["rng"].standard_normal(n ** dim) + 1j * s["rng"].standard_normal(n ** dim)
    for conj in (0, 1):
        o = hm.opts("fgmres", "mg", 2, omega=0.6, correction="tb" if with_tb else "none", conj=conj)
        z = P.precond(to_dev(r), o).cpu().numpy()
        if conj:
            lvc = [mg.Level(n=l.n, A=l.A.conj().tocsr(), mask=l.mask, P=l.P, R=l.R) for l in lv]
            soc = None if so is None else tb.TBSetup(Q=so.Q, Ac=so.Ac.conj(), lu=sla.lu_factor(so.Ac.conj()),
                                                     kept=so.kept)
            ref = mg.vcycle(lvc, r, 0.6, 2, soc)
        else:
            ref = mg.vcycle(lv, r, 0.6, 2, so)
        assert rel(z, ref) < 1e-10, (conj, rel(z, ref))


def test_mg_krylov_reaches_lu_solution():
    import paper_2405_12380_gb300 as hm
    s = small_scene(3, 33, k0=6.0)
    P, so = _tb_problem(s, [3, 32, 32, 16])
    P.mg_setup(3)
    u = spla.spsolve(s["A"].tocsc(), s["b"])
    f = to_dev(s["b"])
    counts = {}
    for method in ("fgmres", "bicgstab"):
        for corr in ("none", "tb"):
            x, st = P.solve(f, None, hm.opts(method, "mg", 2, omega=0.6, correction=corr, tol=1e-9, restart=30,
                                              maxit=3000))
            assert st["status"] == 0, (method, corr, st["status_name"])
            assert rel(x.cpu().numpy(), u) < 1e-6
            counts[(method, corr)] = st["iters"]
    print("MG / DeepONet-MG iterations:", counts)
