"""The paper's boundary-value problem on the GPU (helm_create_bvp: Sommerfeld
condition on the outer faces, Neumann incoming wave on the top face, Dirichlet
scatterer, Eq. 1) against the oracle (oracle/bvp.py):

* operator, residual and right-hand side element by element (2D, odd and even
  3D, with and without the Neumann face, conj for the adjoint);
* damped-Jacobi and red-black Gauss-Seidel sweeps;
* the paper's 2D setting (square scatterer, g = sin(3 pi x) on the top face,
  k = 6): DeepONet-BiCGStab and DeepONet-FGMRES with the trunk basis reach the
  direct LU solution; same iterate as the oracle's BiCGStab for two iterations;
* a 3D cube scatterer under a top-face incoming wave, BiCGStab to 1e-8 against
  the oracle's FP64 residual.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, bvp, krylov, relax, tb
from tests.gpu_common import need_gpu, rel, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _bvp_scene(dim, n, k0=6.0, top=True, seed=0):
    rng = np.random.default_rng(seed)
    lo, hi = scenes.centred_box_nodes(n, max(2, n // 5))
    mask = scenes.box_mask(dim, n, lo, hi).reshape(-1).astype(np.uint8)
    N = n ** dim
    k2 = np.full(N, k0 * k0, complex)
    A = bvp.assemble_bvp(dim, n, k2, mask, k0, neumann_top=top)
    X = scenes.node_coords(dim, n)
    g = np.zeros(N, complex)
    on_top = np.isclose(X[:, dim - 1], 1.0)
    g[on_top] = np.sin(3 * np.pi * X[on_top, 0])
    src = np.where(mask == 0, 0.1 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)), 0)
    b = bvp.rhs_bvp(dim, n, mask, src, g, neumann_top=top)
    return dict(dim=dim, n=n, k0=k0, mask=mask, A=A, b=b, src=src, g=g, rng=rng, top=top)


def _problem(s):
    import paper_2405_12380_gb300 as hm
    return hm.Problem(s["dim"], s["n"], s["k0"], s["mask"], boundary="sommerfeld", neumann_top=s["top"])


@pytest.mark.parametrize("dim,n,top", [(2, 33, True), (2, 24, False), (3, 17, True), (3, 16, True)])
def test_operator_rhs_and_sweeps_match_oracle(dim, n, top):
    s = _bvp_scene(dim, n, top=top)
    P = _problem(s)
    N = n ** dim
    b = P.rhs(to_dev(s["src"]), to_dev(s["g"])).cpu().numpy()
    assert rel(b, s["b"]) < 1e-13
    x = s["rng"].standard_normal(N) + 1j * s["rng"].standard_normal(N)
    for conj in (0, 1):
        Ac = s["A"].conj() if conj else s["A"]
        y = P.apply(to_dev(x), conj=conj).cpu().numpy()
        assert rel(y, Ac @ x) < 1e-13, rel(y, Ac @ x)
        r, nrm = P.residual(to_dev(s["b"]), to_dev(x), conj=conj)
        ro = s["b"] - Ac @ x
        assert rel(r.cpu().numpy(), ro) < 1e-13
        assert abs(nrm.item() - np.vdot(ro, ro).real) <= 1e-12 * np.vdot(ro, ro).real
    xj = P.relax("jacobi", to_dev(s["b"]), to_dev(x), sweeps=3, omega=0.6).cpu().numpy()
    assert rel(xj, relax.jacobi(s["A"], s["b"], x, 0.6, 3)) < 1e-12
    xr = P.relax("rbgs", to_dev(s["b"]), to_dev(x), sweeps=2).cpu().numpy()
    assert rel(xr, relax.rbgs(s["A"], s["b"], x, assemble.colour(dim, n), 2)) < 1e-12


def test_paper_2d_setting_krylov_metasolvers():
    import paper_2405_12380_gb300 as hm
    s = _bvp_scene(2, 65, k0=6.0, top=True)
    s["src"][:] = 0
    s["b"] = bvp.rhs_bvp(2, 65, s["mask"], s["src"], s["g"], neumann_top=True)
    P = _problem(s)
    layers = scenes.glorot_mlp(np.random.default_rng(4), [2, 32, 32, 16])
    P.don_load(layers, 16, tau=1e-3)
    so = tb.tb_setup(s["A"], layers, scenes.node_coords(2, 65), s["mask"], 16, tau=1e-3)
    assert P.kept == so.kept
    f = P.rhs(to_dev(s["src"]), to_dev(s["g"]))
    u = spla.spsolve(s["A"].tocsc(), s["b"])
    M = tb.hybrid_preconditioner(s["A"], so, "rbgs", 2, colours=assemble.colour(2, 65))
    for it in (1, 2):
        x, st = P.solve(f, None, hm.opts("bicgstab", "rbgs", 2, tol=1e-300, maxit=it))
        xo, _ = krylov.bicgstab(s["A"], s["b"], np.zeros_like(s["b"]), M, 1e-300, it)
        assert rel(x.cpu().numpy(), xo) < 1e-10, (it, rel(x.cpu().numpy(), xo))
    for method in ("bicgstab", "fgmres"):
        x, st = P.solve(f, None, hm.opts(method, "rbgs", 2, tol=1e-10, restart=30, maxit=5000))
        assert st["status"] == 0, (method, st["status_name"])
        assert rel(x.cpu().numpy(), u) < 1e-7


def test_3d_top_incoming_wave_bicgstab():
    import paper_2405_12380_gb300 as hm
    s = _bvp_scene(3, 33, k0=8.0, top=True)
    s["src"][:] = 0
    s["b"] = bvp.rhs_bvp(3, 33, s["mask"], s["src"], s["g"], neumann_top=True)
    P = _problem(s)
    layers = scenes.glorot_mlp(np.random.default_rng(5), [3, 32, 32, 24])
    P.don_load(layers, 24, tau=1e-3)
    f = P.rhs(to_dev(s["src"]), to_dev(s["g"]))
    x, st = P.solve(f, None, hm.opts("bicgstab", "rbgs", 3, tol=1e-8, maxit=5000))
    assert st["status"] == 0, st["status_name"]
    xh = x.cpu().numpy()
    assert np.linalg.norm(s["b"] - s["A"] @ xh) <= 1.0001e-8 * np.linalg.norm(s["b"])
