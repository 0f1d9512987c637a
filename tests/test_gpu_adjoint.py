"""Adjoint gradient of the receiver misfit with respect to the per-node k^2:
receiver sampling and its transpose against the oracle's trilinear operator, the
GPU gradient against the oracle's adjoint gradient (direct LU solves) and
against central finite differences of GPU solves, and the complex-symmetry
identity of the conjugate solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import scenes
from oracle import adjoint, assemble
from tests.gpu_common import need_gpu, rel, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _scene(n=21, seed=5):
    rng = np.random.default_rng(seed)
    lo, hi = scenes.centred_box_nodes(n, max(2, n // 5))
    mask = (scenes.ring_mask(3, n) | scenes.box_mask(3, n, lo, hi)).reshape(-1).astype(np.uint8)
    scale = 1.0 + 0.05 * rng.standard_normal(n ** 3)
    k2 = assemble.k2_field(3, n, 7.0, 4, 0.5, scale)
    src = scenes.gaussian_source(3, n, (0.3, 0.35, 0.62), 0.06)
    src[mask == 1] = 0
    b = assemble.rhs(3, n, mask, src.astype(complex), np.zeros(n ** 3, complex))
    rec = scenes.fibonacci_sphere(64, 0.36)
    d = 0.01 * (rng.standard_normal(64) + 1j * rng.standard_normal(64))
    layers = scenes.glorot_mlp(rng, [3, 32, 32, 16])
    return dict(n=n, mask=mask, k2=k2, b=b, rec=rec, d=d, layers=layers, rng=rng)


def _problem(s):
    import paper_2405_12380_gb300 as hm
    P = hm.Problem(3, s["n"], 7.0, s["mask"], layer_cells=4, k2=s["k2"])
    P.don_load(s["layers"], 16, tau=1e-4)
    return P


def test_receiver_sampling_and_transpose():
    s = _scene()
    P = _problem(s)
    S = adjoint.trilinear(s["n"], s["rec"])
    idx, w = P.receivers(s["rec"])
    u = s["rng"].standard_normal(s["n"] ** 3) + 1j * s["rng"].standard_normal(s["n"] ** 3)
    assert rel(P.sample(idx, w, to_dev(u)).cpu().numpy(), S @ u) < 1e-14
    e = s["rng"].standard_normal(64) + 1j * s["rng"].standard_normal(64)
    assert rel(P.sample_adjoint(idx, w, to_dev(e)).cpu().numpy(), S.T @ e) < 1e-14


def test_conjugate_solve_identity():
    """A^H lambda = g equals conj(A^-1 conj(g)) (A complex symmetric)."""
    import paper_2405_12380_gb300 as hm
    s = _scene()
    P = _problem(s)
    g = s["rng"].standard_normal(s["n"] ** 3) + 1j * s["rng"].standard_normal(s["n"] ** 3)
    g[s["mask"] == 1] = 0
    o = hm.opts("fgmres", "rbgs", 1, tol=1e-12, restart=30, maxit=3000)
    oc = hm.opts("fgmres", "rbgs", 1, tol=1e-12, restart=30, maxit=3000, conj=True)
    lam, st1 = P.solve(to_dev(g), None, oc)
    v, st2 = P.solve(to_dev(np.conj(g)), None, o)
    assert st1["status"] == 0 and st2["status"] == 0
    assert rel(lam.cpu().numpy(), np.conj(v.cpu().numpy())) < 1e-9


def _gpu_loss_and_grad(s, P, k2, tol=1e-12):
    import paper_2405_12380_gb300 as hm
    from paper_2405_12380_gb300.autograd import misfit_loss
    o = hm.opts("fgmres", "rbgs", 1, tol=tol, restart=30, maxit=4000)
    idx, w = P.receivers(s["rec"])
    k2t = to_dev(k2).requires_grad_(True)
    L, u = misfit_loss(k2t, to_dev(s["b"]), P, o, idx, w, to_dev(s["d"]))
    L.backward()
    return L.item(), k2t.grad.cpu().numpy(), u.detach().cpu().numpy()


def test_gradient_matches_oracle_adjoint():
    s = _scene()
    P = _problem(s)
    L, g, u = _gpu_loss_and_grad(s, P, s["k2"])
    A = assemble.assemble(3, s["n"], s["k2"], s["mask"])
    S = adjoint.trilinear(s["n"], s["rec"])
    uo = spla.spsolve(A.tocsc(), s["b"])
    go, _ = adjoint.gradient_k2(A, S, uo, s["d"], s["mask"], lambda r: spla.spsolve(A.conj().tocsc(), r))
    assert rel(u, uo) < 1e-9
    assert abs(L - adjoint.loss(S, uo, s["d"])) <= 1e-9 * L
    assert rel(g, go) < 1e-7
    assert np.all(g[s["mask"] == 1] == 0)


def test_gradient_matches_central_differences():
    s = _scene()
    P = _problem(s)
    L, g, u = _gpu_loss_and_grad(s, P, s["k2"])
    fluid = np.flatnonzero(s["mask"] == 0)
    import paper_2405_12380_gb300 as hm
    o = hm.opts("fgmres", "rbgs", 1, tol=1e-13, restart=30, maxit=4000)
    idx, w = P.receivers(s["rec"])
    d = to_dev(s["d"])

    def loss_of(k2):
        P.set_k2(to_dev(k2))
        uu, st = P.solve(to_dev(s["b"]), None, o)
        assert st["status"] == 0
        e = P.sample(idx, w, uu) - d
        return float((e.real ** 2 + e.imag ** 2).sum().item())
    gmax = np.max(np.abs(g))
    for l in s["rng"].choice(fluid, 6, replace=False):
        for unit, part in ((1.0, "re"), (1j, "im")):
            eps = 1e-3 * abs(s["k2"][l])
            kp, km = s["k2"].copy(), s["k2"].copy()
            kp[l] += eps * unit
            km[l] -= eps * unit
            fd = (loss_of(kp) - loss_of(km)) / (2 * eps)
            an = g[l].real if part == "re" else g[l].imag
            assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-2 * gmax), (l, part, fd, an)
