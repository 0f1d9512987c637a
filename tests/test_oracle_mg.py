"""Pins of the multigrid oracle (oracle/mg.py; Sec. 4.3 DeepONet-MG):

* P reproduces affine functions exactly (bi/trilinear interpolation) and full
  weighting R = P^T / 2^d keeps a constant in the interior.
* A two-level cycle equals its closed form built from dense matrices: m damped
  Jacobi sweeps from zero give (I - S^m) A^-1 r with S = I - omega D^-1 A; the
  coarse-grid correction adds P_m M_c R_m (r - A z) (M_c the coarsest level's own
  smoother from zero, masked coarse rows and masked fine rows dropped); the
  post-smoother maps z to S^m z + (I - S^m) A^-1 r.  Checked with and without the
  trunk-basis step of the 2-1-2 smoother (z += Q A_c^-1 Q^T (r - A z) between two
  Jacobi pairs), so an exchanged order of smoothing and correction, a missing
  mask, or R and P swapped fails.
* On a near-Poisson problem (small k, no layer) the V-cycle makes GMRES converge
  in a number of iterations that barely grows with the grid (33^2 -> 65^2).
"""
import numpy as np
import pytest

import scenes
from oracle import assemble, krylov, mg, tb


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_reproduces_affine_and_full_weighting(dim):
    nc = 5
    n = 2 * nc - 1
    Xc = scenes.node_coords(dim, nc)
    Xf = scenes.node_coords(dim, n)
    coef = np.array([0.3, -1.2, 2.5][:dim])
    fc = 0.7 + Xc @ coef
    ff = 0.7 + Xf @ coef
    P = mg.prolongation(dim, nc)
    assert np.allclose(P @ fc, ff, rtol=0, atol=1e-14)
    R = mg.restriction(dim, nc)
    assert np.allclose(R.toarray(), P.toarray().T / 2 ** dim)
    ones = R @ np.ones(n ** dim)
    interior = np.all((Xc > 0) & (Xc < 1), axis=1)
    assert np.allclose(ones[interior], 1.0, rtol=0, atol=1e-15)


def _jacobi_closed(A, m, omega):
    """(S^m, (I - S^m) A^-1) for m damped-Jacobi sweeps from zero."""
    Ad = A.toarray()
    N = Ad.shape[0]
    S = np.eye(N) - omega * Ad / np.diag(Ad)[:, None]
    Sm = np.linalg.matrix_power(S, m)
    return Sm, (np.eye(N) - Sm) @ np.linalg.inv(Ad)


@pytest.mark.parametrize("dim,n,with_tb", [(2, 9, False), (2, 9, True), (3, 9, False), (3, 9, True)])
def test_two_level_cycle_equals_closed_form(dim, n, with_tb):
    omega, n_r = 0.6, 2
    box = (3, 5) if dim == 2 else (3, 5)
    mask = (scenes.ring_mask(dim, n) | scenes.box_mask(dim, n, *box)).reshape(-1).astype(np.uint8)
    k2 = assemble.k2_field(dim, n, 4.0, 2, 0.5)
    lv = mg.hierarchy(dim, n, k2, mask, 2)
    A, Ac = lv[0].A, lv[1].A
    N = n ** dim
    tbs = None
    if with_tb:
        layers = scenes.glorot_mlp(np.random.default_rng(2), [dim, 8, 6])
        tbs = tb.tb_setup(A, layers, scenes.node_coords(dim, n), mask, 6)
    Ad = A.toarray()
    Ainv = np.linalg.inv(Ad)
    I = np.eye(N)
    m = 2 * n_r + 1
    # coarsest level: its own smoother (m sweeps) from zero
    _, Mc = _jacobi_closed(Ac, m, omega)
    Rm = lv[0].R.toarray()
    Rm[lv[1].mask == 1, :] = 0.0
    Pm = lv[0].P.toarray()
    Pm[lv[0].mask == 1, :] = 0.0
    if with_tb:
        Sn, Gn = _jacobi_closed(A, n_r, omega)
        Q = tbs.Q
        C = Q @ np.linalg.inv(Q.T @ Ad @ Q) @ Q.T
        # smoother z -> S^n (z + C (r - A z)) ... written as affine maps in (z, r)
        def smooth(Z, Rr):
            Z = Sn @ Z + Gn @ Rr
            Z = Z + C @ (Rr - Ad @ Z)
            return Sn @ Z + Gn @ Rr
    else:
        Sm, Gm = _jacobi_closed(A, m, omega)

        def smooth(Z, Rr):
            return Sm @ Z + Gm @ Rr
    Z = smooth(np.zeros((N, N)), I)
    Z = Z + Pm @ Mc @ Rm @ (I - Ad @ Z)
    Mdense = smooth(Z, I)
    rng = np.random.default_rng(1)
    for _ in range(3):
        r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        z = mg.vcycle(lv, r, omega, n_r, tbs)
        assert np.linalg.norm(z - Mdense @ r) <= 1e-12 * np.linalg.norm(Mdense @ r)


def test_mg_gmres_near_mesh_independent_on_poisson_like_problem():
    its = []
    for n in (33, 65):
        mask = (scenes.ring_mask(2, n) | scenes.box_mask(2, n, *scenes.centred_box_nodes(n, n // 5))).reshape(-1)
        mask = mask.astype(np.uint8)
        k2 = assemble.k2_field(2, n, 1.0, 0, 0.0)
        lv = mg.hierarchy(2, n, k2, mask, 4)
        rng = np.random.default_rng(0)
        b = np.where(mask == 0, rng.standard_normal(n * n), 0).astype(complex)
        x, info = krylov.fgmres(lv[0].A, b, np.zeros_like(b), mg.mg_preconditioner(lv), 1e-8, 30, 300)
        assert info["status"] == "converged"
        x0, info0 = krylov.fgmres(lv[0].A, b, np.zeros_like(b), None, 1e-8, 30, 300)
        its.append(info["iters"])
        assert info["iters"] < info0["iters"] / 3
    assert its[1] <= its[0] + 4, its
