"""Pins of the SOR and SSOR relaxations of the oracle (Sec. 3.1.1 lists SOR and
SSOR beside Jacobi and Gauss-Seidel as relaxation backbones), in red-black order:

* SOR with omega = 1 is red-black Gauss-Seidel.
* SOR is the splitting x' = x + omega (D + omega L)^-1 (f - A x) of the
  red-first permuted matrix (L its strictly lower triangle): textbook form,
  solved with scipy's triangular solver.
* One SSOR sweep from zero is a linear map M f whose matrix is complex symmetric
  when A is (A = A^T with the same red-black ordering for both half-sweeps),
  the property that makes SSOR a symmetric preconditioner.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, relax


def _small(n=11, box=(4, 6), dim=2, k0=9.0, seed=0):
    rng = np.random.default_rng(seed)
    mask = (scenes.ring_mask(dim, n) | scenes.box_mask(dim, n, *box)).reshape(-1).astype(np.uint8)
    A = assemble.assemble(dim, n, assemble.k2_field(dim, n, k0, 3, 0.5), mask)
    src = np.where(mask == 0, rng.standard_normal(n ** dim) + 1j * rng.standard_normal(n ** dim), 0)
    b = assemble.rhs(dim, n, mask, src, np.zeros(n ** dim, complex))
    return A, b, assemble.colour(dim, n), rng


def test_sor_omega_one_is_rbgs():
    A, b, col, rng = _small()
    x0 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    assert np.array_equal(relax.sor(A, b, x0, col, 1.0, 3), relax.rbgs(A, b, x0, col, 3))


def test_sor_is_the_permuted_splitting():
    A, b, col, rng = _small(n=12, box=(4, 7))
    omega = 1.3
    perm = np.concatenate([np.flatnonzero(col == 0), np.flatnonzero(col == 1)])
    P = A[perm][:, perm].tocsr()
    bp = b[perm]
    x0 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    xp = x0[perm].copy()
    D = sp.diags(P.diagonal())
    Lw = (D + omega * sp.tril(P, -1)).tocsr()
    for _ in range(2):
        xp = xp + omega * spla.spsolve_triangular(Lw, bp - P @ xp, lower=True)
    y = relax.sor(A, b, x0, col, omega, 2)
    assert np.linalg.norm(y[perm] - xp) <= 1e-12 * np.linalg.norm(xp)


def test_ssor_preconditioner_is_complex_symmetric():
    A, b, col, rng = _small(n=9, box=(3, 5))
    N = b.size
    omega = 1.2
    M = np.zeros((N, N), complex)
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1.0
        M[:, j] = relax.ssor(A, e, np.zeros(N, complex), col, omega, 1)
    assert np.linalg.norm(M - M.T) <= 1e-13 * np.linalg.norm(M)
    # and SOR (forward only) is not
    S = np.zeros((N, N), complex)
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1.0
        S[:, j] = relax.sor(A, e, np.zeros(N, complex), col, omega, 1)
    assert np.linalg.norm(S - S.T) > 1e-3 * np.linalg.norm(S)
