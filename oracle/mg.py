"""Geometric multigrid V-cycle with a DeepONet-Jacobi smoother (Sec. 4.3,
DeepONet-MG-Krylov; the paper compares it with MG using a Jacobi smoother and 5
smoothing steps, and uses the "2-1-2" strategy for the DeepONet smoother: two
relaxation steps, one neural-operator step, two relaxation steps).

Reading of the paper's description (it gives no further detail):
* Levels: vertex-centred coarsening n -> (n + 1) / 2 (n odd), coarse node I at
  fine node 2I, h_c = 2h.  The mask and k^2 of a coarse node are those of the
  fine node 2I (injection; with the layer formula this is the layer of L/2 cells
  for an even L), and the operator is rediscretised on each level (the stencil
  of Eq. 1 with the coarse h).
* Transfer: P is (bi/tri)linear interpolation (tensor product of the 1D
  interpolation [1/2, 1, 1/2]), R = P^T / 2^d (full weighting).  Coarse
  right-hand sides are zero on masked coarse nodes; corrections are not added on
  masked fine nodes.
* Smoother S(r, z): with the trunk basis (finest level only), n_r damped-Jacobi
  sweeps, the trunk-basis correction z += M2 (r - A z) (App. C), n_r sweeps
  (2-1-2 for n_r = 2); without it, 2 n_r + 1 damped-Jacobi sweeps (5 for
  n_r = 2, the same number of steps).
* V-cycle as a preconditioner z = V(r): z = S(r, 0); z += P V_c(R (r - A z));
  z = S(r, z); the coarsest level applies only its smoother from zero.  The
  cycle is linear in r, so it can precondition BiCGStab as well as FGMRES.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import assemble, relax, tb


def interp_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc coarse to 2 nc - 1 fine nodes (1D)."""
    n = 2 * nc - 1
    rows, cols, vals = [], [], []
    for I in range(nc):
        rows.append(2 * I); cols.append(I); vals.append(1.0)
        if I + 1 < nc:
            rows += [2 * I + 1, 2 * I + 1]
            cols += [I, I + 1]
            vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))


def prolongation(dim: int, nc: int) -> sp.csr_matrix:
    """P for flat index i + n (j + n k) (x fastest): kron(P_z, P_y, P_x)."""
    p1 = interp_1d(nc)
    P = p1
    for _ in range(dim - 1):
        P = sp.kron(p1, P)
    return P.tocsr()


def restriction(dim: int, nc: int) -> sp.csr_matrix:
    return (prolongation(dim, nc).T / 2.0 ** dim).tocsr()


def inject(dim: int, n: int, a: np.ndarray) -> np.ndarray:
    """Values at the coarse nodes (fine nodes 2I)."""
    shape = (n,) * dim
    sl = tuple(slice(None, None, 2) for _ in range(dim))
    return np.ascontiguousarray(np.asarray(a).reshape(shape)[sl]).reshape(-1)


@dataclass
class Level:
    n: int
    A: sp.csr_matrix
    mask: np.ndarray
    P: sp.csr_matrix | None = None       # from the next coarser level to this one
    R: sp.csr_matrix | None = None


def hierarchy(dim: int, n: int, k2: np.ndarray, mask: np.ndarray, levels: int) -> list:
    """Levels 0 (the given grid) .. levels - 1, each with its rediscretised operator."""
    out = []
    for l in range(levels):
        out.append(Level(n=n, A=assemble.assemble(dim, n, k2, mask), mask=np.asarray(mask).reshape(-1)))
        if l == levels - 1:
            break
        if n % 2 == 0 or n < 5:
            raise ValueError("vertex coarsening needs an odd n >= 5")
        nc = (n + 1) // 2
        out[-1].P = prolongation(dim, nc)
        out[-1].R = restriction(dim, nc)
        k2, mask, n = inject(dim, n, k2), inject(dim, n, mask), nc
    return out


def smoother(lev: Level, r, z, omega: float, n_r: int, tbs=None):
    if tbs is not None:
        z = relax.jacobi(lev.A, r, z, omega, n_r)
        z = z + tb.tb_correct(tbs, r - lev.A @ z)
        return relax.jacobi(lev.A, r, z, omega, n_r)
    return relax.jacobi(lev.A, r, z, omega, 2 * n_r + 1)


def vcycle(levels: list, r, omega: float = 0.6, n_r: int = 2, tbs=None, l: int = 0):
    """z = V(r) on level l (tbs: the trunk basis of level 0, or None)."""
    lev = levels[l]
    t = tbs if l == 0 else None
    z = smoother(lev, r, np.zeros_like(r, dtype=np.complex128), omega, n_r, t)
    if l == len(levels) - 1:
        return z
    rc = lev.R @ (r - lev.A @ z)
    rc[levels[l + 1].mask == 1] = 0.0
    corr = lev.P @ vcycle(levels, rc, omega, n_r, tbs, l + 1)
    corr[lev.mask == 1] = 0.0
    z = z + corr
    return smoother(lev, r, z, omega, n_r, t)


def mg_preconditioner(levels: list, omega: float = 0.6, n_r: int = 2, tbs=None):
    return lambda r: vcycle(levels, np.asarray(r, dtype=np.complex128), omega, n_r, tbs)
