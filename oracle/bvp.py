"""The paper's own boundary-value problem (Eq. 1) in finite differences: a
first-order absorbing (Sommerfeld) condition du/dn - i k u = 0 on the outer
faces and a Neumann incoming-wave condition du/dn = g on the top face
(y = 1 in 2D, z = 1 in 3D), the scatterer Dirichlet, no absorbing layer.

Each outer-boundary node is an unknown.  Its row is the 5/7-point row with the
ghost node beyond each boundary face eliminated through the central difference
of the face's condition, written for an outward normal along axis a:

* Sommerfeld face, du/dn - i k u = q:   u_ghost = u_inward + 2 h (i k u_l + q),
* Neumann face,    du/dn = g:           u_ghost = u_inward + 2 h g,

so that the inward neighbour enters the row twice, a Sommerfeld face adds
2 i k / h to the diagonal, and the data move to the right-hand side as
-(2 / h) q (or g).  A row of a node lying on b faces is then multiplied by 2^-b;
this makes the matrix complex symmetric.  Scatterer rows are the identity with
the Dirichlet values lifted to the right-hand side (as in assemble.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _ijk(dim: int, n: int):
    l = np.arange(n ** dim)
    return [l % n, (l // n) % n] + ([l // (n * n)] if dim == 3 else [])


def faces(dim: int, n: int):
    """Per node: list over axes of -1 (low face), +1 (high face) or 0."""
    return [np.where(c == 0, -1, np.where(c == n - 1, 1, 0)) for c in _ijk(dim, n)]


def assemble_bvp(dim: int, n: int, k2: np.ndarray, mask: np.ndarray, k0: float, neumann_top: bool = True,
                 scaled: bool = True) -> sp.csr_matrix:
    """Sparse A of the Sommerfeld / Neumann problem (scaled rows unless scaled=False)."""
    N = n ** dim
    h = 1.0 / (n - 1)
    fluid = np.asarray(mask).reshape(-1) == 0
    idx = _ijk(dim, n)
    fc = faces(dim, n)
    stride = [1, n, n * n][:dim]
    A = sp.lil_matrix((N, N), dtype=np.complex128)
    for l in range(N):
        if not fluid[l]:
            A[l, l] = 1.0
            continue
        diag = complex(k2[l]) - 2.0 * dim / h ** 2
        for a in range(dim):
            top = neumann_top and a == dim - 1 and fc[a][l] == 1
            for s in (-1, 1):
                if (s == -1 and idx[a][l] == 0) or (s == 1 and idx[a][l] == n - 1):
                    # ghost node beyond this face: its value is the inward neighbour's
                    # plus 2 h (i k u_l) on a Sommerfeld face (data go to the rhs)
                    inward = l - s * stride[a]
                    if fluid[inward]:
                        A[l, inward] += 1.0 / h ** 2
                    if not top:
                        diag += 2j * k0 / h
                    continue
                m = l + s * stride[a]
                if fluid[m]:
                    A[l, m] += 1.0 / h ** 2
        A[l, l] += diag
    A = A.tocsr()
    if scaled:
        b = sum(np.abs(f) for f in fc)
        A = (sp.diags(np.where(fluid, 2.0 ** -b, 1.0)) @ A).tocsr()
    A.sum_duplicates()
    return A


def rhs_bvp(dim: int, n: int, mask: np.ndarray, src: np.ndarray, g: np.ndarray, neumann_top: bool = True,
            q_face=None, scaled: bool = True) -> np.ndarray:
    """Right-hand side: Dirichlet values g on masked nodes (lifted into fluid rows),
    the Neumann datum g on the top face and, optionally, Sommerfeld data
    q_face(axis, side, l) (default zero) on the other faces."""
    N = n ** dim
    h = 1.0 / (n - 1)
    fluid = np.asarray(mask).reshape(-1) == 0
    idx = _ijk(dim, n)
    fc = faces(dim, n)
    stride = [1, n, n * n][:dim]
    b = np.where(fluid, src, g).astype(np.complex128)
    for l in range(N):
        if not fluid[l]:
            continue
        for a in range(dim):
            for s in (-1, 1):
                if (s == -1 and idx[a][l] == 0) or (s == 1 and idx[a][l] == n - 1):
                    top = neumann_top and a == dim - 1 and s == 1
                    datum = g[l] if top else (q_face(a, s, l) if q_face is not None else 0.0)
                    b[l] -= 2.0 / h * datum
                    inward = l - s * stride[a]
                    if not fluid[inward]:
                        b[l] -= g[inward] / h ** 2
                    continue
                m = l + s * stride[a]
                if not fluid[m]:
                    b[l] -= g[m] / h ** 2
    if scaled:
        bnum = sum(np.abs(f) for f in fc)
        b = np.where(fluid, b * 2.0 ** -bnum, b)
    return b
