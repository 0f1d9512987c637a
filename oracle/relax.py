"""Relaxation sweeps as preconditioned Richardson steps (Eq. 2, Sec. 3.1.1).

With M = (diagonal of A)^-1 the Richardson step is Jacobi (here damped by omega);
with M = (lower triangle of A)^-1 it is Gauss-Seidel.  Gauss-Seidel is taken in
red-black order: all red nodes ((i+j+k) even) first, then all black nodes with
the new red values.  Because the 5-/7-point stencil couples a node only to
nodes of the other colour (and masked rows are the identity), updating one
colour from the full residual is exactly one half-sweep of Gauss-Seidel.
SOR scales each half-step by omega; SSOR follows the forward sweep by the
backward one (black, then red).
"""
from __future__ import annotations

import numpy as np


def jacobi(A, f, x, omega: float, sweeps: int):
    """x <- x + omega D^-1 (f - A x), `sweeps` times; D = diag(A)."""
    D = A.diagonal()
    x = np.array(x, dtype=np.complex128, copy=True)
    for _ in range(sweeps):
        x = x + omega * (f - A @ x) / D
    return x


def rbgs(A, f, x, colours, sweeps: int):
    """Red-black Gauss-Seidel: per sweep, red update then black update."""
    D = A.diagonal()
    x = np.array(x, dtype=np.complex128, copy=True)
    for _ in range(sweeps):
        for c in (0, 1):
            sel = colours == c
            r = f - A @ x
            x[sel] = x[sel] + r[sel] / D[sel]
    return x


def sor(A, f, x, colours, omega: float, sweeps: int):
    """Successive over-relaxation in red-black order (Sec. 3.1.1 names SOR beside
    Jacobi and Gauss-Seidel): per sweep a red then a black half-step, each
    x_l <- x_l + omega D_l^-1 (f - A x)_l with the latest neighbours.  omega = 1 is
    red-black Gauss-Seidel."""
    D = A.diagonal()
    x = np.array(x, dtype=np.complex128, copy=True)
    for _ in range(sweeps):
        for c in (0, 1):
            sel = colours == c
            r = f - A @ x
            x[sel] = x[sel] + omega * r[sel] / D[sel]
    return x


def ssor(A, f, x, colours, omega: float, sweeps: int):
    """Symmetric SOR in red-black order: per sweep the forward SOR sweep (red,
    black) followed by the backward one (black, red)."""
    D = A.diagonal()
    x = np.array(x, dtype=np.complex128, copy=True)
    for _ in range(sweeps):
        for c in (0, 1, 1, 0):
            sel = colours == c
            r = f - A @ x
            x[sel] = x[sel] + omega * r[sel] / D[sel]
    return x
