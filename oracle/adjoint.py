"""Receiver-misfit loss and its gradient with respect to the per-node complex k^2
(adjoint method on the discrete problem of oracle.assemble).

A(k^2) u = f with (A u)_l = ... + k^2_l u_l on fluid rows (Eq. 1, FD reading).
Receivers sample u by trilinear interpolation, (S u)_r = sum of 8 corner weights.
L = sum_r |(S u)_r - d_r|^2.  With e = S u - d and the adjoint
    A^H lambda = S^T (2 e)      (A^H = conj(A): A is complex symmetric)
the gradient in PyTorch's convention (dL/dRe k^2 + i dL/dIm k^2) is
    g_l = -lambda_l conj(u_l) on fluid nodes, 0 on Dirichlet nodes,
since dA/dk^2_l = e_l e_l^T on fluid rows and dL = Re(G^H du), du = -A^-1 (dA) u.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def trilinear(n: int, pts) -> sp.csr_matrix:
    """S (R x N): each receiver's value is the trilinear interpolant of the 8
    nodes of the grid cell that contains it (nodes at i h, h = 1/(n-1))."""
    h = 1.0 / (n - 1)
    rows, cols, vals = [], [], []
    for r, p in enumerate(np.asarray(pts, dtype=np.float64)):
        s = p / h
        c = np.minimum(np.floor(s).astype(int), n - 2)
        t = s - c
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                    rows.append(r)
                    cols.append((c[0] + dx) + n * ((c[1] + dy) + n * (c[2] + dz)))
                    vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(pts), n ** 3))


def loss(S, u, d) -> float:
    e = S @ u - d
    return float(np.vdot(e, e).real)


def gradient_k2(A, S, u, d, mask, solve_adjoint):
    """g = -lambda conj(u) on fluid nodes; solve_adjoint(b) solves conj(A) lambda = b."""
    e = S @ u - d
    lam = solve_adjoint(S.T @ (2.0 * e))
    g = -lam * np.conj(u)
    g[np.asarray(mask).reshape(-1) == 1] = 0.0
    return g, lam
