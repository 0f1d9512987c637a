"""Finite-difference restatement of the complex Helmholtz problem (Eq. 1).

Eq. 1 poses  Delta u + k(x)^2 u = f  in Omega with an absorbing outer boundary
and u = 0 on the scatterer.  This restatement (the reading used throughout):

* nodes x_i = i h on [0,1]^d, h = 1/(n-1), flat index i + n(j + n k);
* the outer node ring and the staircased scatterer form the Dirichlet set M;
* absorbing layer instead of the first-order ABC: within `cells` nodes of the
  outer boundary, k^2 = k0^2 (1 + i * strength * eta^2) with
  eta = max over axes of max(0, cells - dist_a)/cells, dist_a = min(i_a, n-1-i_a);
* fluid rows: (A x)_l = h^-2 sum_{fluid nbr m} x_m + (k_l^2 - 2 d h^-2) x_l;
  masked rows: (A x)_l = x_l  (identity, Dirichlet);
* right-hand side: b_l = src_l - h^-2 sum_{masked nbr m} g_m  on fluid rows,
  b_l = g_l on masked rows (the Dirichlet values moved to the right, App. D).

A is complex symmetric (A^T = A), so A^H = conj(A).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def layer_eta(dim: int, n: int, cells: int) -> np.ndarray:
    """Absorbing-layer depth eta in [0, 1] per node (flat)."""
    idx = np.arange(n)
    dist = np.minimum(idx, n - 1 - idx)
    if cells <= 0:
        return np.zeros(n ** dim)
    depth = np.maximum(0, cells - dist) / float(cells)
    if dim == 2:
        eta = np.maximum(depth[None, :], depth[:, None])
    else:
        eta = np.maximum(np.maximum(depth[None, None, :], depth[None, :, None]), depth[:, None, None])
    return eta.reshape(-1)


def k2_field(dim: int, n: int, k0: float, cells: int, strength: float, scale=None) -> np.ndarray:
    """k^2 per node: k0^2 * scale * (1 + i strength eta^2); scale defaults to 1."""
    eta = layer_eta(dim, n, cells)
    base = k0 * k0 * (np.ones_like(eta) if scale is None else np.asarray(scale, dtype=np.float64))
    return base * (1.0 + 1j * strength * eta * eta)


def neighbours(dim: int, n: int):
    """Yield (l, m) flat-index arrays of every in-grid neighbour pair l -> m."""
    N = n ** dim
    l = np.arange(N)
    idx = [l % n, (l // n) % n] + ([l // (n * n)] if dim == 3 else [])
    stride = [1, n, n * n][:dim]
    for a in range(dim):
        for s in (-1, 1):
            ok = (idx[a] + s >= 0) & (idx[a] + s <= n - 1)
            yield l[ok], l[ok] + s * stride[a]


def assemble(dim: int, n: int, k2: np.ndarray, mask: np.ndarray) -> sp.csr_matrix:
    """Sparse complex128 A of the FD Helmholtz operator (module docstring)."""
    N = n ** dim
    h = 1.0 / (n - 1)
    fluid = np.asarray(mask).reshape(-1) == 0
    rows, cols, vals = [], [], []
    diag = np.where(fluid, k2 - 2.0 * dim / (h * h), 1.0).astype(np.complex128)
    rows.append(np.arange(N)); cols.append(np.arange(N)); vals.append(diag)
    for l, m in neighbours(dim, n):
        keep = fluid[l] & fluid[m]
        rows.append(l[keep]); cols.append(m[keep])
        vals.append(np.full(keep.sum(), 1.0 / (h * h), dtype=np.complex128))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    return A


def rhs(dim: int, n: int, mask: np.ndarray, src: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Lifted right-hand side b (module docstring)."""
    h = 1.0 / (n - 1)
    fluid = np.asarray(mask).reshape(-1) == 0
    b = np.where(fluid, src, g).astype(np.complex128)
    for l, m in neighbours(dim, n):
        sel = fluid[l] & ~fluid[m]
        np.add.at(b, l[sel], -g[m[sel]] / (h * h))
    return b


def colour(dim: int, n: int) -> np.ndarray:
    """Red-black colour (i + j + k) mod 2 per node; 0 = red (updated first)."""
    l = np.arange(n ** dim)
    s = l % n + (l // n) % n + ((l // (n * n)) if dim == 3 else 0)
    return (s % 2).astype(np.int8)


def problem(scene):
    """(A, b, k2) for a `scenes.Scene`."""
    k2 = k2_field(scene.dim, scene.n, scene.k0, scene.layer_cells, scene.layer_strength,
                  scene.k2_scale)
    A = assemble(scene.dim, scene.n, k2, scene.mask)
    b = rhs(scene.dim, scene.n, scene.mask, scene.src, scene.g)
    return A, b, k2
