"""Pins for oracle.assemble: closed forms, brute force, manufactured solutions,
free-space Green's functions (Eq. 1, FD reading)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import hankel1

import scenes
from oracle import assemble


def _ring(dim, n):
    return scenes.ring_mask(dim, n).reshape(-1).astype(np.uint8)


@pytest.mark.parametrize("dim,n,a,b", [(2, 17, 1, 2), (2, 33, 3, 1), (3, 9, 1, 2), (3, 12, 2, 3)])
def test_discrete_sine_eigenfunction(dim, n, a, b):
    """With constant k, no layer and only the outer ring masked, the grid sine
    modes are exact eigenvectors: eigenvalue k^2 - (4/h^2) sum sin^2(a pi h/2)."""
    k0 = 7.0
    h = 1.0 / (n - 1)
    k2 = assemble.k2_field(dim, n, k0, 0, 0.5)
    A = assemble.assemble(dim, n, k2, _ring(dim, n))
    X = scenes.node_coords(dim, n)
    modes = [a, b, a + b][:dim]
    v = np.ones(X.shape[0])
    for ax, m in enumerate(modes):
        v *= np.sin(m * np.pi * X[:, ax])
    lam = k0 * k0 - (4.0 / h ** 2) * sum(np.sin(m * np.pi * h / 2) ** 2 for m in modes)
    Av = A @ v
    # ring rows are identity and v vanishes there up to sin(m pi) rounding
    assert np.max(np.abs(Av - lam * v)) <= 1e-12 * np.max(np.abs(lam * v)) + 1e-12


def _dense_by_loops(dim, n, k2, mask):
    h = 1.0 / (n - 1)
    N = n ** dim
    D = np.zeros((N, N), dtype=np.complex128)
    for l in range(N):
        i, j = l % n, (l // n) % n
        k = l // (n * n) if dim == 3 else 0
        if mask[l]:
            D[l, l] = 1.0
            continue
        D[l, l] = k2[l] - 2 * dim / h ** 2
        offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)] + ([(0, 0, 1), (0, 0, -1)] if dim == 3 else [])
        for di, dj, dk in offs:
            ii, jj, kk = i + di, j + dj, k + dk
            if not (0 <= ii < n and 0 <= jj < n and 0 <= kk < (n if dim == 3 else 1)):
                continue
            m = ii + n * (jj + n * kk)
            if not mask[m]:
                D[l, m] += 1.0 / h ** 2
    return D


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 5)])
def test_brute_force_dense(dim, n):
    rng = np.random.default_rng(3)
    mask = _ring(dim, n)
    inner = rng.random(n ** dim) < 0.2
    mask = (mask | inner).astype(np.uint8)
    k2 = assemble.k2_field(dim, n, 5.0, 2, 0.5)
    A = assemble.assemble(dim, n, k2, mask).toarray()
    D = _dense_by_loops(dim, n, k2, mask)
    assert np.array_equal(A, D)
    assert np.array_equal(A, A.T)                       # complex symmetric
    for l in np.flatnonzero(mask):
        e = np.zeros(n ** dim); e[l] = 1
        assert np.array_equal(A[l], e)


def test_layer_values():
    """eta: 1 on the outer ring, (cells - dist)/cells inside the layer, 0 beyond;
    corners take the max over axes."""
    n, cells, k0, s = 40, 8, 3.0, 0.5
    k2 = assemble.k2_field(2, n, k0, cells, s).reshape(n, n)
    assert k2[0, 0] == k0 ** 2 * (1 + 0.5j)
    assert k2[20, 4] == k0 ** 2 * (1 + 1j * s * (4 / 8) ** 2)
    assert k2[20, 8] == k0 ** 2
    assert k2[20, 20] == k0 ** 2
    assert k2[2, 5] == k0 ** 2 * (1 + 1j * s * (6 / 8) ** 2)    # max(depth_y=6/8, depth_x=3/8)
    assert k2[n - 1 - 3, 20] == k0 ** 2 * (1 + 1j * s * (5 / 8) ** 2)


def test_manufactured_second_order():
    """u* = sin(pi x) sin(2 pi y) (sin(pi z)): the FD error falls by ~4 per halving of h."""
    errs = []
    for n in (17, 33, 65):
        k0 = 5.0
        dim = 2
        X = scenes.node_coords(dim, n)
        u = np.sin(np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1])
        f = (k0 ** 2 - 5 * np.pi ** 2) * u
        mask = _ring(dim, n)
        k2 = assemble.k2_field(dim, n, k0, 0, 0.5)
        A = assemble.assemble(dim, n, k2, mask)
        b = assemble.rhs(dim, n, mask, f, np.zeros(n ** dim, complex))
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(np.max(np.abs(uh - u)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


def test_manufactured_3d():
    errs = []
    for n in (9, 17, 33):
        k0 = 4.0
        X = scenes.node_coords(3, n)
        u = np.sin(np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        f = (k0 ** 2 - 6 * np.pi ** 2) * u
        mask = _ring(3, n)
        A = assemble.assemble(3, n, assemble.k2_field(3, n, k0, 0, 0.5), mask)
        b = assemble.rhs(3, n, mask, f, np.zeros(n ** 3, complex))
        errs.append(np.max(np.abs(spla.spsolve(A.tocsc(), b) - u)))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.6 < errs[1] / errs[2] < 4.4, errs


def test_lift_equals_unlifted_system():
    """Moving Dirichlet values to the right-hand side gives the same solution as
    the system that keeps the fluid-to-masked couplings with u = g imposed."""
    dim, n = 2, 21
    rng = np.random.default_rng(1)
    mask = (_ring(dim, n) | scenes.box_mask(dim, n, 8, 12).reshape(-1)).astype(np.uint8)
    k2 = assemble.k2_field(dim, n, 6.0, 4, 0.5)
    g = np.where(mask == 1, rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n), 0)
    src = np.where(mask == 0, rng.standard_normal(n * n), 0).astype(complex)
    A = assemble.assemble(dim, n, k2, mask)
    b = assemble.rhs(dim, n, mask, src, g)
    u = spla.spsolve(A.tocsc(), b)
    # full-coupling system: fluid rows see every neighbour, masked rows identity
    h = 1.0 / (n - 1)
    B = sp.lil_matrix((n * n, n * n), dtype=complex)
    for l in range(n * n):
        if mask[l]:
            B[l, l] = 1
            continue
        B[l, l] = k2[l] - 4 / h ** 2
        i, j = l % n, l // n
        for m in (l - 1, l + 1, l - n, l + n):
            B[l, m] = 1 / h ** 2
    rhs_full = np.where(mask == 1, g, src)
    v = spla.spsolve(B.tocsc(), rhs_full)
    assert np.allclose(u, v, rtol=0, atol=1e-12 * np.max(np.abs(v)))
    assert np.allclose(u[mask == 1], g[mask == 1], atol=1e-14)


def test_free_space_2d_hankel():
    """Point source delta/h^2, ring-only mask, a wide absorbing layer: the field
    follows the outgoing free-space solution -(i/4) H0^(1)(k r) for r in [0.1, 0.2]
    within a few percent (layer reflection + dispersion), and |u| ~ r^-1/2.
    A wrong layer sign (amplifying instead of absorbing) or a wrong stencil sign
    fails this by orders of magnitude."""
    n, k0 = 257, 16.0
    h = 1.0 / (n - 1)
    mask = _ring(2, n)
    k2 = assemble.k2_field(2, n, k0, 96, 2.0)
    A = assemble.assemble(2, n, k2, mask)
    c = (n // 2) + n * (n // 2)
    f = np.zeros(n * n, complex); f[c] = 1.0 / h ** 2
    u = spla.spsolve(A.tocsc(), assemble.rhs(2, n, mask, f, np.zeros(n * n, complex)))
    X = scenes.node_coords(2, n)
    r = np.linalg.norm(X - X[c], axis=1)
    sel = (r >= 0.1) & (r <= 0.2)
    ref = -0.25j * hankel1(0, k0 * r[sel])
    rel = np.linalg.norm(u[sel] - ref) / np.linalg.norm(ref)
    assert rel < 0.04, rel
    slope = np.polyfit(np.log(r[sel]), np.log(np.abs(u[sel])), 1)[0]
    assert -0.6 < slope < -0.4, slope


def test_layer_values_3d_and_reciprocity():
    """3D layer depth is the max over the three axes; G(x, y) = G(y, x)."""
    n, k0 = 17, 6.0
    k2 = assemble.k2_field(3, n, k0, 4, 0.5).reshape(n, n, n)
    assert k2[1, 2, 3] == k0 ** 2 * (1 + 0.5j * (3 / 4) ** 2)     # dist (3, 2, 1) -> depth 3/4
    assert k2[8, 8, 15] == k0 ** 2 * (1 + 0.5j * (3 / 4) ** 2)    # x dist 1
    assert k2[8, 8, 8] == k0 ** 2
    mask = _ring(3, n)
    A = assemble.assemble(3, n, k2.reshape(-1), mask).tocsc()
    lu = spla.splu(A)
    c = 8 + n * (8 + n * 8)
    d = 3 + n * (12 + n * 5)
    f1 = np.zeros(n ** 3, complex); f1[c] = 1.0
    f2 = np.zeros(n ** 3, complex); f2[d] = 1.0
    assert abs(lu.solve(f1)[d] - lu.solve(f2)[c]) <= 1e-12 * abs(lu.solve(f1)[d])


def test_direct_lu_matches_dense_solve():
    n = 12
    rng = np.random.default_rng(0)
    mask = (_ring(2, n) | scenes.box_mask(2, n, 4, 7).reshape(-1)).astype(np.uint8)
    A = assemble.assemble(2, n, assemble.k2_field(2, n, 9.0, 3, 0.5), mask)
    b = assemble.rhs(2, n, mask, np.where(mask == 0, rng.standard_normal(n * n), 0).astype(complex),
                     np.zeros(n * n, complex))
    u1 = spla.splu(A.tocsc()).solve(b)
    u2 = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u2)
    assert np.linalg.norm(A @ u1 - b) <= 1e-13 * np.linalg.norm(b)
