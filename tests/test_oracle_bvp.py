"""Pins of the oracle's Sommerfeld / Neumann boundary-value problem (oracle/bvp.py,
Eq. 1 in finite differences with ghost-point boundary rows):

* the row-scaled matrix is exactly complex symmetric (2D and 3D, with a scatterer);
* a plane wave u = exp(i k d.x) with the matching boundary data (du/dn - i k u on
  the Sommerfeld faces, du/dn on the Neumann face) is reproduced to second order:
  the nodal error falls by ~4 per halving of h (a dropped factor 2 of the ghost
  row, a wrong sign of the i k term or a wrong datum breaks the order);
* a point source with the absorbing condition on every face follows the outgoing
  free-space solution -(i/4) H0^(1)(k r) near the source (within the reflection of
  a first-order condition), and |u| decays like r^-1/2.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.special import hankel1

import scenes
from oracle import bvp


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 6)])
def test_scaled_matrix_is_complex_symmetric(dim, n):
    mask = np.zeros(n ** dim, np.uint8)
    mask[(n // 2) * (1 + n + (n * n if dim == 3 else 0))] = 1
    rng = np.random.default_rng(0)
    k2 = 30.0 + 5.0 * rng.random(n ** dim) + 1j * rng.random(n ** dim)
    for top in (True, False):
        A = bvp.assemble_bvp(dim, n, k2, mask, 5.0, neumann_top=top)
        assert abs(A - A.T).max() == 0.0
        U = bvp.assemble_bvp(dim, n, k2, mask, 5.0, neumann_top=top, scaled=False)
        assert abs(U - U.T).max() > 0.1          # the unscaled ghost rows are not symmetric


def _plane_wave_error(n, k0=6.0, theta=0.7):
    dim = 2
    X = scenes.node_coords(dim, n)
    d = np.array([np.cos(theta), np.sin(theta)])
    u = np.exp(1j * k0 * X @ d)
    mask = np.zeros(n * n, np.uint8)
    k2 = np.full(n * n, k0 * k0, complex)
    # outward normals: axis a, side s -> s e_a; du/dn = i k (s d_a) u
    q = lambda a, s, l: 1j * k0 * (s * d[a] - 1.0) * u[l]
    g = 1j * k0 * d[1] * u                   # Neumann datum on the top face (y = 1, outward +y)
    A = bvp.assemble_bvp(dim, n, k2, mask, k0, neumann_top=True)
    b = bvp.rhs_bvp(dim, n, mask, np.zeros(n * n, complex), g, neumann_top=True, q_face=q)
    x = spla.spsolve(A.tocsc(), b)
    return np.max(np.abs(x - u))


def test_plane_wave_second_order():
    e = [_plane_wave_error(n) for n in (17, 33, 65)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.3 < r1 < 4.8 and 3.5 < r2 < 4.5, (e, r1, r2)
    assert e[2] < 1e-2


def test_point_source_all_sommerfeld_follows_hankel():
    n, k0 = 129, 24.0
    dim = 2
    h = 1.0 / (n - 1)
    mask = np.zeros(n * n, np.uint8)
    c = (n // 2) * (1 + n)
    f = np.zeros(n * n, complex)
    f[c] = 1.0 / h ** 2
    A = bvp.assemble_bvp(dim, n, np.full(n * n, k0 * k0, complex), mask, k0, neumann_top=False)
    b = bvp.rhs_bvp(dim, n, mask, f, np.zeros(n * n, complex), neumann_top=False)
    u = spla.spsolve(A.tocsc(), b)
    X = scenes.node_coords(dim, n)
    r = np.linalg.norm(X - X[c], axis=1)
    sel = (r >= 0.08) & (r <= 0.2)
    ref = -0.25j * hankel1(0, k0 * r[sel])
    err = np.linalg.norm(u[sel] - ref) / np.linalg.norm(ref)
    assert err < 0.05, err
    slope = np.polyfit(np.log(r[sel]), np.log(np.abs(u[sel])), 1)[0]
    assert -0.7 < slope < -0.3, slope
    # the opposite sign of the i k term (an incoming condition) is far off
    Abad = bvp.assemble_bvp(dim, n, np.full(n * n, k0 * k0, complex), mask, -k0, neumann_top=False)
    ubad = spla.spsolve(Abad.tocsc(), b)
    assert np.linalg.norm(ubad[sel] - ref) / np.linalg.norm(ref) > 0.5
