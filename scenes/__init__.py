"""Seeded synthetic inputs for the Helmholtz meta-solvers (data only).

This module is the one place that both the CUDA path and the CPU oracle take
their inputs from.  It holds no arithmetic of the method itself: no stencil,
no absorbing-layer profile, no relaxation, projection or Krylov step.  What it
produces is *data* that the paper's experiments feed into the solver:

* node masks (outer Dirichlet ring plus a staircased scatterer, Sec. 4.2 uses
  "stair-casing" on a uniform grid: 1 inside the scatterer, 0 outside),
* forcing terms (a Gaussian source; Gaussian-random-field samples, App. A),
* incident plane-wave Dirichlet data for a scattered-field solve,
* seeded trunk / branch weights (Glorot-normal, zero bias),
* receivers and smooth wavenumber bumps for the receiver-misfit loss.

Grid convention: ``dim`` in {2, 3}; ``n`` nodes per axis on [0, 1];
``h = 1/(n-1)``; node (i, j, k) sits at (i h, j h, k h); the flat index is
``l = i + n*(j + n*k)`` (x fastest), i.e. numpy arrays of shape (n,)*dim in C
order indexed ``a[k, j, i]``.

All randomness goes through ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAYER_CELLS = 8          # width of the absorbing layer in grid cells
LAYER_STRENGTH = 0.5     # Im k^2 ramps 0 -> LAYER_STRENGTH * k0^2


def shape_of(dim: int, n: int) -> tuple:
    return (n,) * dim


def node_axes(dim: int, n: int):
    """Integer node indices per axis, broadcast to the grid (x last)."""
    idx = np.arange(n)
    if dim == 2:
        j, i = np.meshgrid(idx, idx, indexing="ij")
        return (i, j)
    k, j, i = np.meshgrid(idx, idx, idx, indexing="ij")
    return (i, j, k)


def node_coords(dim: int, n: int) -> np.ndarray:
    """(N, dim) float64 node coordinates in flat order (x fastest)."""
    h = 1.0 / (n - 1)
    ax = node_axes(dim, n)
    return np.stack([a.reshape(-1) * h for a in ax], axis=1)


# --------------------------------------------------------------------- masks
def ring_mask(dim: int, n: int) -> np.ndarray:
    """1 on the outermost node ring (homogeneous Dirichlet)."""
    ax = node_axes(dim, n)
    m = np.zeros(shape_of(dim, n), dtype=bool)
    for a in ax:
        m |= (a == 0) | (a == n - 1)
    return m


def box_mask(dim: int, n: int, lo: int, hi: int) -> np.ndarray:
    """1 on nodes with lo <= index <= hi on every axis (a centred square/cube)."""
    ax = node_axes(dim, n)
    m = np.ones(shape_of(dim, n), dtype=bool)
    for a in ax:
        m &= (a >= lo) & (a <= hi)
    return m


def centred_box_nodes(n: int, width_nodes: int) -> tuple:
    """Node range of a centred box `width_nodes` wide (symmetric about (n-1)/2)."""
    lo = (n - width_nodes) // 2
    return lo, lo + width_nodes - 1


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised 4-vector of N(0,1) draws."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _body_coords(n: int, centre, rot: np.ndarray, scale: float = 1.0):
    """Node coordinates mapped into the body frame of a rotated, scaled shape."""
    X = node_coords(3, n) - np.asarray(centre)[None, :]
    return (X @ rot) / scale          # rot columns are the body axes


def sphere_mask(n: int, centre, radius: float) -> np.ndarray:
    X = node_coords(3, n) - np.asarray(centre)[None, :]
    return (np.einsum("ij,ij->i", X, X) <= radius * radius).reshape(shape_of(3, n))


def rotated_cube_mask(n: int, centre, half: float, rot: np.ndarray) -> np.ndarray:
    B = _body_coords(n, centre, rot)
    return (np.abs(B) <= half).all(axis=1).reshape(shape_of(3, n))


def submarine_mask(n: int, rot: np.ndarray, scale: float = 1.0, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Parametric submarine, staircased onto the nodes.

    Hull: ellipsoid with semi-axes (0.35, 0.06, 0.06) along body (x, y, z).
    Sail: box 0.08 x 0.02 x 0.05 standing on the hull top (z from +0.06),
    centred at body x = +0.08.  Fins: four 0.05 x 0.005 x 0.04 plates at the
    stern (x = -0.30) in a cruciform.  Plate thicknesses below one grid step
    are widened to one step so the fins survive staircasing.  `scale`
    multiplies every length (1.0 is the nominal size).
    """
    h = 1.0 / (n - 1)
    B = _body_coords(n, centre, rot, scale)
    hs = h / scale                               # one grid step in body units
    x, y, z = B[:, 0], B[:, 1], B[:, 2]
    m = (x / 0.35) ** 2 + (y / 0.06) ** 2 + (z / 0.06) ** 2 <= 1.0

    def box(cx, cy, cz, lx, ly, lz):
        lx, ly, lz = (max(v, hs) for v in (lx, ly, lz))
        return (np.abs(x - cx) <= lx / 2) & (np.abs(y - cy) <= ly / 2) & (np.abs(z - cz) <= lz / 2)

    m |= box(0.08, 0.0, 0.06 + 0.025, 0.08, 0.02, 0.05)             # sail
    fx = -0.30
    m |= box(fx, 0.06 + 0.02, 0.0, 0.05, 0.04, 0.005)               # horizontal fins
    m |= box(fx, -(0.06 + 0.02), 0.0, 0.05, 0.04, 0.005)
    m |= box(fx, 0.0, 0.06 + 0.02, 0.05, 0.005, 0.04)               # vertical fins
    m |= box(fx, 0.0, -(0.06 + 0.02), 0.05, 0.005, 0.04)
    return m.reshape(shape_of(3, n))


# ------------------------------------------------------------------- sources
def gaussian_source(dim: int, n: int, centre, sigma: float) -> np.ndarray:
    """exp(-|x - c|^2 / (2 sigma^2)), amplitude 1, real, flat."""
    X = node_coords(dim, n) - np.asarray(centre)[None, :]
    return np.exp(-np.einsum("ij,ij->i", X, X) / (2.0 * sigma * sigma))


def seeded_centre(rng, dim: int, n: int, sigma: float, avoid_lo=None, avoid_hi=None,
                  layer_cells: int = LAYER_CELLS) -> np.ndarray:
    """Uniform point in [layer + 2 sigma, 1 - layer - 2 sigma]^dim that keeps 2 sigma
    away from the box [avoid_lo, avoid_hi]^dim (coordinates) when one is given."""
    h = 1.0 / (n - 1)
    lo, hi = layer_cells * h + 2 * sigma, 1.0 - layer_cells * h - 2 * sigma
    for _ in range(100000):
        c = rng.uniform(lo, hi, size=dim)
        if avoid_lo is None:
            return c
        if np.any(c < avoid_lo - 2 * sigma) or np.any(c > avoid_hi + 2 * sigma):
            return c
    raise RuntimeError("no admissible source centre")


def unit_vector(rng, dim: int = 3) -> np.ndarray:
    v = rng.standard_normal(dim)
    return v / np.linalg.norm(v)


def plane_wave(dim: int, n: int, k0: float, direction) -> np.ndarray:
    """Incident field exp(i k0 d.x) at the nodes (flat, complex128)."""
    X = node_coords(dim, n)
    return np.exp(1j * k0 * (X @ np.asarray(direction)))


def grf_1d_factor(n: int, length: float, s: float = 1.0, jitter: float = 1e-10) -> np.ndarray:
    """Cholesky factor of the 1D RBF kernel s^2 exp(-|x-y|^2/(2 l^2)) on the nodes."""
    x = np.linspace(0.0, 1.0, n)
    K = s * s * np.exp(-(x[:, None] - x[None, :]) ** 2 / (2 * length * length))
    return np.linalg.cholesky(K + jitter * np.eye(n))


def grf_samples(rng, dim: int, n: int, count: int, length: float = 0.1) -> np.ndarray:
    """`count` samples of a zero-mean separable RBF Gaussian random field
    (App. A: f has independent real and imaginary GRF parts, l = 0.1, s = 1).
    Returns (count, N) complex128."""
    L = grf_1d_factor(n, length)
    out = np.empty((count, n ** dim), dtype=np.complex128)
    for c in range(count):
        parts = []
        for _ in range(2):
            xi = rng.standard_normal(shape_of(dim, n))
            # apply L along every axis: (L_z (x) L_y (x) L_x) xi
            for ax in range(dim):
                xi = np.moveaxis(np.tensordot(L, np.moveaxis(xi, ax, 0), axes=(1, 0)), 0, ax)
            parts.append(xi.reshape(-1))
        out[c] = parts[0] + 1j * parts[1]
    return out


# ------------------------------------------------------------------- weights
def glorot_mlp(rng, widths, dtype=np.float64):
    """Glorot-normal weights N(0, 2/(fan_in+fan_out)) and zero biases.
    Returns a list of (W[out, in], b[out])."""
    layers = []
    for a, b in zip(widths[:-1], widths[1:]):
        W = rng.standard_normal((b, a)) * math.sqrt(2.0 / (a + b))
        layers.append((W.astype(dtype), np.zeros(b, dtype=dtype)))
    return layers


def pack_mlp(layers) -> np.ndarray:
    """Flat packing used by the C ABI: for each layer, W (row-major out x in) then b."""
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


# ----------------------------------------------------------------- receivers
def fibonacci_sphere(count: int, radius: float, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    i = np.arange(count) + 0.5
    z = 1.0 - 2.0 * i / count
    r = np.sqrt(1.0 - z * z)
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.asarray(centre)[None, :] + radius * pts


def gaussian_bumps(rng, n: int, count: int = 8, sigma: float = 0.08, amp: float = 0.05,
                   avoid_lo=None, avoid_hi=None, layer_cells: int = LAYER_CELLS) -> np.ndarray:
    """Real multiplicative perturbation 1 + sum_b a_b exp(-|x-c_b|^2/(2 sigma^2)),
    a_b ~ U[-amp, amp], centres in the interior box away from the scatterer."""
    X = node_coords(3, n)
    s = np.zeros(X.shape[0])
    for _ in range(count):
        c = seeded_centre(rng, 3, n, sigma / 3.0, avoid_lo, avoid_hi, layer_cells)
        a = rng.uniform(-amp, amp)
        d = X - c[None, :]
        s += a * np.exp(-np.einsum("ij,ij->i", d, d) / (2 * sigma * sigma))
    return 1.0 + s


# ------------------------------------------------------------------- configs
@dataclass
class Scene:
    """One synthetic problem: everything the solver consumes, nothing it computes."""
    name: str
    dim: int
    n: int
    k0: float
    mask: np.ndarray            # (N,) uint8, 1 = Dirichlet node (ring + scatterer)
    src: np.ndarray             # (N,) complex128 forcing on fluid nodes
    g: np.ndarray               # (N,) complex128 Dirichlet values on masked nodes
    trunk: list = field(default_factory=list)    # [(W, b)], tanh hidden layers
    p: int = 0
    k2_scale: np.ndarray | None = None           # optional real per-node multiplier of k0^2
    layer_cells: int = LAYER_CELLS
    layer_strength: float = LAYER_STRENGTH
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return 1.0 / (self.n - 1)

    @property
    def N(self) -> int:
        return self.n ** self.dim


def _finish(name, dim, n, k0, scat, src, g=None, trunk=None, p=0, **kw):
    mask = (ring_mask(dim, n) | scat).reshape(-1).astype(np.uint8)
    src = np.asarray(src, dtype=np.complex128).reshape(-1).copy()
    src[mask == 1] = 0.0
    if g is None:
        g = np.zeros(n ** dim, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128).reshape(-1).copy()
    g[mask == 0] = 0.0
    return Scene(name=name, dim=dim, n=n, k0=k0, mask=mask, src=src, g=g,
                 trunk=trunk or [], p=p, **kw)


def square2d(seed: int = 0, n: int = 64, k0: float = 10.0, width: int = 12, p: int = 32,
             sigma: float = 0.05) -> Scene:
    """2D: 64x64 grid, k = 10, centred 12x12-node sound-soft square, Gaussian
    source sigma = 0.05 at a seeded point, seeded trunk [2, 64, 64, p]."""
    rng = np.random.default_rng(seed)
    lo, hi = centred_box_nodes(n, width)
    h = 1.0 / (n - 1)
    scat = box_mask(2, n, lo, hi)
    c = seeded_centre(rng, 2, n, sigma, np.full(2, lo * h), np.full(2, hi * h))
    trunk = glorot_mlp(rng, [2, 64, 64, p])
    return _finish("square2d", 2, n, k0, scat, gaussian_source(2, n, c, sigma), trunk=trunk, p=p,
                   extra={"centre": c})


def cube3d(seed: int = 0, n: int = 64, k0: float = 16.0, width: int = 16, p: int = 128,
           sigma: float = 0.04, trunk_widths=(3, 128, 128, 128)) -> Scene:
    """3D: n^3 grid, k = 16, centred 16^3-node sound-soft cube, Gaussian source
    sigma = 0.04 at a seeded point, trunk [3, 128, 128, 128]."""
    rng = np.random.default_rng(seed)
    lo, hi = centred_box_nodes(n, width)
    h = 1.0 / (n - 1)
    scat = box_mask(3, n, lo, hi)
    c = seeded_centre(rng, 3, n, sigma, np.full(3, lo * h), np.full(3, hi * h))
    widths = list(trunk_widths[:-1]) + [p] if trunk_widths[-1] != p else list(trunk_widths)
    trunk = glorot_mlp(rng, widths)
    return _finish("cube3d", 3, n, k0, scat, gaussian_source(3, n, c, sigma), trunk=trunk, p=p,
                   extra={"centre": c})


def submarine3d(seed: int = 0, n: int = 128, k0: float = 32.0, p: int = 256) -> Scene:
    """3D mixed-precision workload: n^3 grid, k = 32, seeded-rotation submarine,
    scattered-field solve for a seeded incident plane wave (g = -u_inc on the
    scatterer, 0 on the outer ring, zero forcing), seeded trunk [3,256,256,p]."""
    rng = np.random.default_rng(seed)
    rot = random_rotation(rng)
    d = unit_vector(rng, 3)
    scat = submarine_mask(n, rot)
    uinc = plane_wave(3, n, k0, d)
    g = np.where(scat.reshape(-1), -uinc, 0.0)
    trunk = glorot_mlp(rng, [3, 256, 256, p])
    return _finish("submarine3d", 3, n, k0, scat, np.zeros(n ** 3), g=g, trunk=trunk, p=p,
                   extra={"direction": d, "rotation": rot})


def bump_cube3d(seed: int = 0, n: int = 96, k0: float = 20.0, width: int | None = None,
                p: int = 128, sigma: float = 0.04, n_receivers: int = 256) -> Scene:
    """Adjoint workload: n^3, k = 20, centred cube (1/8 of the domain per side),
    k^2 multiplied by 1 + 8 seeded Gaussian bumps (amplitude within +-5%),
    256 receivers on the sphere of radius 0.4, Gaussian source sigma = 0.04."""
    rng = np.random.default_rng(seed)
    width = width or max(2, n // 4)
    lo, hi = centred_box_nodes(n, width)
    h = 1.0 / (n - 1)
    scat = box_mask(3, n, lo, hi)
    c = seeded_centre(rng, 3, n, sigma, np.full(3, lo * h), np.full(3, hi * h))
    scale = gaussian_bumps(rng, n, avoid_lo=np.full(3, lo * h), avoid_hi=np.full(3, hi * h))
    trunk = glorot_mlp(rng, [3, 128, 128, p])
    rec = fibonacci_sphere(n_receivers, 0.4)
    return _finish("bump_cube3d", 3, n, k0, scat, gaussian_source(3, n, c, sigma), trunk=trunk,
                   p=p, k2_scale=scale, extra={"centre": c, "receivers": rec})


# ----------------------------------------------------------------- workloads
# Solver settings of the timed workloads (parameters only, no arithmetic).
BENCH_WORKLOADS = {
    # 3D FP64: 64^3, k = 16, centred 16^3 cube, Gaussian source sigma = 0.04, trunk
    # [3,128,128,128] (p = 128, natural-order selection with tau = 1e-6),
    # DeepONet-BiCGStab with n_r = 3 red-black GS sweeps per trunk-basis correction
    # (the cube experiment's ratio, Sec. 4.1), to 1e-8.
    "cube3d-64": dict(scene="cube3d", n=64, seed=0, method="bicgstab", relax="rbgs", n_r=3,
                      correction="tb", tau=1e-6, tol=1e-8, maxit=20000, restart=30),
    # 3D mixed precision: 128^3, k = 32, seeded submarine, seeded plane wave, seeded
    # trunk [3,256,256,256] (p = 256, tau = 1e-6); DeepONet-BiCGStab with 3 red-black
    # GS sweeps + the trunk-basis correction per preconditioner application (restarted
    # FGMRES(50) stagnates near 1e-5 on this cavity with a seeded trunk), to 1e-6.
    # precision "mixed": complex64 vectors, operator and preconditioner (BF16 basis)
    # with FP64 reliable updates; the same solve on an FP64 handle is the comparison.
    "submarine3d-128": dict(scene="submarine3d", n=128, seed=0, method="bicgstab", relax="rbgs", n_r=3,
                            correction="tb", tau=1e-6, tol=1e-6, maxit=40000, restart=50,
                            precision="mixed"),
}


def make_scene(name: str, **kw) -> Scene:
    return {"square2d": square2d, "cube3d": cube3d, "submarine3d": submarine3d,
            "bump_cube3d": bump_cube3d}[name](**kw)


def batch_scenes(seed: int = 0, count: int = 64, n_min: int = 48, n_max: int = 128, k_range=(8.0, 32.0),
                 p: int = 32, trunk_widths=(3, 64, 64, 32), sigma: float = 0.04, layer_cells: int = LAYER_CELLS):
    """Batched workload: `count` problems on uneven cubic grids, k ~ U[k_range] with at
    least 10 points per wavelength (n >= 10 k / (2 pi) + 1), scatterer drawn from
    {cube, sphere, submarine} with scale U[0.1, 0.3] and a seeded rotation, one
    Gaussian source each (seeded centre outside the scatterer's bounding box)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        k0 = float(rng.uniform(*k_range))
        lo_n = max(n_min, int(math.ceil(10.0 * k0 / (2 * math.pi))) + 1)
        n = int(rng.integers(lo_n, max(lo_n, n_max) + 1))
        shape = ["cube", "sphere", "submarine"][int(rng.integers(3))]
        scale = float(rng.uniform(0.1, 0.3))
        rot = random_rotation(rng)
        if shape == "cube":
            scat = rotated_cube_mask(n, (0.5, 0.5, 0.5), scale / 2, rot)
        elif shape == "sphere":
            scat = sphere_mask(n, (0.5, 0.5, 0.5), scale / 2)
        else:
            scat = submarine_mask(n, rot, scale=scale / 0.7)
        # source centre in the interior box, outside a sphere that encloses the scatterer
        radius = (scale / 2) * (math.sqrt(3.0) if shape == "cube" else 1.0) + 2 * sigma
        h = 1.0 / (n - 1)
        lo, hi = layer_cells * h + sigma, 1.0 - layer_cells * h - sigma
        if hi <= lo or np.linalg.norm(np.full(3, hi) - 0.5) <= radius:
            raise ValueError(f"no room for a source outside the scatterer (n={n}, layer={layer_cells})")
        for _ in range(100000):
            c = rng.uniform(lo, hi, size=3)
            if np.linalg.norm(c - 0.5) > radius:
                break
        else:
            raise RuntimeError("no admissible source centre")
        trunk = glorot_mlp(rng, list(trunk_widths[:-1]) + [p])
        sc = _finish(f"batch{b}", 3, n, k0, scat, gaussian_source(3, n, c, sigma), trunk=trunk, p=p,
                     layer_cells=layer_cells, extra={"shape": shape, "scale": scale, "centre": c})
        out.append(sc)
    return out
