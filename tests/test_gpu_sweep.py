"""The fused complex64 red-black sweep (one launch per full sweep, out of place,
halo rows recomputed per block; Sec. 3.1.1's Gauss-Seidel / SOR / SSOR in red-black
order) against the oracle's FP64 sweeps (oracle/relax.py).

Grids: 36^3 (one warp per row, 16-row blocks), 64^3 (several z chunks) and 130^3
(three warps per row with a ragged last warp, 8-row blocks, a ragged last block
row); one, two and three sweeps (both ping-pong parities, and the copy that an odd
launch count from a given x needs); conj; the stored-k^2 field.  The
hybrid cycle from zero (the mixed preconditioner's path) is checked against the
oracle's rounded-basis cycle on an even grid as well.
"""
import numpy as np
import pytest

import scenes
from oracle import assemble, relax, tb as otb
from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _oracle(kind, A, f, x0, col, omega, sweeps):
    if kind == "rbgs":
        return relax.rbgs(A, f, x0, col, sweeps)
    return (relax.sor if kind == "sor" else relax.ssor)(A, f, x0, col, omega, sweeps)


@pytest.mark.parametrize("n", [36, 64, 130])
@pytest.mark.parametrize("kind,omega", [("rbgs", 1.0), ("sor", 1.3), ("ssor", 1.2)])
def test_fused_sweeps_match_oracle(n, kind, omega):
    s = small_scene(3, n)
    P = problem_for(s)
    col = assemble.colour(3, n)
    rng = s["rng"]
    x0 = rng.standard_normal(n ** 3) + 1j * rng.standard_normal(n ** 3)
    f = s["b"]
    fd, xd = to_dev(f, torch.complex64), to_dev(x0, torch.complex64)
    for sweeps in ((1, 2, 3) if n < 100 else (1, 2)):
        for conj in (0, 1):
            A = s["A"].conj() if conj else s["A"]
            ref = _oracle(kind, A, f, x0, col, omega, sweeps)
            x = P.relax(kind, fd, xd.clone(), sweeps=sweeps, omega=omega, conj=conj).cpu().numpy()
            # complex64 arithmetic: a few units of 2^-24 per sweep, times the sweeps' growth
            assert rel(x, ref) < 3e-6 * sweeps, (sweeps, conj, rel(x, ref))
    P.close()


def test_fused_sweep_with_stored_k2_field():
    n = 38
    s = small_scene(3, n)
    scale = 1.0 + 0.05 * s["rng"].standard_normal(n ** 3)
    k2 = assemble.k2_field(3, n, s["k0"], s["cells"], 0.5, scale)
    A = assemble.assemble(3, n, k2, s["mask"])
    P = problem_for(s, k2=k2)
    col = assemble.colour(3, n)
    x0 = s["rng"].standard_normal(n ** 3) + 1j * s["rng"].standard_normal(n ** 3)
    f = s["b"]
    for kind, omega in (("rbgs", 1.0), ("sor", 0.8)):
        ref = _oracle(kind, A, f, x0, col, omega, 2)
        x = P.relax(kind, to_dev(f, torch.complex64), to_dev(x0, torch.complex64), sweeps=2, omega=omega)
        assert rel(x.cpu().numpy(), ref) < 6e-6, (kind, rel(x.cpu().numpy(), ref))


@pytest.mark.parametrize("n_r", [1, 3])
def test_mixed_cycle_from_zero_on_even_grid(n_r):
    """The mixed preconditioner's red-black part runs as fused sweeps from zero on
    even grids; the cycle matches the oracle's FP64 evaluation of the same
    rounded-basis cycle."""
    import paper_2405_12380_gb300 as hm
    n = 36
    s = small_scene(3, n)
    layers = scenes.glorot_mlp(np.random.default_rng(3), [3, 64, 64, 40])
    P = problem_for(s, precision="mixed")
    k = P.don_load(layers, 40, tau=1e-3)
    so = otb.tb_setup(s["A"], layers, scenes.node_coords(3, n), s["mask"], 40, tau=1e-3)
    sm = otb.mixed_setup(so, s["A"])
    assert k == len(sm.kept)
    r = s["rng"].standard_normal(n ** 3) + 1j * s["rng"].standard_normal(n ** 3)
    r[s["mask"] == 1] = 0
    z = P.precond(to_dev(r), hm.opts("bicgstab", "rbgs", n_r)).cpu().numpy()
    ref = otb.hybrid_preconditioner(s["A"], sm, "rbgs", n_r, colours=assemble.colour(3, n))(r)
    assert rel(z, ref) < 1e-4, rel(z, ref)
    # without the correction: the sweeps alone
    z0 = P.precond(to_dev(r), hm.opts("bicgstab", "rbgs", n_r, correction="none")).cpu().numpy()
    ref0 = relax.rbgs(s["A"], r, np.zeros_like(r), assemble.colour(3, n), n_r)
    assert rel(z0, ref0) < 3e-6 * n_r, rel(z0, ref0)
