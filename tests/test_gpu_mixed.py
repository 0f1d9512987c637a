"""Mixed precision (complex64 preconditioner with a BF16 trunk basis inside the FP64
FGMRES): the preconditioner against the oracle's FP64 evaluation of the same
rounded-basis cycle, and solves that reach 1e-6 on the oracle's own residual."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, krylov, tb as otb
from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _mixed_pair(dim=3, n=37, widths=(3, 64, 64, 40), tau=1e-3):
    s = small_scene(dim, n)
    rng = np.random.default_rng(3)
    layers = scenes.glorot_mlp(rng, list(widths))
    p = widths[-1]
    P = problem_for(s, precision="mixed")
    k = P.don_load(layers, p, tau=tau)
    so = otb.tb_setup(s["A"], layers, scenes.node_coords(dim, n), s["mask"], p, tau=tau)
    return s, P, otb.mixed_setup(so, s["A"]), k


@pytest.mark.parametrize("kind,n_r", [("jacobi", 1), ("rbgs", 1), ("none", 0)])
def test_mixed_precond_matches_rounded_basis_oracle(kind, n_r):
    import paper_2405_12380_gb300 as hm
    s, P, sm, k = _mixed_pair()
    assert k == len(sm.kept)
    # the device basis is the BF16 rounding of the device Q
    Qd = P.basis().cpu().numpy()
    assert np.array_equal(Qd, otb.bf16_round(Qd))
    r = s["rng"].standard_normal(s["A"].shape[0]) + 1j * s["rng"].standard_normal(s["A"].shape[0])
    r[s["mask"] == 1] = 0
    z = P.precond(to_dev(r), hm.opts("fgmres", kind, n_r)).cpu().numpy()
    ref = otb.hybrid_preconditioner(s["A"], sm, kind, n_r, colours=assemble.colour(3, 37))(r)
    assert rel(z, ref) < 1e-4, rel(z, ref)


@pytest.mark.parametrize("n_r", [1, 2])
def test_mixed_fgmres_reaches_tolerance(n_r):
    """(FGMRES with one Jacobi sweep + TB stagnates on this scene in the FP64 oracle
    too, so the red-black GS cycle is used.)"""
    import paper_2405_12380_gb300 as hm
    kind = "rbgs"
    s, P, sm, k = _mixed_pair()
    b = s["b"]
    x, st = P.solve(to_dev(b), None, hm.opts("fgmres", kind, n_r, tol=1e-6, restart=30, maxit=3000))
    assert st["status"] == 0, st["status_name"]
    x = x.cpu().numpy()
    res = np.linalg.norm(b - s["A"] @ x) / np.linalg.norm(b)
    assert res <= 1e-6
    u = spla.spsolve(s["A"].tocsc(), b)
    assert rel(x, u) < 1e-3          # error against the FP64 direct solution (cond(A) times 1e-6)
    # the oracle's FGMRES with the same rounded-basis cycle converges in a similar count
    M = otb.hybrid_preconditioner(s["A"], sm, kind, n_r, colours=assemble.colour(3, 37))
    xo, io = krylov.fgmres(s["A"], b, np.zeros_like(b), M, 1e-6, 30, 3000)
    assert abs(st["iters"] - io["iters"]) <= max(5, 0.2 * io["iters"])


def test_mixed_bicgstab_hands_over_to_fp64_bicgstab_after_runaways():
    """A runaway threshold barely above 1 makes the complex64 BiCGStab restart again
    and again; after four restarts the solve continues as the FP64 BiCGStab with the
    same complex64 cycle and still reaches the tolerance on the oracle's residual (the
    restarts and the hand-over show in the cycle count)."""
    import paper_2405_12380_gb300 as hm
    s, P, sm, k = _mixed_pair(n=36)
    b = s["b"]
    o = hm.opts("bicgstab", "rbgs", 3, tol=1e-6, maxit=3000)
    x0, st0 = P.solve(to_dev(b), None, o)
    assert st0["status"] == 0, st0["status_name"]
    P.set_reliable(delta=0.1, runaway=1.0 + 1e-9, guard=1e2)
    x, st = P.solve(to_dev(b), None, o)
    P.set_reliable()
    assert st["status"] == 0, st["status_name"]
    assert st["cycles"] >= 5, st
    res = np.linalg.norm(b - s["A"] @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1.0001e-6, res
    assert rel(x.cpu().numpy(), x0.cpu().numpy()) < 1e-2
