"""Checks at the full sizes of the timed workloads, on outputs the oracle can
compute cheaply: the 128^3 mixed-precision solve against the oracle's own FP64
residual, and the 96^3 adjoint workload against the oracle's receiver data
(tests/golden/adjoint_d_bump_cube3d-96.npz, written by oracle/adjoint_data.py)
with its gradient checked by central differences.

With the seeded (untrained) trunk, restarted FGMRES stagnates near 1e-5 on
these cavities, so both use BiCGStab with three red-black Gauss-Seidel sweeps
and the trunk-basis correction per preconditioner application."""
import os

import numpy as np
import pytest

import scenes
from oracle import adjoint, assemble
from tests.gpu_common import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_mixed_128_reaches_tolerance_on_oracle_residual():
    import paper_2405_12380_gb300 as hm
    w = scenes.BENCH_WORKLOADS["submarine3d-128"]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength,
                   precision="mixed")
    f = P.rhs(to_dev(sc.src), to_dev(sc.g))
    P.don_load(sc.trunk, sc.p, tau=w["tau"])
    o = hm.opts("bicgstab", "rbgs", 3, tol=1e-6, maxit=20000)
    x, st = P.solve(f, None, o)
    assert st["status"] == 0, st["status_name"]
    A = assemble.assemble(3, sc.n, assemble.k2_field(3, sc.n, sc.k0, sc.layer_cells, sc.layer_strength), sc.mask)
    b = assemble.rhs(3, sc.n, sc.mask, sc.src, sc.g)
    assert np.allclose(f.cpu().numpy(), b, rtol=0, atol=1e-12 * np.abs(b).max())
    xh = x.cpu().numpy()
    res = np.linalg.norm(b - A @ xh) / np.linalg.norm(b)
    assert res <= 1.0001e-6, res
    assert abs(res - st["rel_res"]) <= 1e-9, (res, st["rel_res"])
    # against the oracle's own solution (tests/golden/solution_submarine3d-128.npz, written
    # by oracle/reference_data.py: its BiCGStab continued to 1e-10) on the stored node
    # sample: the error of a solve to 1e-6 is set by the conditioning, so it is compared
    # with the error the oracle's own iterate at 1e-6 makes
    gpath = os.path.join(HERE, "golden", "solution_submarine3d-128.npz")
    if os.path.exists(gpath):
        gold = np.load(gpath)
        idx = gold["idx"]
        err = np.linalg.norm(xh[idx] - gold["x"]) / np.linalg.norm(gold["x"])
        err_tol = np.linalg.norm(gold["x_tol"] - gold["x"]) / np.linalg.norm(gold["x"])
        assert err <= max(20 * err_tol, 1e-3), (err, err_tol)


def test_adjoint_96_against_oracle_data_and_central_differences():
    import paper_2405_12380_gb300 as hm
    from paper_2405_12380_gb300.autograd import misfit_loss
    sc = scenes.bump_cube3d(0, n=96)
    gold = np.load(os.path.join(HERE, "golden", "adjoint_d_bump_cube3d-96.npz"))
    d = to_dev(gold["d"])
    k20 = assemble.k2_field(3, sc.n, sc.k0, sc.layer_cells, sc.layer_strength)
    k2 = assemble.k2_field(3, sc.n, sc.k0, sc.layer_cells, sc.layer_strength, sc.k2_scale)
    P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength,
                   k2=to_dev(k20))
    f = P.rhs(to_dev(sc.src), to_dev(sc.g))
    P.don_load(sc.trunk, sc.p, tau=1e-6)
    o = hm.opts("bicgstab", "rbgs", 3, tol=1e-10, maxit=20000)
    idx, w = P.receivers(sc.extra["receivers"])
    # forward solve of the unperturbed field against the oracle's receiver data
    u0, st = P.solve(f, None, o)
    assert st["status"] == 0
    e0 = (P.sample(idx, w, u0) - d).cpu().numpy()
    assert np.linalg.norm(e0) <= 1e-6 * np.linalg.norm(gold["d"]), np.linalg.norm(e0) / np.linalg.norm(gold["d"])
    S = adjoint.trilinear(sc.n, sc.extra["receivers"])
    assert np.allclose(P.sample(idx, w, u0).cpu().numpy(), S @ u0.cpu().numpy(), rtol=1e-13, atol=0)
    # gradient of the misfit of the perturbed field against central differences
    k2t = to_dev(k2).requires_grad_(True)
    L, u = misfit_loss(k2t, f, P, o, idx, w, d)
    L.backward()
    g = k2t.grad.cpu().numpy()
    assert np.all(g[sc.mask.reshape(-1) == 1] == 0)
    gmax = np.abs(g).max()
    rng = np.random.default_rng(11)
    fluid = np.flatnonzero(sc.mask.reshape(-1) == 0)
    for l in rng.choice(fluid, 2, replace=False):
        for unit, part in ((1.0, "re"), (1j, "im")):
            eps = 1e-3 * abs(k2[l])
            vals = []
            for sgn in (1, -1):
                kk = k2.copy()
                kk[l] += sgn * eps * unit
                P.set_k2(to_dev(kk))
                uu, s2 = P.solve(f, None, o)
                assert s2["status"] == 0
                e = P.sample(idx, w, uu) - d
                vals.append(float((e.real ** 2 + e.imag ** 2).sum().item()))
            fd = (vals[0] - vals[1]) / (2 * eps)
            an = g[l].real if part == "re" else g[l].imag
            assert abs(fd - an) <= 2e-3 * max(abs(fd), 1e-2 * gmax), (l, part, fd, an)


def test_batched_bicgstab_config4_problems_at_full_size():
    """The first eight problems of the batched workload (uneven grids 48^3-128^3, k in
    [8, 32], cube / sphere / submarine scatterers, p = 32), solved together by the
    batched complex64 BiCGStab (3 red-black sweeps + trunk basis) to 1e-6; each
    solution is checked on the oracle's own FP64 residual."""
    import paper_2405_12380_gb300 as hm
    scs = scenes.batch_scenes(0, count=64)[:8]
    probs, fs = [], []
    for sc in scs:
        P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, precision="mixed")
        P.don_load(sc.trunk, sc.p, tau=1e-6)
        probs.append(P)
        fs.append(P.rhs(to_dev(sc.src), to_dev(sc.g)))
    B = hm.Batch(probs)
    xs, st = B.solve(fs, None, hm.opts("bicgstab", "rbgs", 3, tol=1e-6, maxit=20000))
    for sc, x, s in zip(scs, xs, st):
        assert s["status"] == 0, (sc.n, sc.k0, s["status_name"], s["iters"], s["rel_res"])
        A = assemble.assemble(3, sc.n, assemble.k2_field(3, sc.n, sc.k0, sc.layer_cells, sc.layer_strength),
                              sc.mask)
        b = assemble.rhs(3, sc.n, sc.mask, sc.src, sc.g)
        res = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
        assert res <= 1.0001e-6, (sc.n, res)
    B.close()
