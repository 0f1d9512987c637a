"""Pins for oracle.relax, oracle.tb and oracle.krylov (Sec. 3.1, Eqs. 2-3, App. C):
library special cases, matrix splittings, invariants and brute force."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble, krylov, relax, tb


def _small(n=20, dim=2, k0=9.0, cells=4, seed=0, box=(8, 11)):
    rng = np.random.default_rng(seed)
    mask = (scenes.ring_mask(dim, n) | scenes.box_mask(dim, n, *box)).reshape(-1).astype(np.uint8)
    k2 = assemble.k2_field(dim, n, k0, cells, 0.5)
    A = assemble.assemble(dim, n, k2, mask)
    N = n ** dim
    src = np.where(mask == 0, rng.standard_normal(N) + 1j * rng.standard_normal(N), 0)
    b = assemble.rhs(dim, n, mask, src, np.zeros(N, complex))
    return A, b, mask, rng


# ----------------------------------------------------------------- relaxation
def test_jacobi_matches_splitting_form():
    """Damped Jacobi written as x' = (1-w) x + w D^-1 (f - (L+U) x)."""
    A, b, mask, rng = _small()
    x0 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    D = sp.diags(A.diagonal())
    LU_ = A - D
    x = x0.copy()
    for _ in range(3):
        x = (1 - 0.6) * x + 0.6 * (b - LU_ @ x) / A.diagonal()
    y = relax.jacobi(A, b, x0, 0.6, 3)
    assert np.linalg.norm(x - y) <= 1e-13 * np.linalg.norm(x)


def test_rbgs_equals_lexicographic_gs_on_permuted_system():
    """Red-black GS = forward GS on the red-first permuted matrix."""
    A, b, mask, rng = _small(n=11, box=(4, 6))
    n, dim = 11, 2
    col = assemble.colour(dim, n)
    perm = np.concatenate([np.flatnonzero(col == 0), np.flatnonzero(col == 1)])
    P = A[perm][:, perm].tocsr()
    bp = b[perm]
    x0 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    xp = x0[perm].copy()
    L = sp.tril(P, 0).tocsr()
    U = sp.triu(P, 1).tocsr()
    for _ in range(2):
        xp = spla.spsolve_triangular(L, bp - U @ xp, lower=True)
    y = relax.rbgs(A, b, x0, col, 2)
    assert np.linalg.norm(y[perm] - xp) <= 1e-12 * np.linalg.norm(xp)


def test_residual_after_black_half_sweep_lives_on_red_rows():
    """After a red-black sweep that ends with the black half-sweep, f - A x is zero
    (to rounding) on black rows (each was just solved given its red neighbours, the
    only ones it couples to) and on masked rows (x = f there): the projection of
    the hybrid cycle needs only the red rows."""
    for dim, n, box in ((2, 13, (5, 7)), (3, 9, (3, 5))):
        rng = np.random.default_rng(5)
        mask = (scenes.ring_mask(dim, n) | scenes.box_mask(dim, n, *box)).reshape(-1).astype(np.uint8)
        A = assemble.assemble(dim, n, assemble.k2_field(dim, n, 7.0, 2, 0.5), mask)
        N = n ** dim
        f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        col = assemble.colour(dim, n)
        for sweeps in (1, 3):
            x = relax.rbgs(A, f, np.zeros(N, complex), col, sweeps)
            r = f - A @ x
            red_fluid = (col == 0) & (mask == 0)
            rest = ~red_fluid
            assert np.linalg.norm(r[rest]) <= 1e-13 * np.linalg.norm(r[red_fluid]) * max(1.0, np.abs(A).max()), \
                (dim, sweeps, np.linalg.norm(r[rest]), np.linalg.norm(r[red_fluid]))
            assert np.linalg.norm(r[red_fluid]) > 0


def test_colour_is_checkerboard():
    c = assemble.colour(3, 4).reshape(4, 4, 4)
    assert c[0, 0, 0] == 0 and c[0, 0, 1] == 1 and c[1, 1, 0] == 0 and c[1, 2, 3] == 0


def test_relaxations_converge_on_poisson():
    """k = 0 (negative-definite Laplacian): Jacobi and RBGS converge to the LU solution."""
    n = 12
    mask = scenes.ring_mask(2, n).reshape(-1).astype(np.uint8)
    A = assemble.assemble(2, n, np.zeros(n * n, complex), mask)
    rng = np.random.default_rng(0)
    b = np.where(mask == 0, rng.standard_normal(n * n), 0).astype(complex)
    u = spla.spsolve(A.tocsc(), b)
    xj = relax.jacobi(A, b, np.zeros_like(b), 1.0, 2000)
    xg = relax.rbgs(A, b, np.zeros_like(b), assemble.colour(2, n), 800)
    assert np.linalg.norm(xj - u) <= 1e-9 * np.linalg.norm(u)
    assert np.linalg.norm(xg - u) <= 1e-9 * np.linalg.norm(u)


def test_plain_jacobi_diverges_with_scatterer():
    """Sec. 4.1: plain relaxation diverges on the scattering problem."""
    sc = scenes.square2d(0)
    A, b, _ = assemble.problem(sc)
    x, info = krylov.relaxation_metasolver(A, b, np.zeros_like(b), "jacobi", 20, None, max_cycles=200)
    assert info["res"][-1] > 10 * info["res"][0]


# ------------------------------------------------------------------ TB coarse
def _tb_small(p=12):
    A, b, mask, rng = _small()
    X = scenes.node_coords(2, 20)
    layers = scenes.glorot_mlp(rng, [2, 16, 16, p])
    return A, b, mask, rng, X, layers


def test_tb_orthonormal_and_zero_on_mask():
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.tb_setup(A, layers, X, mask, 12)
    assert np.max(np.abs(s.Q.T @ s.Q - np.eye(12))) < 1e-14
    assert np.all(s.Q[mask == 1] == 0)


def test_tb_galerkin_linear_and_basis_invariant():
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.tb_setup(A, layers, X, mask, 12)
    r1 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    r2 = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    z = tb.tb_correct(s, r1)
    # Galerkin: the corrected residual is orthogonal to span(Q)
    assert np.linalg.norm(s.Q.T @ (r1 - A @ z)) <= 1e-12 * np.linalg.norm(s.Q.T @ r1)
    # linear (App. C: M2 is linear, so it may precondition Krylov methods)
    al, be = 0.3 - 1.2j, 2.5 + 0.1j
    lhs = tb.tb_correct(s, al * r1 + be * r2)
    assert np.linalg.norm(lhs - al * z - be * tb.tb_correct(s, r2)) <= 1e-12 * np.linalg.norm(lhs)
    # depends only on span(T): any change of basis (incl. column signs) gives the same M2
    T = tb.trunk_matrix(layers, X, mask, 12)
    G = rng.standard_normal((12, 12)) * np.sign(rng.standard_normal(12))
    Q2, _ = np.linalg.qr(T @ G)
    s2 = tb.tb_setup(A, None, X, mask, 12, Q=Q2)
    assert np.linalg.norm(tb.tb_correct(s2, r1) - z) <= 1e-10 * np.linalg.norm(z)


def test_tb_full_space_is_exact_inverse():
    """p = number of fluid nodes, Q spanning the fluid space: one correction solves A u = f."""
    A, b, mask, rng = _small(n=9, box=(3, 4))
    fluid = np.flatnonzero(mask == 0)
    Q = np.zeros((b.size, fluid.size))
    Q[fluid, np.arange(fluid.size)] = 1.0
    s = tb.tb_setup(A, None, None, mask, fluid.size, Q=Q)
    u = spla.spsolve(A.tocsc(), b)
    z = tb.tb_correct(s, b)          # b = 0 on masked nodes, so u = 0 there too
    assert np.linalg.norm(z - u) <= 1e-12 * np.linalg.norm(u)


def test_hybrid_preconditioner_without_stages_is_identity():
    A, b, mask, rng = _small()
    r = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    assert np.array_equal(tb.hybrid_preconditioner(A, None, "none", 0)(r), r)
    assert np.array_equal(tb.hybrid_preconditioner(A, None, "jacobi", 0)(r), r)


def test_hybrid_preconditioner_p0_is_plain_relaxation():
    A, b, mask, rng = _small()
    r = rng.standard_normal(b.size) + 0j
    M = tb.hybrid_preconditioner(A, None, "jacobi", 3)
    assert np.array_equal(M(r), relax.jacobi(A, r, np.zeros_like(r), 0.6, 3))


def test_mlp_forward_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    layers = scenes.glorot_mlp(rng, [3, 10, 7, 5])
    X = rng.random((13, 3))
    net = []
    for i, (W, bb) in enumerate(layers):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W)); lin.bias.copy_(torch.from_numpy(bb + 0.1 * i))
        net += [lin, torch.nn.Tanh()]
    seq = torch.nn.Sequential(*net[:-1])
    layers_b = [(W, bb + 0.1 * i) for i, (W, bb) in enumerate(layers)]
    ref = seq(torch.from_numpy(X)).detach().numpy()
    assert np.max(np.abs(tb.mlp_forward(layers_b, X) - ref)) < 1e-14


def test_leaky_relu_trunk_matches_torch():
    """The trunk of App. B with Leaky ReLU hidden layers (slope 0.01, PyTorch's default)
    against torch; and the activation's derivative from its output against autograd."""
    torch = pytest.importorskip("torch")
    from oracle import mlp
    rng = np.random.default_rng(8)
    layers = scenes.glorot_mlp(rng, [3, 12, 9, 6])
    X = rng.random((17, 3)) * 2 - 1
    net = []
    for i, (W, bb) in enumerate(layers):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W)); lin.bias.copy_(torch.from_numpy(bb - 0.2 * i))
        net += [lin, torch.nn.LeakyReLU()]
    seq = torch.nn.Sequential(*net[:-1])
    layers_b = [(W, bb - 0.2 * i) for i, (W, bb) in enumerate(layers)]
    ref = seq(torch.from_numpy(X)).detach().numpy()
    out = tb.mlp_forward(layers_b, X, tb.leaky_relu)
    assert np.max(np.abs(out - ref)) < 1e-14
    assert np.max(np.abs(out - tb.mlp_forward(layers_b, X))) > 1e-3      # not the tanh network
    a = torch.linspace(-2, 2, 41, dtype=torch.float64, requires_grad=True)
    y = torch.nn.functional.leaky_relu(a)
    y.sum().backward()
    d = mlp.leaky_relu_deriv(mlp.leaky_relu(a.detach().numpy()))
    assert np.allclose(d[a.detach().numpy() != 0], a.grad.numpy()[a.detach().numpy() != 0], rtol=0, atol=0)


# --------------------------------------------------------------------- Krylov
def test_givens_zeroes_second_component():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, bb = rng.standard_normal(2) @ [1, 1j], rng.standard_normal(2) @ [1, 1j]
        c, s, r = krylov.givens(a, bb)
        assert abs(c * a + s * bb - r) < 1e-14 and abs(-np.conj(s) * a + c * bb) < 1e-14
        assert abs(c ** 2 + abs(s) ** 2 - 1) < 1e-14
    assert krylov.givens(0.0, 2.0 + 0j)[2] == 2.0


def test_fgmres_unpreconditioned_matches_scipy_gmres():
    """Identity preconditioner: the per-step residual estimates equal scipy's GMRES."""
    A, b, mask, rng = _small()
    x, info = krylov.fgmres(A, b, np.zeros_like(b), None, tol=1e-10, m=20, maxit=20)
    ref = []
    spla.gmres(A, b, rtol=1e-14, restart=20, maxiter=1, callback=lambda pr: ref.append(pr),
               callback_type="pr_norm")
    ref = np.asarray(ref[: len(info["est"])])
    assert np.allclose(info["est"], ref, rtol=1e-8, atol=0)


def test_fgmres_flexible_arnoldi_relation_and_monotone():
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.tb_setup(A, layers, X, mask, 12)
    M = tb.hybrid_preconditioner(A, s, "jacobi", 1)
    x, info = krylov.fgmres(A, b, np.zeros_like(b), M, tol=1e-14, m=15, maxit=15, keep_first=True)
    f = info["first"]
    k = f["k"]
    V, Z, H = f["V"][: k + 1], f["Z"][:k], f["H"][: k + 1, :k]
    AZ = np.stack([A @ z for z in Z])
    assert np.linalg.norm(AZ.T - V.T @ H) <= 1e-12 * np.linalg.norm(AZ)
    assert np.max(np.abs(V.conj() @ V.T - np.eye(k + 1))) < 1e-13     # CGS2 orthogonality
    est = np.asarray(info["est"])
    assert np.all(np.diff(est) <= 1e-15)
    # the Givens estimate equals the true residual at the end of the cycle
    assert abs(info["res"][-1] - est[-1]) <= 1e-9 * est[-1]


def test_gmres_full_space_terminates():
    """GMRES(m >= N) on a tiny system reaches 1e-12 in at most N steps."""
    A, b, mask, rng = _small(n=6, box=(2, 3))
    N = b.size
    x, info = krylov.fgmres(A, b, np.zeros_like(b), None, tol=1e-12, m=N, maxit=N)
    assert info["status"] == "converged" and info["iters"] <= N


def test_bicgstab_unpreconditioned_matches_scipy():
    """Identity preconditioner: the iterates equal scipy's BiCGStab step by step."""
    A, b, mask, rng = _small()
    xs = []
    spla.bicgstab(A, b, x0=np.zeros_like(b), rtol=1e-30, maxiter=8, callback=lambda xk: xs.append(xk.copy()))
    for k in (1, 3, 8):
        x, info = krylov.bicgstab(A, b, np.zeros_like(b), None, tol=1e-30, maxit=k)
        assert np.linalg.norm(x - xs[k - 1]) <= 1e-10 * np.linalg.norm(xs[k - 1])


def test_krylov_metasolvers_reach_lu_solution():
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.tb_setup(A, layers, X, mask, 12)
    u = spla.spsolve(A.tocsc(), b)
    for method in ("fgmres", "bicgstab"):
        M = tb.hybrid_preconditioner(A, s, "jacobi" if method == "fgmres" else "rbgs", 1,
                                     colours=assemble.colour(2, 20))
        if method == "fgmres":
            x, info = krylov.fgmres(A, b, np.zeros_like(b), M, tol=1e-11, m=30, maxit=500)
        else:
            x, info = krylov.bicgstab(A, b, np.zeros_like(b), M, tol=1e-11, maxit=500)
        assert info["status"] == "converged"
        assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
        assert np.linalg.norm(x - u) <= 1e-8 * np.linalg.norm(u)


def test_don_krylov_fewer_iterations_than_plain():
    """Sec. 4.1 (qualitative): the DeepONet-Krylov method needs far fewer iterations."""
    sc = scenes.square2d(0)
    A, b, _ = assemble.problem(sc)
    s = tb.tb_setup(A, sc.trunk, scenes.node_coords(2, sc.n), sc.mask, sc.p)
    M = tb.hybrid_preconditioner(A, s, "jacobi", 1)
    _, i1 = krylov.bicgstab(A, b, np.zeros_like(b), M, 1e-8, 2000)
    _, i0 = krylov.bicgstab(A, b, np.zeros_like(b), None, 1e-8, 2000)
    assert i1["status"] == "converged" and i1["iters"] * 2 < i0["iters"]


def test_natural_order_select_matches_householder_span():
    """tau = 0 and a well-conditioned T: same span as numpy's Householder QR;
    dependent columns are dropped; kept columns are orthonormal."""
    rng = np.random.default_rng(6)
    T = rng.standard_normal((200, 8))
    Q, kept = tb.natural_order_select(T, 0.0)
    Qh, _ = np.linalg.qr(T)
    assert kept == list(range(8))
    assert np.linalg.norm(Q @ Q.T - Qh @ Qh.T) < 1e-13
    # plant two dependent columns: a copy and a combination
    T2 = np.column_stack([T[:, 0], T[:, 1], 2 * T[:, 0], T[:, 2], T[:, 1] - T[:, 2] + 1e-12 * T[:, 3]])
    Q2, kept2 = tb.natural_order_select(T2, 1e-6)
    assert kept2 == [0, 1, 3]
    assert np.max(np.abs(Q2.T @ Q2 - np.eye(3))) < 1e-14
    Qh3, _ = np.linalg.qr(T[:, :3])
    assert np.linalg.norm(Q2 @ Q2.T - Qh3 @ Qh3.T) < 1e-13
    # kmax stops early
    assert tb.natural_order_select(T, 0.0, kmax=3)[1] == [0, 1, 2]


def test_oracle_bicgstab_rounding_sensitivity():
    """Documents why BiCGStab iterates are compared only over the first steps: a
    relative perturbation of 1e-15 in f grows by many orders of magnitude within
    ten iterations (while both runs still converge to the same solution)."""
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.tb_setup(A, layers, X, mask, 12)
    M = tb.hybrid_preconditioner(A, s, "rbgs", 1, colours=assemble.colour(2, 20))
    bp = b * (1 + 1e-15 * rng.standard_normal(b.size))
    x1, _ = krylov.bicgstab(A, b, np.zeros_like(b), M, 1e-30, 2)
    x2, _ = krylov.bicgstab(A, bp, np.zeros_like(b), M, 1e-30, 2)
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
    y1, _ = krylov.bicgstab(A, b, np.zeros_like(b), M, 1e-12, 500)
    y2, _ = krylov.bicgstab(A, bp, np.zeros_like(b), M, 1e-12, 500)
    assert np.linalg.norm(y1 - y2) <= 1e-9 * np.linalg.norm(y1)


def test_bf16_round_matches_torch_bfloat16():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    q = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 3, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.5e-3]])
    ref = torch.from_numpy(q.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(tb.bf16_round(q), ref)


def test_mixed_setup_keeps_galerkin_property():
    A, b, mask, rng, X, layers = _tb_small()
    s = tb.mixed_setup(tb.tb_setup(A, layers, X, mask, 12), A)
    r = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
    z = tb.tb_correct(s, r)
    assert np.linalg.norm(s.Q.T @ (r - A @ z)) <= 1e-11 * np.linalg.norm(s.Q.T @ r)
    assert np.max(np.abs(s.Q.T @ s.Q - np.eye(12))) > 1e-5        # BF16 basis is only nearly orthonormal


def test_adjoint_gradient_matches_central_differences():
    """Oracle adjoint gradient against central finite differences of the loss in
    the real and imaginary parts of k^2 on seeded voxels (direct LU solves)."""
    from oracle import adjoint
    n = 13
    rng = np.random.default_rng(11)
    mask = (scenes.ring_mask(3, n) | scenes.box_mask(3, n, 5, 7)).reshape(-1).astype(np.uint8)
    k2 = assemble.k2_field(3, n, 6.0, 3, 0.5) * (1 + 0.05 * rng.standard_normal(n ** 3))
    src = np.where(mask == 0, rng.standard_normal(n ** 3), 0).astype(complex)
    b = assemble.rhs(3, n, mask, src, np.zeros(n ** 3, complex))
    S = adjoint.trilinear(n, scenes.fibonacci_sphere(20, 0.35))
    d = rng.standard_normal(20) + 1j * rng.standard_normal(20)

    def solve(kk):
        return spla.spsolve(assemble.assemble(3, n, kk, mask).tocsc(), b)
    A = assemble.assemble(3, n, k2, mask)
    u = solve(k2)
    g, lam = adjoint.gradient_k2(A, S, u, d, mask, lambda r: spla.spsolve(A.conj().tocsc(), r))
    fluid = np.flatnonzero(mask == 0)
    for l in rng.choice(fluid, 6, replace=False):
        for part, unit in (("re", 1.0), ("im", 1j)):
            eps = 1e-4 * abs(k2[l])
            kp, km = k2.copy(), k2.copy()
            kp[l] += eps * unit
            km[l] -= eps * unit
            fd = (adjoint.loss(S, solve(kp), d) - adjoint.loss(S, solve(km), d)) / (2 * eps)
            an = g[l].real if part == "re" else g[l].imag
            assert abs(fd - an) <= 2e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (l, part, fd, an)
    assert np.all(g[mask == 1] == 0)


def test_trilinear_reproduces_linear_functions():
    from oracle import adjoint
    n = 9
    pts = np.random.default_rng(2).uniform(0.05, 0.95, (30, 3))
    S = adjoint.trilinear(n, pts)
    X = scenes.node_coords(3, n)
    f = 0.3 + 1.7 * X[:, 0] - 0.4 * X[:, 1] + 2.2 * X[:, 2]
    ref = 0.3 + 1.7 * pts[:, 0] - 0.4 * pts[:, 1] + 2.2 * pts[:, 2]
    assert np.max(np.abs(S @ f - ref)) < 1e-13
    assert np.allclose(np.asarray(S.sum(axis=1)).ravel(), 1.0)


def _tiny_deeponet(rng):
    branch = scenes.glorot_mlp(rng, [10, 7, 6, 8])
    trunk = scenes.glorot_mlp(rng, [3, 5, 5, 4])
    branch = [(W, b + 0.1 * rng.standard_normal(b.shape)) for W, b in branch]
    trunk = [(W, b + 0.1 * rng.standard_normal(b.shape)) for W, b in trunk]
    X = rng.standard_normal((3, 10))
    Xc = rng.random((9, 3))
    Y = rng.standard_normal((3, 18))
    return branch, trunk, X, Xc, Y


def test_deeponet_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    from oracle import mlp
    rng = np.random.default_rng(12)
    branch, trunk, X, Xc, Y = _tiny_deeponet(rng)
    pred, ba, ta = mlp.deeponet_forward(branch, trunk, X, Xc)
    loss, dpred = mlp.rel_l2(pred, Y)
    gb, gt = mlp.deeponet_backward(branch, trunk, ba, ta, dpred)
    tb_ = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in branch]
    tt_ = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in trunk]
    h = torch.tensor(X)
    for i, (W, b) in enumerate(tb_):
        h = h @ W.T + b
        if i < len(tb_) - 1:
            h = torch.relu(h)
    t = torch.tensor(Xc)
    for i, (W, b) in enumerate(tt_):
        t = t @ W.T + b
        if i < len(tt_) - 1:
            t = torch.tanh(t)
    p = t.shape[1]
    pr = torch.cat([h[:, :p] @ t.T, h[:, p:] @ t.T], dim=1)
    Yt = torch.tensor(Y)
    L = (((pr - Yt) ** 2).sum(1) / (Yt ** 2).sum(1)).mean()
    L.backward()
    assert abs(L.item() - loss.mean()) < 1e-13
    for (W, b), (dW, db) in zip(tb_ + tt_, gb + gt):
        assert np.max(np.abs(W.grad.numpy() - dW)) < 1e-12
        assert np.max(np.abs(b.grad.numpy() - db)) < 1e-12


def test_deeponet_backward_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(13)
    branch, trunk, X, Xc, Y = _tiny_deeponet(rng)

    def L(br, tr):
        return mlp.rel_l2(mlp.deeponet_forward(br, tr, X, Xc)[0], Y)[0].mean()
    pred, ba, ta = mlp.deeponet_forward(branch, trunk, X, Xc)
    gb, gt = mlp.deeponet_backward(branch, trunk, ba, ta, mlp.rel_l2(pred, Y)[1])
    for which, layers, grads in (("b", branch, gb), ("t", trunk, gt)):
        for _ in range(10):
            li = rng.integers(len(layers))
            W, b = layers[li]
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            eps = 1e-6
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += eps
            Wm[i, j] -= eps
            lp = [(Wp if k == li else w, bb) for k, (w, bb) in enumerate(layers)]
            lm = [(Wm if k == li else w, bb) for k, (w, bb) in enumerate(layers)]
            fd = (L(lp, trunk) - L(lm, trunk)) / (2 * eps) if which == "b" else (L(branch, lp) - L(branch, lm)) / (2 * eps)
            assert abs(fd - grads[li][0][i, j]) < 1e-7 * max(1.0, abs(fd))


def test_nonlinear_correction_is_positively_homogeneous():
    from oracle import mlp
    rng = np.random.default_rng(14)
    N, p = 12, 4
    branch = scenes.glorot_mlp(rng, [2 * N, 9, 2 * p])
    T = rng.standard_normal((N, p))
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    z = mlp.nonlinear_correction(branch, T, r)
    assert np.linalg.norm(mlp.nonlinear_correction(branch, T, 3.7 * r) - 3.7 * z) < 1e-12 * np.linalg.norm(z)
    assert np.all(mlp.nonlinear_correction(branch, T, 0 * r) == 0)


def test_adam_first_step_moves_by_lr():
    from oracle import mlp
    p, m, v = mlp.adam_step(np.array([1.0, -2.0]), np.array([0.3, -5.0]), np.zeros(2), np.zeros(2), 1, lr=1e-3)
    assert np.allclose(p, [1.0 - 1e-3, -2.0 + 1e-3], atol=1e-9)
