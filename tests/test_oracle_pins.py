"""Pins of oracle functions against values worked out by hand, a library routine
and a closed form, chosen so that a plausible slip in each fails:

* Adam (App. B: Adam, constant learning rate): three steps with gradients 1, 2, -1
  against the moments worked out by hand from Kingma and Ba's definition, and
  against torch.optim.Adam.  Swapping beta1 and beta2, or dropping either bias
  correction at t >= 2, changes the second step.
* The nonlinear DeepONet correction (Eq. 3 with M2 = DeepONet inference; App. B:
  the branch output splits into a real and an imaginary coefficient group): a
  two-node case whose answer changes if the groups are swapped, if the input is
  ordered [Im, Re], if the scale s = ||r|| is not restored, or if the ReLU of the
  hidden layer is dropped.
* The hybrid iteration (Eq. 3): the correction acts on the residual after the
  relaxation step, f - A u^(i+1/2); a 2 x 2 case where acting on the pre-sweep
  residual gives another iterate.
* The 3D operator against the free-space Green's function (Eq. 1 without a
  scatterer): a point source in a cube with a wide absorbing layer gives
  -exp(ikr) / (4 pi r) within a few percent for r in [0.1, 0.3], |u| ~ r^-1, and
  the outgoing phase (a layer of the wrong sign gives an incoming wave).
"""
import numpy as np
import pytest

import scenes
from oracle import assemble, krylov, mlp


# ------------------------------------------------------------------ Adam
# beta1 = 0.9, beta2 = 0.999, lr = 0.1, parameter 0, gradients g1 = 1, g2 = 2, g3 = -1:
#   m1 = 0.1             v1 = 0.001             m^1 = 1                 v^1 = 1
#   m2 = 0.09 + 0.2      v2 = 0.000999 + 0.004  m^2 = 0.29 / 0.19       v^2 = 0.004999 / 0.001999
#   m3 = 0.261 - 0.1     v3 = 0.004994001 + .001 m^3 = 0.161 / 0.271     v^3 = 0.005994001 / 0.002997001
# (1 - 0.9^2 = 0.19, 1 - 0.999^2 = 0.001999, 1 - 0.9^3 = 0.271, 1 - 0.999^3 = 0.002997001)
ADAM_M = [0.1, 0.29, 0.161]
ADAM_V = [0.001, 0.004999, 0.005994001]
ADAM_STEP = [1.0, (29 / 19) / np.sqrt(4999 / 1999), (161 / 271) / np.sqrt(5994001 / 2997001)]


def test_adam_three_steps_by_hand():
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    expect = 0.0
    for t, g in enumerate([1.0, 2.0, -1.0], start=1):
        p, m, v = mlp.adam_step(p, np.array([g]), m, v, t, lr=0.1, eps=0.0)
        expect -= 0.1 * ADAM_STEP[t - 1]
        assert m[0] == pytest.approx(ADAM_M[t - 1], rel=1e-13)
        assert v[0] == pytest.approx(ADAM_V[t - 1], rel=1e-13)
        assert p[0] == pytest.approx(expect, rel=1e-13)


def test_adam_matches_torch_optimizer():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(7)
    grads = [rng.standard_normal(7) for _ in range(4)]
    w = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(7), np.zeros(7)
    for t, g in enumerate(grads, start=1):
        opt.zero_grad()
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=1e-2)
        assert np.allclose(p, w.detach().numpy(), rtol=0, atol=1e-14)


# -------------------------------------------------- nonlinear correction
def test_nonlinear_correction_by_hand():
    # r = (3 + 4i, 0): s = 5, branch input [Re r, Im r] / s = [0.6, 0, 0.8, 0]
    r = np.array([3 + 4j, 0.0])
    T = np.array([[2.0], [1.0]])                   # p = 1, raw trunk values at the two nodes
    # one linear layer picking b_re = x0 + 0.1 and b_im = x2 - 0.2
    lin = [(np.array([[1.0, 0, 0, 0], [0, 0, 1.0, 0]]), np.array([0.1, -0.2]))]
    z = mlp.nonlinear_correction(lin, T, r)
    # b = 0.7 + 0.6i; z = s T b = 5 (2, 1) (0.7 + 0.6i)
    assert np.allclose(z, [7 + 6j, 3.5 + 3j], rtol=0, atol=1e-14)
    # a ReLU hidden layer: h = relu(x0, -x0) = (0.6, 0); out = (h0 + h1, 2 h1) = (0.6, 0)
    hid = [(np.array([[1.0, 0, 0, 0], [-1.0, 0, 0, 0]]), np.zeros(2)),
           (np.array([[1.0, 1.0], [0.0, 2.0]]), np.zeros(2))]
    z = mlp.nonlinear_correction(hid, T, r)
    assert np.allclose(z, [6.0, 3.0], rtol=0, atol=1e-14)


# ------------------------------------------------------------ Eq. 3 order
def test_hybrid_iteration_corrects_the_post_sweep_residual():
    # A = [[2, 1], [1, 3]], f = (1, 0), u0 = 0, one undamped Jacobi step, M2 r = r / 2:
    #   u^(1/2) = D^-1 f = (0.5, 0); f - A u^(1/2) = (0, -0.5); u^1 = (0.5, -0.25)
    # (the pre-sweep residual f - A u0 = (1, 0) would give (1, 0));
    #   f - A u^1 = (0.25, 0.25), relative norm sqrt(0.125) / 1
    A = np.array([[2.0, 1.0], [1.0, 3.0]], dtype=complex)
    f = np.array([1.0, 0.0], dtype=complex)
    x, info = krylov.relaxation_metasolver(A, f, np.zeros(2, complex), "jacobi", 1, correction=lambda r: 0.5 * r,
                                           omega=1.0, tol=1e-300, max_cycles=1)
    assert np.allclose(x, [0.5, -0.25], rtol=0, atol=1e-15)
    assert info["res"][0] == 1.0
    assert info["res"][1] == pytest.approx(np.sqrt(0.125), rel=1e-14)


# ------------------------------------------------------- 3D free space
def test_free_space_3d_green_function():
    n, k0 = 49, 16.0
    h = 1.0 / (n - 1)
    mask = scenes.ring_mask(3, n).reshape(-1).astype(np.uint8)
    A = assemble.assemble(3, n, assemble.k2_field(3, n, k0, 10, 2.0), mask)
    c = (n // 2) * (1 + n + n * n)
    f = np.zeros(n ** 3, complex)
    f[c] = 1.0 / h ** 3
    b = assemble.rhs(3, n, mask, f, np.zeros(n ** 3, complex))
    u, info = krylov.bicgstab(A, b, np.zeros_like(b), None, 1e-10, 5000)
    assert info["status"] == "converged"
    X = scenes.node_coords(3, n)
    r = np.linalg.norm(X - X[c], axis=1)
    sel = (r >= 0.1) & (r <= 0.3)
    ref = -np.exp(1j * k0 * r[sel]) / (4 * np.pi * r[sel])
    assert np.linalg.norm(u[sel] - ref) / np.linalg.norm(ref) < 0.05
    slope = np.polyfit(np.log(r[sel]), np.log(np.abs(u[sel])), 1)[0]
    assert -1.1 < slope < -0.9, slope
    # outgoing: the phase of u advances like +k r
    assert abs(np.angle(np.vdot(ref, u[sel]))) < 0.1
