"""DeepONet kernels: FP32 GEMM, a full training step (forward, backward, Adam)
and the nonlinear branch correction, against the FP64 oracle (oracle/mlp.py)."""
import ctypes as C

import numpy as np
import pytest

import scenes
from oracle import assemble, krylov, mlp, tb as otb
from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("ta,tb,M,N,K", [(0, 0, 70, 130, 33), (1, 0, 64, 65, 17), (0, 1, 5, 300, 1000),
                                         (1, 1, 33, 31, 129), (0, 1, 1, 96, 40000), (1, 0, 96, 4000, 7)])
def test_nn_gemm(ta, tb, M, N, K):
    from paper_2405_12380_gb300 import _lib as L
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    ref = 0.7 * (A.T if ta else A).astype(np.float64) @ (B.T if tb else B).astype(np.float64) - 1.3 * C0
    Ad, Bd, Cd = to_dev(A), to_dev(B), to_dev(C0)
    st = L.lib().nn_gemm(ta, tb, M, N, K, 0.7, C.c_void_p(Ad.data_ptr()), A.shape[1], C.c_void_p(Bd.data_ptr()),
                         B.shape[1], -1.3, C.c_void_p(Cd.data_ptr()), N, None)
    assert st == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(Cd.cpu().numpy() - ref)) <= 2e-6 * np.sqrt(K) * np.max(np.abs(ref)) + 1e-5


@pytest.mark.parametrize("act", [1, 2, 3])
def test_bias_act_and_backward(act):
    """nn_bias_act / nn_act_backward for ReLU, tanh and the trunk's Leaky ReLU (App. B)
    against the oracle's activations and their derivatives from the outputs."""
    from paper_2405_12380_gb300 import _lib as L
    rng = np.random.default_rng(act)
    X = rng.standard_normal((37, 53)).astype(np.float32)
    b = rng.standard_normal(53).astype(np.float32)
    dY = rng.standard_normal((37, 53)).astype(np.float32)
    f, df = {1: (mlp.relu, lambda H: (H > 0).astype(np.float64)),
             2: (np.tanh, lambda H: 1.0 - H * H),
             3: (mlp.leaky_relu, mlp.leaky_relu_deriv)}[act]
    ref = f(X.astype(np.float64) + b)
    Xd, bd, dd = to_dev(X), to_dev(b), to_dev(dY)
    lib = L.lib()
    assert lib.nn_bias_act(37, 53, C.c_void_p(Xd.data_ptr()), C.c_void_p(bd.data_ptr()), act, None) == 0
    torch.cuda.synchronize()
    Y = Xd.cpu().numpy()
    assert np.max(np.abs(Y - ref)) <= 1e-6 * (1 + np.max(np.abs(ref)))
    assert lib.nn_act_backward(Y.size, C.c_void_p(dd.data_ptr()), C.c_void_p(Xd.data_ptr()), act, None) == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(dd.cpu().numpy() - dY * df(Y.astype(np.float64)))) <= 1e-6 * np.max(np.abs(dY))


@pytest.mark.parametrize("B,Ci,D,Co,stride,pad", [(4, 3, 17, 8, 2, 0), (3, 8, 8, 8, 1, 1), (2, 8, 8, 12, 2, 0)])
def test_conv3d_layers_match_oracle(B, Ci, D, Co, stride, pad):
    """The CNN branch's convolution layers (App. B; the three layer shapes of the 3D
    branch with fewer channels): forward and all three gradients against the FP64
    oracle (oracle/cnn.py)."""
    from oracle import cnn
    from paper_2405_12380_gb300 import _lib as L
    rng = np.random.default_rng(B + Ci + D)
    X = rng.standard_normal((B, Ci, D, D, D)).astype(np.float32)
    W = (rng.standard_normal((Co, Ci, 3, 3, 3)) / np.sqrt(27 * Ci)).astype(np.float32)
    b = rng.standard_normal(Co).astype(np.float32)
    Do = cnn.out_size(D, stride, pad)
    dY = rng.standard_normal((B, Co, Do, Do, Do)).astype(np.float32)
    Xd, Wd, bd, dYd = to_dev(X), to_dev(W), to_dev(b), to_dev(dY)
    Yd = torch.empty((B, Co, Do, Do, Do), dtype=torch.float32, device="cuda")
    dXd, dWd, dbd = torch.empty_like(Xd), torch.empty_like(Wd), torch.empty_like(bd)
    p = lambda t: C.c_void_p(t.data_ptr())
    lib = L.lib()
    assert lib.nn_conv3d(B, Ci, D, Co, stride, pad, p(Xd), p(Wd), p(bd), p(Yd), None) == 0
    assert lib.nn_conv3d_backward(B, Ci, D, Co, stride, pad, p(Xd), p(Wd), p(dYd), p(dXd), p(dWd), p(dbd), None) == 0
    torch.cuda.synchronize()
    Y = cnn.conv3d(X, W, b, stride, pad)
    dX, dW, db = cnn.conv3d_backward(X, W, dY, stride, pad)
    # FP32 sums of up to B Do^3 = 2048 products (fixed order)
    assert rel(Yd.cpu().numpy(), Y) < 1e-5
    assert rel(dXd.cpu().numpy(), dX) < 1e-5
    assert rel(dWd.cpu().numpy(), dW) < 1e-5
    assert rel(dbd.cpu().numpy(), db) < 1e-5
    # invalid shapes are rejected before any launch
    assert lib.nn_conv3d(B, Ci, 2, Co, 1, 0, p(Xd), p(Wd), p(bd), p(Yd), None) == L.HELM_BAD_ARG


def test_training_step_matches_oracle():
    from paper_2405_12380_gb300 import train
    rng = np.random.default_rng(21)
    net = train.DeepONet.init([40, 24, 16, 10], [3, 12, 12, 5], seed=4)
    for l in net.branch + net.trunk:                       # non-zero biases
        l.b.copy_(torch.from_numpy((0.1 * rng.standard_normal(l.b.shape[0])).astype(np.float32)))
    X = rng.standard_normal((6, 40)).astype(np.float32)
    Xc = rng.random((23, 3)).astype(np.float32)
    Y = rng.standard_normal((6, 46)).astype(np.float32)
    branch, trunk = net.numpy_layers("branch"), net.numpy_layers("trunk")
    pred, ba, ta_ = mlp.deeponet_forward(branch, trunk, X, Xc)
    loss_o, dpred = mlp.rel_l2(pred, Y.astype(np.float64))
    gb, gt = mlp.deeponet_backward(branch, trunk, ba, ta_, dpred)
    loss = train.train_step(net, to_dev(X), to_dev(Xc), to_dev(Y), lr=1e-3)
    torch.cuda.synchronize()
    assert rel(loss.cpu().numpy(), loss_o) < 1e-5
    for l, (dW, db) in zip(net.branch + net.trunk, gb + gt):
        assert rel(l.gW.cpu().numpy(), dW) < 1e-4
        assert rel(l.gb.cpu().numpy(), db) < 1e-4
    # the first Adam step moves every parameter with a clear gradient by about lr
    for l, (W0, _) in zip(net.branch, branch):
        moved = np.abs(l.W.double().cpu().numpy() - W0)
        g = np.abs(l.gW.cpu().numpy())
        assert np.allclose(moved[g > 1e-4], 1e-3, rtol=1e-2)


def test_three_training_steps_match_oracle_adam():
    """Three forward/backward/Adam steps on the same batch: after each step the
    device parameters equal the oracle's (FP64 gradients of the oracle network at
    the device's current parameters, then oracle Adam with bias correction at
    t = 1, 2, 3; moments carried over)."""
    from paper_2405_12380_gb300 import train
    rng = np.random.default_rng(31)
    net = train.DeepONet.init([30, 20, 12], [2, 10, 10, 6], seed=6)
    X = rng.standard_normal((5, 30)).astype(np.float32)
    Xc = rng.random((17, 2)).astype(np.float32)
    Y = rng.standard_normal((5, 34)).astype(np.float32)
    layers = net.branch + net.trunk
    params = [[l.W.double().cpu().numpy(), l.b.double().cpu().numpy()] for l in layers]
    moments = [[np.zeros_like(a) for a in pr] + [np.zeros_like(a) for a in pr] for pr in params]
    lr = 2e-3
    # entries whose oracle gradient stays clear of zero (an FP32 gradient of a
    # near-zero FP64 one may have the other sign, and Adam moves both by ~lr)
    clear = [[np.ones(a.shape, bool) for a in pr] for pr in params]
    for t in (1, 2, 3):
        nb = len(net.branch)
        branch = [(w, b) for w, b in params[:nb]]
        trunk = [(w, b) for w, b in params[nb:]]
        pred, ba, ta_ = mlp.deeponet_forward(branch, trunk, X, Xc)
        _, dpred = mlp.rel_l2(pred, Y.astype(np.float64))
        gb, gt = mlp.deeponet_backward(branch, trunk, ba, ta_, dpred)
        for q, (dW, db) in enumerate(gb + gt):
            clear[q][0] &= np.abs(dW) > 1e-4
            clear[q][1] &= np.abs(db) > 1e-4
            mW, mb, vW, vb = moments[q]
            params[q][0], mW, vW = mlp.adam_step(params[q][0], dW, mW, vW, t, lr=lr)
            params[q][1], mb, vb = mlp.adam_step(params[q][1], db, mb, vb, t, lr=lr)
            moments[q] = [mW, mb, vW, vb]
        train.train_step(net, to_dev(X), to_dev(Xc), to_dev(Y), lr=lr)
        torch.cuda.synchronize()
        for l, (W, b), (cW, cb) in zip(layers, params, clear):
            # a slip in Adam (betas swapped, a bias correction dropped) moves an
            # entry by several percent of lr at t = 2
            assert np.max(np.abs(l.W.double().cpu().numpy() - W)[cW]) < 5e-3 * lr, t
            assert np.max(np.abs(l.b.double().cpu().numpy() - b)[cb], initial=0) < 5e-3 * lr, t
            assert cW.mean() > 0.5


def test_nonlinear_correction_matches_oracle():
    s = small_scene(3, 21)
    rng = np.random.default_rng(7)
    N = 21 ** 3
    trunk = scenes.glorot_mlp(rng, [3, 16, 16, 8])
    branch = [(W.astype(np.float32).astype(np.float64), b) for W, b in scenes.glorot_mlp(rng, [2 * N, 32, 16])]
    P = problem_for(s)
    P.don_load(trunk, 8, tau=1e-4)
    P.don_load_branch(branch)
    r = s["b"] - s["A"] @ (0.1 * rng.standard_normal(N))
    r[s["mask"] == 1] = 0
    z = P.don_correct_nonlinear(to_dev(r)).cpu().numpy()
    T = otb.trunk_matrix(trunk, scenes.node_coords(3, 21), s["mask"], 8)
    ref = mlp.nonlinear_correction(branch, T, r)
    assert rel(z, ref) < 1e-5
    # positive homogeneity holds on the device too
    z2 = P.don_correct_nonlinear(to_dev(2.5 * r)).cpu().numpy()
    assert rel(z2, 2.5 * z) < 1e-6


def test_nonlinear_relaxation_metasolver_same_iterate():
    import paper_2405_12380_gb300 as hm
    s = small_scene(2, 45)
    rng = np.random.default_rng(9)
    N = 45 ** 2
    trunk = scenes.glorot_mlp(rng, [2, 16, 16, 8])
    branch = [(W.astype(np.float32).astype(np.float64), b) for W, b in scenes.glorot_mlp(rng, [2 * N, 24, 16])]
    P = problem_for(s)
    P.don_load(trunk, 8, tau=1e-4)
    P.don_load_branch(branch)
    x, st = P.solve(to_dev(s["b"]), None, hm.opts("relax", "rbgs", 2, correction="nonlinear", tol=1e-14, maxit=2))
    T = otb.trunk_matrix(trunk, scenes.node_coords(2, 45), s["mask"], 8)
    xo, io = krylov.relaxation_metasolver(s["A"], s["b"], np.zeros_like(s["b"]), "rbgs", 2,
                                          lambda r: mlp.nonlinear_correction(branch, T, r),
                                          colours=assemble.colour(2, 45), tol=1e-14, max_cycles=2)
    assert st["iters"] == io["iters"] == 2
    assert rel(x.cpu().numpy(), xo) < 1e-5


def test_training_reduces_loss_on_scatterer_free_problem():
    import paper_2405_12380_gb300 as hm
    from paper_2405_12380_gb300 import train
    n = 33
    mask = scenes.ring_mask(2, n).reshape(-1).astype(np.uint8)
    P = hm.Problem(2, n, 6.0, mask, layer_cells=4)
    rng = np.random.default_rng(0)
    fs = scenes.grf_samples(rng, 2, n, 48)
    fs[:, mask == 1] = 0
    X, Y, scales = train.make_dataset(P, fs, hm.opts("bicgstab", "rbgs", 2, correction="none", tol=1e-6,
                                                     maxit=3000), log=lambda *a: None)
    net = train.DeepONet.init([2 * n * n, 64, 32], [2, 32, 32, 16], seed=1)
    coords = scenes.node_coords(2, n)
    fluid = np.flatnonzero(mask == 0)
    before = train.evaluate(net, X, Y, coords, range(40, 48))
    train.train(net, X[:40], Y[:40], coords, fluid, steps=400, batch=16, nodes=512, lr=1e-3, log=lambda *a: None)
    after_train = train.evaluate(net, X, Y, coords, range(0, 8))
    assert after_train < 0.5 * before


def _bf16_reference_step(branch, trunk, X, Xc, Y):
    """Loss and gradients of one DeepONet training step in FP64 with every operand of
    every product rounded to BF16 first (oracle/tb.py bf16_round), in the order of
    the products train_step forms; ReLU / tanh, biases and the loss in FP64."""
    from oracle.tb import bf16_round as bf
    acts_b, acts_t = [np.asarray(X, np.float64)], [np.asarray(Xc, np.float64)]
    for li, (W, b) in enumerate(branch):
        H = bf(acts_b[-1]) @ bf(W).T + b
        acts_b.append(np.maximum(H, 0) if li < len(branch) - 1 else H)
    for li, (W, b) in enumerate(trunk):
        H = bf(acts_t[-1]) @ bf(W).T + b
        acts_t.append(np.tanh(H) if li < len(trunk) - 1 else H)
    Bo, T = acts_b[-1], acts_t[-1]
    p = T.shape[1]
    pred = np.concatenate([bf(Bo[:, :p]) @ bf(T).T, bf(Bo[:, p:]) @ bf(T).T], axis=1)
    loss, dpred = mlp.rel_l2(pred, np.asarray(Y, np.float64))
    P = T.shape[0]
    dBo = np.concatenate([bf(dpred[:, :P]) @ bf(T), bf(dpred[:, P:]) @ bf(T)], axis=1)
    dT = bf(dpred[:, :P]).T @ bf(Bo[:, :p]) + bf(dpred[:, P:]).T @ bf(Bo[:, p:])

    def back(layers, acts, d, deriv):
        grads = [None] * len(layers)
        for li in range(len(layers) - 1, -1, -1):
            if li < len(layers) - 1:
                d = d * deriv(acts[li + 1])
            grads[li] = (bf(d).T @ bf(acts[li]), d.sum(axis=0))
            d = bf(d) @ bf(layers[li][0])
        return grads
    gb = back(branch, acts_b, dBo, lambda H: (H > 0).astype(np.float64))
    gt = back(trunk, acts_t, dT, lambda H: 1.0 - H * H)
    return loss, gb, gt


def test_training_step_on_tensor_cores():
    """The same training step with the dense-layer products on the tcgen05 tensor
    cores (BF16 operands, FP32 accumulation) against the oracle's FP64 arithmetic
    with the operands of every product rounded to BF16 (what remains is the FP32
    accumulation and BF16 ties of nearly equal FP32 / FP64 values: 1e-2), and the
    loss falls over a short run."""
    from paper_2405_12380_gb300 import train
    rng = np.random.default_rng(23)
    net = train.DeepONet.init([64, 48, 32, 20], [3, 24, 24, 10], seed=5)
    X = rng.standard_normal((8, 64)).astype(np.float32)
    Xc = rng.random((40, 3)).astype(np.float32)
    Y = rng.standard_normal((8, 80)).astype(np.float32)
    branch, trunk = net.numpy_layers("branch"), net.numpy_layers("trunk")
    loss_o, gb, gt = _bf16_reference_step(branch, trunk, X, Xc, Y)
    train.set_tensor_cores(True)
    try:
        loss = train.train_step(net, to_dev(X), to_dev(Xc), to_dev(Y), lr=1e-3)
        torch.cuda.synchronize()
        assert rel(loss.cpu().numpy(), loss_o) < 1e-2
        for l, (dW, db) in zip(net.branch + net.trunk, gb + gt):
            assert rel(l.gW.cpu().numpy(), dW) < 1e-2, rel(l.gW.cpu().numpy(), dW)
            assert rel(l.gb.cpu().numpy(), db) < 1e-2, rel(l.gb.cpu().numpy(), db)
        l0 = float(loss.mean())
        for _ in range(60):
            loss = train.train_step(net, to_dev(X), to_dev(Xc), to_dev(Y), lr=1e-3)
        assert float(loss.mean()) < 0.97 * l0
    finally:
        train.set_tensor_cores(False)
    import ctypes as C
    from paper_2405_12380_gb300 import _lib as L
    flag = C.c_int(-1)
    assert L.lib().nn_gemm_bf16_status(C.byref(flag)) == 0 and flag.value == 0
