"""The CNN-branch convolution of the oracle (oracle/cnn.py, App. B) against torch's
conv3d and its autograd gradients in FP64 (an independent implementation), at the
three layer shapes of the 3D branch (17 -> 8 valid stride 2, 8 -> 8 same stride 1,
8 -> 3 valid stride 2) with small channel counts."""
import numpy as np
import pytest

from oracle import cnn


@pytest.mark.parametrize("B,Ci,D,Co,stride,pad", [(2, 3, 17, 4, 2, 0), (2, 4, 8, 5, 1, 1), (3, 5, 8, 6, 2, 0)])
def test_conv3d_matches_torch(B, Ci, D, Co, stride, pad):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(B * 100 + Ci * 10 + D)
    X = rng.standard_normal((B, Ci, D, D, D))
    W = rng.standard_normal((Co, Ci, 3, 3, 3))
    b = rng.standard_normal(Co)
    Do = cnn.out_size(D, stride, pad)
    Xt = torch.from_numpy(X).requires_grad_(True)
    Wt = torch.from_numpy(W).requires_grad_(True)
    bt = torch.from_numpy(b).requires_grad_(True)
    Yt = torch.nn.functional.conv3d(Xt, Wt, bt, stride=stride, padding=pad)
    Y = cnn.conv3d(X, W, b, stride, pad)
    assert Y.shape == (B, Co, Do, Do, Do) == tuple(Yt.shape)
    assert np.max(np.abs(Y - Yt.detach().numpy())) < 1e-12
    dY = rng.standard_normal(Y.shape)
    Yt.backward(torch.from_numpy(dY))
    dX, dW, db = cnn.conv3d_backward(X, W, dY, stride, pad)
    assert np.max(np.abs(dX - Xt.grad.numpy())) < 1e-11
    assert np.max(np.abs(dW - Wt.grad.numpy())) < 1e-10
    assert np.max(np.abs(db - bt.grad.numpy())) < 1e-11


def test_branch_shapes_give_the_fnn_width():
    """17 -> 8 -> 8 -> 3 with 60 channels: 60 x 3^3 = 1620 inputs of the branch FNN."""
    D = 17
    for stride, pad in ((2, 0), (1, 1), (2, 0)):
        D = cnn.out_size(D, stride, pad)
    assert D == 3 and 60 * D ** 3 == 1620
