"""3D convolution layers of the DeepONet's CNN branch (App. B), NumPy FP64.

App. B: the branch of the 3D DeepONet is a CNN on a 17 x 17 x 17 input with channels
[3, 40, 40, 60] (the wave number and the real and imaginary parts of the forcing),
3 x 3 x 3 kernels, valid padding except one layer with same padding, ReLU, then a
fully connected net from 1620 = 60 x 3^3 inputs.  Reading of the garbled strides:
17 -> 8 (valid, stride 2), 8 -> 8 (same, stride 1), 8 -> 3 (valid, stride 2), which is
the only assignment that gives the 60 x 3^3 = 1620 inputs of the FNN.

Layout [batch][channel][z][y][x]; kernel W[out][in][kz][ky][kx]; output size
Do = (D + 2 pad - 3) // stride + 1.  The convolution is the cross-correlation of
deep-learning practice:
    Y[b, o, z, y, x] = bias[o] + sum_{i, kz, ky, kx} W[o, i, kz, ky, kx]
                       X[b, i, z s + kz - pad, y s + ky - pad, x s + kx - pad]
with zeros outside the input.  TEST INFRASTRUCTURE ONLY (the GPU kernels are checked
against it); it shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

K = 3


def out_size(D: int, stride: int, pad: int) -> int:
    return (D + 2 * pad - K) // stride + 1


def _padded(X, pad):
    if pad == 0:
        return X
    return np.pad(X, ((0, 0), (0, 0), (pad, pad), (pad, pad), (pad, pad)))


def conv3d(X, W, bias, stride: int, pad: int):
    """Forward: the sum above, one kernel offset at a time (a strided slice of the
    padded input times the offset's Co x Ci weights)."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    B, Ci, D = X.shape[0], X.shape[1], X.shape[2]
    Co = W.shape[0]
    Do = out_size(D, stride, pad)
    Xp = _padded(X, pad)
    Y = np.zeros((B, Co, Do, Do, Do))
    span = stride * (Do - 1) + 1
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                patch = Xp[:, :, kz:kz + span:stride, ky:ky + span:stride, kx:kx + span:stride]
                Y += np.einsum("oi,bizyx->bozyx", W[:, :, kz, ky, kx], patch)
    return Y + np.asarray(bias, np.float64)[None, :, None, None, None]


def conv3d_backward(X, W, dY, stride: int, pad: int):
    """Gradients (dX, dW, db) of sum(dY * conv3d(X, W, b)) -- the adjoints of the
    offset-by-offset sum: dW[o, i, k] = sum over b and outputs of dY X at the offset,
    dX scatters dY W back to the input positions each offset read."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    dY = np.asarray(dY, np.float64)
    B, Ci, D = X.shape[0], X.shape[1], X.shape[2]
    Do = dY.shape[2]
    Xp = _padded(X, pad)
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(W)
    span = stride * (Do - 1) + 1
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                sl = (slice(None), slice(None), slice(kz, kz + span, stride), slice(ky, ky + span, stride),
                      slice(kx, kx + span, stride))
                dW[:, :, kz, ky, kx] = np.einsum("bozyx,bizyx->oi", dY, Xp[sl])
                dXp[sl] += np.einsum("oi,bozyx->bizyx", W[:, :, kz, ky, kx], dY)
    dX = dXp[:, :, pad:pad + D, pad:pad + D, pad:pad + D] if pad else dXp
    return dX, dW, dY.sum(axis=(0, 2, 3, 4))
