"""DeepONet forward/backward, relative-L2 loss and Adam in NumPy FP64 (App. B).

Branch: fully connected, ReLU on hidden layers, input [Re f, Im f] (2N), output
2p coefficients split into a real and an imaginary group.  Trunk: fully
connected, tanh on hidden layers, input node coordinates, output p basis values.
DeepONet output at node x_l: u_l = sum_j b_re,j T_j(x_l) + i sum_j b_im,j T_j(x_l).
Loss: mean over the batch of ||u_pred - u||^2 / ||u||^2 on the sampled nodes.
Adam: Kingma & Ba with bias correction.
"""
from __future__ import annotations

import numpy as np


def mlp_forward_all(layers, X, act):
    """Returns the list of activations [X, H1, ..., out] (act on hidden layers)."""
    acts = [np.asarray(X, dtype=np.float64)]
    for li, (W, b) in enumerate(layers):
        H = acts[-1] @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if li < len(layers) - 1:
            H = act(H)
        acts.append(H)
    return acts


def relu(x):
    return np.maximum(x, 0.0)


LEAKY_SLOPE = 0.01   # Leaky ReLU slope of the trunk (App. B; PyTorch's default)


def leaky_relu(x):
    return np.where(x > 0, x, LEAKY_SLOPE * x)


def leaky_relu_deriv(H):
    """Derivative from the activation output (same sign as its input)."""
    return np.where(H > 0, 1.0, LEAKY_SLOPE)


def mlp_backward(layers, acts, dout, act_deriv):
    """Gradients (dW, db) per layer given d(loss)/d(output); act_deriv(H) = act'(pre) from the output H."""
    grads = [None] * len(layers)
    d = dout
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li < len(layers) - 1:
            d = d * act_deriv(acts[li + 1])
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        d = d @ np.asarray(W, np.float64)
    return grads


def deeponet_forward(branch, trunk, X, Xc):
    """pred (B x 2P): real parts then imaginary parts on the sampled nodes."""
    ba = mlp_forward_all(branch, X, relu)
    ta = mlp_forward_all(trunk, Xc, np.tanh)
    Bo, T = ba[-1], ta[-1]
    p = T.shape[1]
    pred = np.concatenate([Bo[:, :p] @ T.T, Bo[:, p:] @ T.T], axis=1)
    return pred, ba, ta


def rel_l2(pred, target):
    num = ((pred - target) ** 2).sum(axis=1)
    den = (target ** 2).sum(axis=1)
    loss = num / den
    dpred = 2.0 * (pred - target) / (den[:, None] * pred.shape[0])
    return loss, dpred


def deeponet_backward(branch, trunk, ba, ta, dpred):
    Bo, T = ba[-1], ta[-1]
    p = T.shape[1]
    P = T.shape[0]
    dre, dim = dpred[:, :P], dpred[:, P:]
    dBo = np.concatenate([dre @ T, dim @ T], axis=1)
    dT = dre.T @ Bo[:, :p] + dim.T @ Bo[:, p:]
    gb = mlp_backward(branch, ba, dBo, lambda H: (H > 0).astype(np.float64))
    gt = mlp_backward(trunk, ta, dT, lambda H: 1.0 - H * H)
    return gb, gt


def adam_step(p, g, m, v, t, lr=1e-4, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v


def nonlinear_correction(branch, Traw, r):
    """M2(r) = s (T b_re + i T b_im), b = Branch([Re r, Im r] / s), s = ||r|| (positively homogeneous)."""
    s = np.linalg.norm(r)
    if s == 0:
        return np.zeros_like(r)
    x = np.concatenate([r.real, r.imag])[None, :] / s
    b = mlp_forward_all(branch, x, relu)[-1][0]
    p = Traw.shape[1]
    return s * (Traw @ b[:p] + 1j * (Traw @ b[p:]))
