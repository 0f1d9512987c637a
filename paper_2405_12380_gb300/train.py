"""DeepONet training on scatterer-free problems (Sec. 3.2, App. B).

The operator learned is the solution operator of Eq. 1 without the scatterer,
f -> u.  Training data come from the library's own solver: forcing terms drawn
from a Gaussian random field (real and imaginary parts independent, RBF kernel,
App. B), solved on a handle whose mask is the outer ring only.  Pairs are
normalised by ||f|| (the correction is applied as s * DeepONet(r / s)).

Network: branch [2N, hidden..., 2p] with ReLU, trunk [d, hidden..., p] with
tanh, output u_l = sum_j b_re,j T_j(x_l) + i sum_j b_im,j T_j(x_l); loss: relative
L2 on a random subset of nodes per step; Adam (App. B: constant learning rate).
Every forward, backward and optimiser step runs in libhelm's kernels (nn_gemm,
nn_bias_act, nn_act_backward, nn_bias_grad, nn_rel_l2, nn_adam, nn_gather);
torch only provides device buffers.  The dense-layer products run in FP32 on the
CUDA cores, or -- set_tensor_cores(True) -- with BF16 operands and FP32
accumulation on the tcgen05 tensor cores (nn_gemm_bf16; master weights, Adam and
the loss stay FP32).
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


_TENSOR_CORES = False


def set_tensor_cores(on: bool):
    """Dense-layer products of training on the tcgen05 tensor cores (BF16 operands,
    FP32 accumulation) instead of the FP32 CUDA-core GEMM."""
    global _TENSOR_CORES
    _TENSOR_CORES = bool(on)


def _gemm(lib, *args):
    return (lib.nn_gemm_bf16 if _TENSOR_CORES else lib.nn_gemm)(*args)


def _ck(st, what):
    if st != 0:
        raise RuntimeError(f"{what}: {L.STATUS_NAMES.get(st, st)}")


@dataclass
class Layer:
    W: torch.Tensor          # out x in, FP32, cuda
    b: torch.Tensor          # out
    mW: torch.Tensor = None
    vW: torch.Tensor = None
    mb: torch.Tensor = None
    vb: torch.Tensor = None
    gW: torch.Tensor = None
    gb: torch.Tensor = None

    def __post_init__(self):
        for name in ("mW", "vW", "gW"):
            setattr(self, name, torch.zeros_like(self.W))
        for name in ("mb", "vb", "gb"):
            setattr(self, name, torch.zeros_like(self.b))


@dataclass
class DeepONet:
    branch: list = field(default_factory=list)
    trunk: list = field(default_factory=list)
    step: int = 0

    @staticmethod
    def init(branch_widths, trunk_widths, seed=0):
        import scenes
        rng = np.random.default_rng(seed)
        mk = lambda ws: [Layer(torch.from_numpy(W.astype(np.float32)).cuda(), torch.from_numpy(b.astype(np.float32)).cuda())
                         for W, b in scenes.glorot_mlp(rng, ws)]
        return DeepONet(mk(branch_widths), mk(trunk_widths))

    def numpy_layers(self, part):
        return [(l.W.cpu().numpy().astype(np.float64), l.b.cpu().numpy().astype(np.float64)) for l in getattr(self, part)]

    def save(self, path):
        d = {"step": self.step}
        for part in ("branch", "trunk"):
            for i, l in enumerate(getattr(self, part)):
                for nm in ("W", "b", "mW", "vW", "mb", "vb"):
                    d[f"{part}{i}_{nm}"] = getattr(l, nm).cpu().numpy()
        np.savez(path, **d)

    @staticmethod
    def load(path):
        z = np.load(path)
        net = DeepONet(step=int(z["step"]))
        for part in ("branch", "trunk"):
            i = 0
            while f"{part}{i}_W" in z:
                l = Layer(torch.from_numpy(z[f"{part}{i}_W"]).cuda(), torch.from_numpy(z[f"{part}{i}_b"]).cuda())
                for nm in ("mW", "vW", "mb", "vb"):
                    getattr(l, nm).copy_(torch.from_numpy(z[f"{part}{i}_{nm}"]))
                getattr(net, part).append(l)
                i += 1
        return net


def _forward_mlp(layers, X, act, stream):
    """Activations [X, H1, ..., out]; act on hidden layers."""
    lib = L.lib()
    acts = [X]
    for i, l in enumerate(layers):
        rows, fin = acts[-1].shape
        H = torch.empty(rows, l.W.shape[0], dtype=torch.float32, device="cuda")
        _ck(_gemm(lib, 0, 1, rows, l.W.shape[0], fin, 1.0, _p(acts[-1]), fin, _p(l.W), fin, 0.0, _p(H),
                        l.W.shape[0], stream), "nn_gemm")
        _ck(lib.nn_bias_act(rows, l.W.shape[0], _p(H), _p(l.b), act if i < len(layers) - 1 else 0, stream),
            "nn_bias_act")
        acts.append(H)
    return acts


def _backward_mlp(layers, acts, dout, act, stream, need_input_grad=False):
    lib = L.lib()
    d = dout
    for i in range(len(layers) - 1, -1, -1):
        l = layers[i]
        rows = d.shape[0]
        fout, fin = l.W.shape
        if i < len(layers) - 1:
            _ck(lib.nn_act_backward(d.numel(), _p(d), _p(acts[i + 1]), act, stream), "nn_act_backward")
        _ck(_gemm(lib, 1, 0, fout, fin, rows, 1.0, _p(d), fout, _p(acts[i]), fin, 0.0, _p(l.gW), fin, stream), "dW")
        _ck(lib.nn_bias_grad(rows, fout, _p(d), _p(l.gb), stream), "db")
        if i > 0 or need_input_grad:
            dn = torch.empty(rows, fin, dtype=torch.float32, device="cuda")
            _ck(_gemm(lib, 0, 0, rows, fin, fout, 1.0, _p(d), fout, _p(l.W), fin, 0.0, _p(dn), fin, stream), "dX")
            d = dn


def train_step(net, X, Xc, Y, lr=1e-4, stream=None):
    """One Adam step on a batch: X (B x 2N) branch inputs, Xc (P x d) trunk inputs,
    Y (B x 2P) targets on the sampled nodes (real parts then imaginary).  Returns
    the per-sample relative-L2 losses (before the step)."""
    lib = L.lib()
    s = stream if stream is not None else C.c_void_p(torch.cuda.current_stream().cuda_stream)
    B, P = X.shape[0], Xc.shape[0]
    ba = _forward_mlp(net.branch, X, 1, s)
    ta = _forward_mlp(net.trunk, Xc, 2, s)
    Bo, T = ba[-1], ta[-1]
    p = T.shape[1]
    pred = torch.empty(B, 2 * P, dtype=torch.float32, device="cuda")
    _ck(_gemm(lib, 0, 1, B, P, p, 1.0, _p(Bo), 2 * p, _p(T), p, 0.0, _p(pred), 2 * P, s), "pred re")
    _ck(_gemm(lib, 0, 1, B, P, p, 1.0, C.c_void_p(Bo.data_ptr() + 4 * p), 2 * p, _p(T), p, 0.0,
                    C.c_void_p(pred.data_ptr() + 4 * P), 2 * P, s), "pred im")
    dpred = torch.empty_like(pred)
    loss = torch.empty(B, dtype=torch.float32, device="cuda")
    _ck(lib.nn_rel_l2(B, 2 * P, _p(pred), _p(Y), _p(dpred), _p(loss), s), "nn_rel_l2")
    dBo = torch.empty_like(Bo)
    _ck(_gemm(lib, 0, 0, B, p, P, 1.0, _p(dpred), 2 * P, _p(T), p, 0.0, _p(dBo), 2 * p, s), "dB re")
    _ck(_gemm(lib, 0, 0, B, p, P, 1.0, C.c_void_p(dpred.data_ptr() + 4 * P), 2 * P, _p(T), p, 0.0,
                    C.c_void_p(dBo.data_ptr() + 4 * p), 2 * p, s), "dB im")
    dT = torch.empty_like(T)
    _ck(_gemm(lib, 1, 0, P, p, B, 1.0, _p(dpred), 2 * P, _p(Bo), 2 * p, 0.0, _p(dT), p, s), "dT re")
    _ck(_gemm(lib, 1, 0, P, p, B, 1.0, C.c_void_p(dpred.data_ptr() + 4 * P), 2 * P,
                    C.c_void_p(Bo.data_ptr() + 4 * p), 2 * p, 1.0, _p(dT), p, s), "dT im")
    _backward_mlp(net.branch, ba, dBo, 1, s)
    _backward_mlp(net.trunk, ta, dT, 2, s)
    net.step += 1
    for l in net.branch + net.trunk:
        _ck(lib.nn_adam(l.W.numel(), _p(l.W), _p(l.gW), _p(l.mW), _p(l.vW), lr, 0.9, 0.999, 1e-8, net.step, s), "adam W")
        _ck(lib.nn_adam(l.b.numel(), _p(l.b), _p(l.gb), _p(l.mb), _p(l.vb), lr, 0.9, 0.999, 1e-8, net.step, s), "adam b")
    return loss


def make_dataset(problem, fs, opts, log=print):
    """Solve the scatterer-free problem for each forcing in fs (S x N complex numpy).
    Returns X (S x 2N) and Y (S x 2N) FP32 device tensors and the scales (c_in,
    c_out): X = c_in [Re f, Im f] / ||f|| (entries of unit RMS) and
    Y = c_out [Re u, Im u] / ||f|| (c_out set from the first samples so that the
    targets have unit RMS).  The network learns Y from X; export_branch() folds
    the two scales back into the first and last branch layers."""
    S, N = fs.shape
    X = torch.empty(S, 2 * N, dtype=torch.float32, device="cuda")
    Y = torch.empty(S, 2 * N, dtype=torch.float32, device="cuda")
    c_in = float(np.sqrt(2.0 * N))
    c_out = None
    t0 = time.time()
    iters = []
    for i in range(S):
        f = torch.from_numpy(fs[i]).cuda()
        u, st = problem.solve(f, None, opts)
        if st["status"] != 0:
            raise RuntimeError(f"training solve {i}: {st['status_name']}")
        iters.append(st["iters"])
        nf = float(np.linalg.norm(fs[i]))
        un = u.cpu().numpy() / nf
        if c_out is None:
            c_out = 1.0 / float(np.sqrt(np.mean(un.real ** 2 + un.imag ** 2) / 2.0))
        X[i].copy_(torch.from_numpy((np.concatenate([fs[i].real, fs[i].imag]) * (c_in / nf)).astype(np.float32)))
        Y[i].copy_(torch.from_numpy((np.concatenate([un.real, un.imag]) * c_out).astype(np.float32)))
    log(f"dataset: {S} solves, mean {np.mean(iters):.0f} iterations, {time.time() - t0:.1f} s; "
        f"scales c_in {c_in:.4g} c_out {c_out:.4g}")
    return X, Y, (c_in, c_out)


def export_branch(net, scales):
    """Branch layers (FP64 numpy) acting on [Re r, Im r]/||r|| and producing
    coefficients of u/||r||: the input scale multiplies the first layer's weights,
    the output scale divides the last layer."""
    c_in, c_out = scales
    layers = net.numpy_layers("branch")
    W0, b0 = layers[0]
    layers[0] = (W0 * c_in, b0)
    Wl, bl = layers[-1]
    layers[-1] = (Wl / c_out, bl / c_out)
    return layers


def train(net, X, Y, coords, fluid_idx, steps, batch=32, nodes=8192, lr=1e-4, seed=0, log=print,
          log_every=100, checkpoint=None):
    """Adam on random batches and random node subsets (fluid nodes only)."""
    lib = L.lib()
    rng = np.random.default_rng(seed)
    S, N2 = X.shape
    N = N2 // 2
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    hist = []
    Xb = torch.empty(batch, N2, dtype=torch.float32, device="cuda")
    Yb = torch.empty(batch, 2 * nodes, dtype=torch.float32, device="cuda")
    t0 = time.time()
    for step in range(steps):
        rows = torch.from_numpy(rng.choice(S, batch, replace=False).astype(np.int32)).cuda()
        nid = rng.choice(fluid_idx, nodes, replace=False).astype(np.int32)
        cols = torch.from_numpy(np.concatenate([nid, nid + N]).astype(np.int32)).cuda()
        Xc = torch.from_numpy(coords[nid].astype(np.float32)).cuda()
        _ck(lib.nn_gather(batch, N2, _p(X), N2, _p(rows), None, _p(Xb), s), "gather X")
        _ck(lib.nn_gather(batch, 2 * nodes, _p(Y), N2, _p(rows), _p(cols), _p(Yb), s), "gather Y")
        loss = train_step(net, Xb, Xc, Yb, lr=lr, stream=s)
        if step % log_every == 0 or step == steps - 1:
            l = float(loss.cpu().numpy().mean())
            hist.append((step, l))
            log(f"step {step:6d} rel-L2^2 {l:.4e} ({time.time() - t0:.1f} s)")
        if checkpoint and (step + 1) % 1000 == 0:
            net.save(checkpoint)
    return hist


def evaluate(net, X, Y, coords, rows):
    """Mean relative L2 error (not squared) of the DeepONet on the given samples, all nodes."""
    lib = L.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    N = X.shape[1] // 2
    Xc = torch.from_numpy(coords.astype(np.float32)).cuda()
    ta = _forward_mlp(net.trunk, Xc, 2, s)
    T = ta[-1]
    p = T.shape[1]
    errs = []
    for r in rows:
        ba = _forward_mlp(net.branch, X[r:r + 1], 1, s)
        Bo = ba[-1]
        pred = torch.empty(1, 2 * N, dtype=torch.float32, device="cuda")
        _ck(_gemm(lib, 0, 1, 1, N, p, 1.0, _p(Bo), 2 * p, _p(T), p, 0.0, _p(pred), 2 * N, s), "pred re")
        _ck(_gemm(lib, 0, 1, 1, N, p, 1.0, C.c_void_p(Bo.data_ptr() + 4 * p), 2 * p, _p(T), p, 0.0,
                        C.c_void_p(pred.data_ptr() + 4 * N), 2 * N, s), "pred im")
        d = torch.empty_like(pred)
        lo = torch.empty(1, dtype=torch.float32, device="cuda")
        _ck(lib.nn_rel_l2(1, 2 * N, _p(pred), _p(Y[r:r + 1]), _p(d), _p(lo), s), "rel_l2")
        errs.append(math.sqrt(float(lo.cpu().numpy()[0])))
    return float(np.mean(errs))


def train_workload(name, samples=1024, steps=10000, batch=32, nodes=16384, lr=1e-4, seed=0, solve_tol=1e-3,
                   out=None, log=print):
    """Train the DeepONet of a workload on its scatterer-free problem (same grid,
    wavenumber and layer; mask = outer ring) and save the weights."""
    import os
    import scenes
    from . import helm as hm
    w = scenes.BENCH_WORKLOADS[name]
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    mask = scenes.ring_mask(sc.dim, sc.n).reshape(-1).astype(np.uint8)
    P = hm.Problem(sc.dim, sc.n, sc.k0, mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    rng = np.random.default_rng(seed + 1000)
    t0 = time.time()
    fs = scenes.grf_samples(rng, sc.dim, sc.n, samples)
    fs[:, mask == 1] = 0
    log(f"GRF samples: {samples} in {time.time() - t0:.1f} s")
    X, Y, scales = make_dataset(P, fs, hm.opts("bicgstab", "rbgs", 3, correction="none", tol=solve_tol, maxit=20000),
                                log=log)
    N = sc.N
    trunk_widths = [sc.dim] + [W.shape[0] for W, _ in sc.trunk]
    net = DeepONet.init([2 * N, 256, 256, 2 * sc.p], trunk_widths, seed=seed)
    coords = scenes.node_coords(sc.dim, sc.n)
    fluid = np.flatnonzero(mask == 0)
    n_train = int(samples * 0.9)
    t0 = time.time()
    hist = train(net, X[:n_train], Y[:n_train], coords, fluid, steps, batch=batch, nodes=min(nodes, fluid.size),
                 lr=lr, seed=seed, log=log, log_every=max(1, steps // 20))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    held = evaluate(net, X, Y, coords, range(n_train, samples))
    seen = evaluate(net, X, Y, coords, range(0, min(32, n_train)))
    log(f"training {steps} steps in {t_train:.1f} s; relative L2: held-out {held:.3f}, training {seen:.3f}")
    info = {"samples": samples, "steps": steps, "batch": batch, "nodes": nodes, "lr": lr, "train_s": t_train,
            "held_out_rel_l2": held, "train_rel_l2": seen, "loss_history": hist, "scales": scales,
            "solve_tol": solve_tol}
    if out:
        os.makedirs(os.path.dirname(out) or ".", exist_ok=True)
        tr = net.numpy_layers("trunk")
        np.savez(out + "_trunk.npz", **{f"W{i}": W for i, (W, _) in enumerate(tr)},
                 **{f"b{i}": b for i, (_, b) in enumerate(tr)}, info=json_dump(info))
    return net, info


def json_dump(d):
    import json
    return np.array(json.dumps(d))


def load_trunk(path):
    """[(W, b)] FP64 trunk layers from a file written by train_workload."""
    z = np.load(path)
    layers = []
    i = 0
    while f"W{i}" in z:
        layers.append((z[f"W{i}"].astype(np.float64), z[f"b{i}"].astype(np.float64)))
        i += 1
    return layers


if __name__ == "__main__":
    import argparse
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube3d-64")
    ap.add_argument("--samples", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--nodes", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--out", default=None)
    ap.add_argument("--full", default=None, help="also save the full network and Adam state (.npz)")
    ap.add_argument("--tensor-cores", action="store_true", help="BF16 dense-layer products on tcgen05")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    set_tensor_cores(a.tensor_cores)
    net, info = train_workload(a.workload, a.samples, a.steps, a.batch, a.nodes, a.lr, out=a.out)
    if a.full:
        net.save(a.full)
