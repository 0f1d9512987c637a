"""Differentiable solves: torch.autograd.Function wrappers over the C ABI.

HelmSolve.apply(k2, f, problem, opts) -> u solves A(k2) u = f with the
meta-solver of `opts`; its backward is the adjoint solve conj(A) lambda = G with
the same meta-solver (conj = 1, conjugated hybrid cycle), G being the incoming
gradient dL/dRe u + i dL/dIm u (PyTorch's convention for complex tensors), and
returns dL/dk2 = -lambda conj(u) on fluid nodes (0 on Dirichlet nodes) and
dL/df = lambda.  ReceiverSample.apply(u, problem, idx, w) samples u at
receivers by trilinear interpolation; its backward scatters with S^T.

Only the converged u is kept for the backward pass (the continuous-adjoint
gradient needs nothing else).  Every operation runs in libhelm's kernels.
"""
from __future__ import annotations

import torch


class HelmSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k2, f, problem, o):
        problem.set_k2(k2.detach())
        u, st = problem.solve(f.detach().contiguous(), None, o)
        if st["status"] != 0:
            raise RuntimeError(f"forward solve: {st['status_name']} after {st['iters']} iterations")
        ctx.problem, ctx.o = problem, o
        ctx.forward_stats = st
        ctx.save_for_backward(k2.detach(), u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        k2, u = ctx.saved_tensors
        P = ctx.problem
        P.set_k2(k2)
        o = ctx.o
        oa = type(o)(o.method, o.relax, o.n_r, o.omega, o.correction, o.tol, o.restart, o.maxit,
                     1 - int(o.conj))
        lam, st = P.solve(grad_u.contiguous(), None, oa)
        if st["status"] != 0:
            raise RuntimeError(f"adjoint solve: {st['status_name']} after {st['iters']} iterations")
        g = P.k2_gradient(lam, u)
        return g, lam, None, None


class ReceiverSample(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, problem, idx, w):
        ctx.problem, ctx.idx, ctx.w = problem, idx, w
        return problem.sample(idx, w, u.detach())

    @staticmethod
    def backward(ctx, grad_out):
        return ctx.problem.sample_adjoint(ctx.idx, ctx.w, grad_out.contiguous()), None, None, None


def misfit_loss(k2, f, problem, o, idx, w, d):
    """L = sum_r |u(x_r) - d_r|^2 with u = A(k2)^-1 f."""
    u = HelmSolve.apply(k2, f, problem, o)
    e = ReceiverSample.apply(u, problem, idx, w) - d
    return (e.real ** 2 + e.imag ** 2).sum(), u
