"""Outer loops of the meta-solvers (Sec. 3.1): FGMRES(m), BiCGStab and the
relaxation meta-solver (hybrid Richardson, Eq. 3).

* FGMRES(m) (Saad, flexible GMRES) with right preconditioning: Arnoldi on A M,
  the preconditioned vectors z_j are stored; classical Gram-Schmidt applied twice
  (CGS2) for orthogonalisation; complex Givens rotations
  [c, s; -conj(s), c] with real c; x += Z y at the end of a cycle; the true
  residual is recomputed at every restart and decides convergence.
* BiCGStab (van der Vorst) with right preconditioning, shadow vector r0.
  <a, b> = a^H b.  When the recursive residual meets the tolerance the true
  residual is computed; if it does not meet it the method restarts from x.
* relaxation meta-solver: per cycle n_r relaxation sweeps on A u = f, then one
  correction M2 on the new residual, convergence checked on ||f - A u||/||f||
  before every cycle.

Every routine returns (x, info) with info = {"iters", "res" (list of relative
residual norms), "status"}.  Iteration counting: one Arnoldi step, one full
BiCGStab iteration, one relaxation cycle.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import relax


def givens(a: complex, b: complex):
    """(c, s, r) with [c s; -conj(s) c] [a; b] = [r; 0], c real >= 0."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b)
    t = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    ph = a / abs(a)
    return abs(a) / t, ph * np.conj(b) / t, ph * t


def fgmres(A, b, x0, M=None, tol=1e-8, m=30, maxit=1000, max_cycles=None, keep_first=False):
    """`keep_first` also returns the first cycle's V, Z and unrotated H in info."""
    M = M or (lambda v: v.copy())
    bnorm = np.linalg.norm(b)
    x = np.array(x0, dtype=np.complex128, copy=True)
    hist, est, iters, cycles, status = [], [], 0, 0, "maxit"
    first = None
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            status = "converged"
            break
        if iters >= maxit or (max_cycles is not None and cycles >= max_cycles):
            break
        cycles += 1
        V = np.zeros((m + 1, b.size), dtype=np.complex128)
        Z = np.zeros((m, b.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A @ Z[j]
            h = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if keep_first and cycles == 1:
                if first is None:
                    first = {"V": V, "Z": Z, "H": np.zeros((m + 1, m), dtype=np.complex128)}
                first["H"][: j + 2, j] = H[: j + 2, j]
            for i in range(j):
                a_, b_ = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a_ + sn[i] * b_
                H[i + 1, j] = -np.conj(sn[i]) * a_ + cs[i] * b_
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            est.append(abs(g[j + 1]) / bnorm)
            if hn != 0.0:
                V[j + 1] = w / hn
            if hn == 0.0 or abs(g[j + 1]) <= tol * bnorm or iters >= maxit:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + Z[:k].T @ y
        if first is not None and "k" not in first:
            first["k"] = k
    info = {"iters": iters, "res": hist, "est": est, "status": status, "cycles": cycles}
    if keep_first:
        info["first"] = first
    return x, info


def bicgstab(A, b, x0, M=None, tol=1e-8, maxit=1000):
    M = M or (lambda v: v.copy())
    vdot = np.vdot
    bnorm = np.linalg.norm(b)
    x = np.array(x0, dtype=np.complex128, copy=True)
    r = b - A @ x
    hist = [np.linalg.norm(r) / bnorm]
    if hist[-1] <= tol:
        return x, {"iters": 0, "res": hist, "status": "converged"}
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(r)
    p = np.zeros_like(r)
    iters, status = 0, "maxit"
    while iters < maxit:
        rho = vdot(rhat, r)
        if rho == 0:
            status = "breakdown"
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = M(p)
        v = A @ phat
        alpha = rho / vdot(rhat, v)
        s = r - alpha * v
        iters += 1
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * phat
            r = s
        else:
            shat = M(s)
            t = A @ shat
            tt = vdot(t, t)
            if tt == 0:
                status = "breakdown"
                break
            omega = vdot(t, s) / tt
            x = x + alpha * phat + omega * shat
            r = s - omega * t
            rho_old = rho
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= tol:
            rt = b - A @ x
            if np.linalg.norm(rt) <= tol * bnorm:
                hist[-1] = np.linalg.norm(rt) / bnorm
                status = "converged"
                break
            r = rt                                   # restart from the current iterate
            rhat = r.copy()
            rho_old = alpha = omega = 1.0 + 0.0j
            v = np.zeros_like(r)
            p = np.zeros_like(r)
        if omega == 0:
            status = "breakdown"
            break
    return x, {"iters": iters, "res": hist, "status": status}


def relaxation_metasolver(A, b, x0, kind: str, n_r: int, correction=None, omega: float = 0.6,
                          colours=None, tol=1e-8, max_cycles=1000):
    """Hybrid Richardson (Eq. 3): per cycle n_r sweeps, then u += M2(f - A u)."""
    bnorm = np.linalg.norm(b)
    x = np.array(x0, dtype=np.complex128, copy=True)
    hist, cycles, status = [], 0, "maxit"
    while True:
        res = np.linalg.norm(b - A @ x) / bnorm
        hist.append(res)
        if res <= tol:
            status = "converged"
            break
        if not np.isfinite(res) or res > 1e8:
            status = "diverged"
            break
        if cycles >= max_cycles:
            break
        if kind == "jacobi":
            x = relax.jacobi(A, b, x, omega, n_r)
        elif kind == "rbgs":
            x = relax.rbgs(A, b, x, colours, n_r)
        if correction is not None:
            x = x + correction(b - A @ x)
        cycles += 1
    return x, {"iters": cycles, "res": hist, "status": status}
