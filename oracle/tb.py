"""Trunk-basis (TB) coarse correction and the hybrid cycle (App. C, Eq. 3).

App. C: evaluate the trunk network at the nodes, T_ij = T_j(x_i) (Eq. 6); pick
columns in natural order to form P; orthonormalise P by QR and use Q;
restriction R = P* (= Q^T, Q being real); coarse operator A_c = R A P; the
correction is M2 = P A_c^-1 R, which is linear and so may precondition Krylov
methods.  Rows of T on Dirichlet nodes are set to zero, so M2 never writes a
Dirichlet node (App. D: the residual vanishes there).

Eq. 3 (hybrid iteration): n_r relaxation steps (M1), then one M2 step on the
new residual.  As a preconditioner z = M(r) this is: z = n_r sweeps on A z = r
from z = 0, then z += M2(r - A z).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import relax


LEAKY_SLOPE = 0.01   # Leaky ReLU slope (the paper names the function only; PyTorch's default)


def leaky_relu(a):
    """Leaky ReLU, the trunk's activation in App. B: a for a > 0, LEAKY_SLOPE * a else."""
    return np.where(a > 0, a, LEAKY_SLOPE * a)


def mlp_forward(layers, X, act=np.tanh):
    """Fully connected net: act on hidden layers, linear output (App. B)."""
    a = np.asarray(X, dtype=np.float64)
    for li, (W, b) in enumerate(layers):
        a = a @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        if li < len(layers) - 1:
            a = act(a)
    return a


@dataclass
class TBSetup:
    Q: np.ndarray          # (N, k) real, orthonormal columns, zero rows on M
    Ac: np.ndarray         # (k, k) complex, Q^T A Q
    lu: tuple              # scipy lu_factor of Ac
    kept: list | None = None   # trunk columns selected (natural order)

    @property
    def p(self) -> int:
        return self.Q.shape[1]


def trunk_matrix(layers, coords, mask, p: int, act=np.tanh) -> np.ndarray:
    """T with natural-order first p columns and zeroed Dirichlet rows."""
    T = mlp_forward(layers, coords, act)[:, :p].copy()
    T[np.asarray(mask).reshape(-1) == 1, :] = 0.0
    return T


def natural_order_select(T, tau: float, kmax: int | None = None):
    """Natural-order column selection with orthonormalisation (App. C).

    Columns are visited in natural order; column j is kept when the part of it
    orthogonal to the columns kept so far (classical Gram-Schmidt applied twice)
    has norm > tau * ||T_j||.  Kept columns are normalised.  tau = 0 keeps every
    nonzero column (plain QR in natural order); tau > 0 drops columns that are
    numerically dependent on earlier ones, which keeps span(Q) well determined
    when the trunk's columns are nearly collinear.  Returns (Q, kept)."""
    N, p = T.shape
    kmax = p if kmax is None else kmax
    Qbuf = np.zeros((N, min(p, kmax)))
    kept = []
    for j in range(p):
        t = T[:, j]
        tn = np.linalg.norm(t)
        if tn == 0.0:
            continue
        u = t.copy()
        if kept:
            Qk = Qbuf[:, : len(kept)]
            u = u - Qk @ (Qk.T @ u)
            u = u - Qk @ (Qk.T @ u)
        un = np.linalg.norm(u)
        if un > tau * tn:
            Qbuf[:, len(kept)] = u / un
            kept.append(j)
            if len(kept) == kmax:
                break
    return Qbuf[:, : len(kept)].copy(), kept


def bf16_round(Q):
    """Round FP64 values to the nearest BF16 value (ties to even), through FP32
    first (the rounding the mixed-precision basis uses).  BF16 keeps the top 16
    bits of an FP32 number."""
    x = np.asarray(Q, dtype=np.float64).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return rounded.view(np.float32).astype(np.float64)


def tb_setup(A, layers, coords, mask, p: int, Q=None, tau: float = 0.0, act=np.tanh) -> TBSetup:
    """P = natural-order selection of the first p trunk columns (drop tolerance
    tau), Q orthonormal with span(Q) = span(P), A_c = Q^T A Q, LU with partial
    pivoting.  A caller may pass its own orthonormal Q (e.g. a rounded copy).
    act: the trunk's hidden-layer activation (tanh, or leaky_relu as in App. B)."""
    kept = None
    if Q is None:
        T = trunk_matrix(layers, coords, mask, p, act)
        if tau > 0:
            Q, kept = natural_order_select(T, tau)
        else:
            fluid = np.asarray(mask).reshape(-1) == 0
            Q = np.zeros_like(T)
            Q[fluid], _ = np.linalg.qr(T[fluid])   # masked rows of T are zero: keep them exactly zero
            kept = list(range(p))
    Ac = Q.T @ (A @ Q)
    return TBSetup(Q=Q, Ac=Ac, lu=sla.lu_factor(Ac), kept=kept)


def tb_correct(s: TBSetup, r):
    """M2 r = Q A_c^-1 Q^T r.  Q is real, so Q^T r = Q^T Re r + i Q^T Im r and
    Q y = Q Re y + i Q Im y: both products are taken on the two real columns."""
    c = s.Q.T @ np.stack([r.real, r.imag], axis=1)
    y = sla.lu_solve(s.lu, c[:, 0] + 1j * c[:, 1])
    z = s.Q @ np.stack([y.real, y.imag], axis=1)
    return z[:, 0] + 1j * z[:, 1]


def mixed_setup(s: TBSetup, A) -> TBSetup:
    """Mixed precision: the basis is rounded to BF16 and the coarse operator is
    rebuilt from the same rounded basis, A_c = Qr^T A Qr, so that the Galerkin
    property holds for the basis actually used."""
    Qr = bf16_round(s.Q)
    Ac = Qr.T @ (A @ Qr)
    return TBSetup(Q=Qr, Ac=Ac, lu=sla.lu_factor(Ac), kept=s.kept)


def hybrid_preconditioner(A, s: "TBSetup | None", kind: str, n_r: int, omega: float = 0.6,
                          colours=None):
    """z = M(r): n_r relaxation sweeps from zero, then the TB correction.
    With neither sweeps nor a correction M is the identity (plain Krylov)."""
    if (kind == "none" or n_r <= 0) and s is None:
        return lambda r: np.array(r, dtype=np.complex128, copy=True)

    def M(r):
        z = np.zeros_like(r, dtype=np.complex128)
        if kind == "jacobi" and n_r > 0:
            z = relax.jacobi(A, r, z, omega, n_r)
        elif kind == "rbgs" and n_r > 0:
            z = relax.rbgs(A, r, z, colours, n_r)
        elif kind not in ("none", "jacobi", "rbgs"):
            raise ValueError(kind)
        if s is not None:
            z = z + tb_correct(s, r - A @ z)
        return z
    return M
