"""Algorithm 4 (randomized SVD of an implicit operator), oracle side.

Step order, with A given only through A X and A^H Y (Sec. IV-A):
  Omega <- random N x l block (Algorithm 4, first line; see philox.sketch)
  P <- orth(A Omega)
  repeat q times:  Q <- orth(A^H P);  P <- orth(A Q)
  B <- P^H A  (formed as (A^H P)^H);  U~, Sigma, V^H <- SVD(B)
  U <- P U~
"orthogonalize" is Householder QR (LAPACK, through torch.linalg); when the
block is numerically rank deficient (|R_ii| <= rtol max|R_ii|) the
orthonormal basis of its range comes from an SVD instead, padded with zero
columns, which is the role of
the Gram eigen-route of Algorithm 5 for a rank-deficient input.

Readings of points the paper leaves open (all shared with the GPU path):
  * rank k = min(m, M, N); block width l = min(k + p, M, N) (oversampling p);
  * singular values <= rtol * sigma_1 count as zero: their U columns and W
    rows are set to zero so the bond keeps its static size k;
  * gauge: each left singular vector u_c is multiplied by the conjugate phase
    of <g, u_c> (g a fixed Philox vector, tag 1) and the matching W row by the
    phase, so <g, u_c> is real and non-negative (a sign in the real case);
  * Sigma is absorbed into the right factor, W = Sigma V^H, then W is divided
    by sigma_1 and log(sigma_1) is returned (the scale is carried as a log).
"""
from __future__ import annotations

import numpy as np
import torch

from . import philox
from .implicit import ImplicitOp


def default_rtol(ell: int) -> float:
    """Relative threshold below which a direction counts as numerically zero."""
    return 16.0 * max(ell, 1) * np.finfo(np.float64).eps


def orthogonalize(Y: np.ndarray, rtol: float) -> np.ndarray:
    """Orthonormal basis of range(Y) with the same column count."""
    if Y.shape[1] == 0:
        return Y.copy()
    Qt, Rt = torch.linalg.qr(torch.from_numpy(np.ascontiguousarray(Y)))
    Q, R = Qt.numpy(), Rt.numpy()
    dg = np.abs(np.diag(R))
    big = dg.max() if dg.size else 0.0
    if big == 0.0:
        return np.zeros_like(Y)
    if np.all(dg > rtol * big):
        return Q
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    keep = s > rtol * s[0]
    out = np.zeros_like(Y)
    out[:, : int(keep.sum())] = U[:, keep]
    return out


def fix_gauge(U: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Make <g, u_c> real and non-negative for every column c of U."""
    phi = g.conj() @ U
    mag = np.abs(phi)
    if np.iscomplexobj(U) or np.iscomplexobj(phi):
        rho = np.where(mag > 0, phi / np.where(mag > 0, mag, 1.0), 1.0)
        return U * np.conj(rho)[None, :], W * rho[:, None]
    rho = np.where(phi < 0, -1.0, 1.0)
    return U * rho[None, :], W * rho[:, None]


def rsvd_implicit(op: ImplicitOp, k: int, ell: int, q: int, omega: np.ndarray,
                  rtol: float):
    """Algorithm 4 on the implicit operator; returns (P, U~, sigma, V^H)."""
    P = orthogonalize(op.matvec(omega), rtol)
    for _ in range(q):
        Q = orthogonalize(op.rmatvec(P), rtol)
        P = orthogonalize(op.matvec(Q), rtol)
    Z = op.rmatvec(P)                  # (P^H A)^H
    B = torch.from_numpy(np.ascontiguousarray(Z)).mH
    Ut, s, Vh = (x.resolve_conj().numpy() for x in torch.linalg.svd(B, full_matrices=False))
    return P, Ut[:, :k], s[:k], Vh[:k]


def block_sizes(m: int, p: int, M: int, N: int):
    k = min(m, M, N)
    ell = min(k + p, M, N)
    return k, ell


def einsumsvd(V, S, K, Kb, m: int, p: int, q: int, seed: int, instance: int,
              sketch_kind: str = "gauss", rtol: float | None = None,
              return_all: bool = False, absorb: str = "right"):
    """One zip-up einsumsvd step (Algorithm 3) with Algorithm 4 inside.

    Returns U [kL][t][k] (new boundary site), W [k][x X][b][e E] (new carry,
    divided by sigma_1), sigma (k values, unnormalised) and log(sigma_1).
    absorb="right" puts Sigma into the carry (W = Sigma V^H / sigma_1, U with
    orthonormal columns); absorb="left" into the finished site (U = U~ Sigma /
    sigma_1, W = V^H with orthonormal rows), the other canonical choice of
    Sec. III-A's zip-up.
    """
    op = ImplicitOp(V, S, K, Kb)
    is_c = op.is_complex
    k, ell = block_sizes(m, p, op.M, op.N)
    if rtol is None:
        rtol = default_rtol(ell)
    omega = philox.sketch(op.N, ell, seed, instance, is_c, sketch_kind)
    P, Ut, s, Vh = rsvd_implicit(op, k, ell, q, omega, rtol)
    zero = s <= rtol * (s[0] if s.size else 0.0)
    U = P @ Ut
    W = s[:, None] * Vh
    U[:, zero] = 0
    W[zero, :] = 0
    s = np.where(zero, 0.0, s)
    g = philox.gauge_vector(op.M, seed, instance, is_c)
    U, W = fix_gauge(U, W, g)
    s1 = s[0] if s.size else 0.0
    logs1 = float(np.log(s1)) if s1 > 0 else float("-inf")
    if absorb == "left":
        # W rows back to V^H (zero rows stay zero), Sigma / sigma_1 into U
        inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        W = W * inv[:, None]
        if s1 > 0:
            U = U * (s / s1)[None, :]
    elif s1 > 0:
        W = W / s1
    kL, t = op.dims["kL"], op.dims["t"]
    Dx, DX, b, De, DE = op.col_shape
    U = U.reshape(kL, t, k)
    W = W.reshape(k, Dx * DX, b, De * DE)
    if return_all:
        return U, W, s, logs1, dict(op=op, k=k, ell=ell, P=P, omega=omega)
    return U, W, s, logs1
