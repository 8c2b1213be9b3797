"""Operator application by QR-SVD (Algorithm 1) and one TEBD layer (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A two-site operator G (Eq. 5, G[i1 i2, j1 j2]: outgoing physical pair
(i1, i2), incoming (j1, j2)) acts on neighbouring sites M1 = M^(p,q) and
M2 = M^(p,q+1) (horizontal bond: M1's right bond is M2's left bond) or
M^(p+1,q) (vertical bond: M1's down bond is M2's up bond).  Sites are
[d][left][up][down][right].  Algorithm 1:

  Q1, R1 <- QR(M1)    M1 as a matrix [(the three outer bonds), (s, shared)]
  Q2, R2 <- QR(M2)    M2 likewise
  R1~, R2~ <- einsumsvd(G, R1, R2)
  M1~ <- Q1 R1~,  M2~ <- Q2 R2~

The einsumsvd contracts Theta[(r1, i1), (r2, i2)] = sum_{j1, j2, b}
G[i1 i2, j1 j2] R1[r1, (j1, b)] R2[r2, (j2, b)] and truncates it to rank
k = min(D_max, rows, columns).  Theta is small (d times the QR rank on each
side), so its SVD is a dense LAPACK SVD (the randomized SVD of Algorithm 4
would return the same factors up to its approximation error).

Readings of points the paper leaves open (all shared with the GPU path):
  * QR is Householder QR; the R factor has min(outer, d * shared) rows, and
    an R row whose diagonal is numerically zero (the oracle's rank rule,
    16 n eps |R|) is kept as a zero row;
  * Sigma is split evenly: R1~ = U sqrt(Sigma), R2~ = sqrt(Sigma) V^H;
    directions with sigma <= 16 n eps sigma_1 are returned as zeros, so the
    new bond always has k = D_max entries when D_max <= the rank bound, or
    the full rank bound otherwise (static shapes);
  * phases: column c of the updated first site, as a matrix
    [(outer bonds, s)][c], is multiplied by the conjugate phase of its inner
    product with g (the Philox gauge vector of the bond's stream, tag 1, one
    entry per row) and the second site's column c by that phase, so the
    choice does not depend on the orthonormal basis the QR picks;
  * a site with no more outer entries than d * shared is not factorised
    (Q = identity, R = the site itself); the result is the same for any
    orthonormal Q;
  * the stream of the bond between sites a and b (row-major indices) is
    (4 << 32) | (a << 16) | b;
  * a TEBD layer applies G to every horizontal bond (columns 0-1, 2-3, ...,
    then 1-2, 3-4, ...), then to every vertical bond (rows 0-1, 2-3, ...,
    then 1-2, ...): the bonds of one pass share no site;
  * a layer may carry one operator per bond, listed in bond order (every
    horizontal bond by its left site in row-major order, then every
    vertical bond by its upper site in row-major order), and one-site
    operators (Eq. 4), applied to every site before the bonds;
  * for imaginary-time evolution the new bond may be normalised: Sigma is
    divided by sigma_1 before the split (R1~ = U sqrt(Sigma / sigma_1),
    R2~ = sqrt(Sigma / sigma_1) V^H), so each bond update applies G up to
    one positive factor and the state's scale stays bounded over many
    layers.
"""
from __future__ import annotations

import numpy as np

from . import philox

TEBD_DIRECTION = 4


def bond_stream(a: int, b: int) -> int:
    return (TEBD_DIRECTION << 32) | (a << 16) | b


def _qr(Mmat: np.ndarray):
    """Householder QR with the zero-row rule for the R factor."""
    Q, R = np.linalg.qr(Mmat)
    dg = np.abs(np.diag(R))
    big = dg.max() if dg.size else 0.0
    tol = 16.0 * max(R.shape) * np.finfo(np.float64).eps * big
    dead = dg <= tol
    Q = Q.copy()
    R = R.copy()
    Q[:, dead] = 0
    R[dead, :] = 0
    return Q, R


def _svd_truncate(Theta: np.ndarray, kmax: int, unit: bool = False):
    U, s, Vh = np.linalg.svd(Theta, full_matrices=False)
    k = min(kmax, len(s))
    U, s, Vh = U[:, :k], s[:k], Vh[:k]
    tol = 16.0 * max(Theta.shape) * np.finfo(np.float64).eps * (s[0] if s.size else 0.0)
    zero = s <= tol
    s = np.where(zero, 0.0, s)
    w = s / s[0] if unit and s.size and s[0] > 0 else s
    r = np.sqrt(w)
    return U * r[None, :], r[:, None] * Vh, s


def _factor(Amat: np.ndarray):
    """QR of a site matrix, or (identity, itself) when it has no more rows
    than columns."""
    if Amat.shape[0] <= Amat.shape[1]:
        return np.eye(Amat.shape[0], dtype=Amat.dtype), Amat.copy()
    return _qr(Amat)


def apply_one_site(M, g):
    """Eq. 4: M~[i, ...] = sum_j g[i, j] M[j, ...]."""
    return np.einsum("ij,j...->i...", np.asarray(g), M)


def apply_two_site(M1, M2, G, D_max, vertical, seed, stream, unit=False):
    """Algorithm 1 on one bond; returns (M1~, M2~, singular values kept)."""
    d = M1.shape[0]
    if vertical:
        # shared bond: M1's down (axis 3), M2's up (axis 2)
        A1 = np.transpose(M1, (1, 2, 4, 0, 3))          # [l][u][e][s][x]
        A2 = np.transpose(M2, (1, 3, 4, 0, 2))          # [l][x][e][s][u]
    else:
        # shared bond: M1's right (axis 4), M2's left (axis 1)
        A1 = np.transpose(M1, (1, 2, 3, 0, 4))          # [l][u][x][s][e]
        A2 = np.transpose(M2, (2, 3, 4, 0, 1))          # [u][x][e][s][l]
    o1, o2 = A1.shape[:3], A2.shape[:3]
    Db = A1.shape[4]
    Q1, R1 = _factor(A1.reshape(-1, d * Db))
    Q2, R2 = _factor(A2.reshape(-1, d * Db))
    r1, r2 = R1.shape[0], R2.shape[0]
    G4 = np.asarray(G).reshape(d, d, d, d)             # [i1][i2][j1][j2]
    T = np.einsum("abjk,rjx,tkx->ratb", G4, R1.reshape(r1, d, Db), R2.reshape(r2, d, Db))
    Theta = T.reshape(r1 * d, r2 * d)
    k = min(D_max, r1 * d, r2 * d)
    R1t, R2t, s = _svd_truncate(Theta, k, unit)
    N1 = (Q1 @ R1t.reshape(r1, d * k)).reshape(-1, k)          # [(o1, s)][k]
    N2 = (Q2 @ R2t.T.reshape(r2, d * k)).reshape(-1, k)        # [(o2, s)][k]
    g = philox.gauge_vector(N1.shape[0], seed, stream, np.iscomplexobj(N1))
    phi = g.conj() @ N1
    mag = np.abs(phi)
    if np.iscomplexobj(N1):
        rho = np.where(mag > 0, phi / np.where(mag > 0, mag, 1.0), 1.0)
        N1, N2 = N1 * np.conj(rho)[None, :], N2 * rho[None, :]
    else:
        rho = np.where(phi < 0, -1.0, 1.0)
        N1, N2 = N1 * rho[None, :], N2 * rho[None, :]
    N1 = N1.reshape(*o1, d, k)
    N2 = N2.reshape(*o2, d, k)
    if vertical:
        M1n = np.transpose(N1, (3, 0, 1, 4, 2))          # [s][l][u][k][e]
        M2n = np.transpose(N2, (3, 0, 4, 1, 2))          # [s][l][k][x][e]
    else:
        M1n = np.transpose(N1, (3, 0, 1, 2, 4))          # [s][l][u][x][k]
        M2n = np.transpose(N2, (3, 4, 0, 1, 2))          # [s][k][u][x][e]
    return np.ascontiguousarray(M1n), np.ascontiguousarray(M2n), s


def tebd_bonds(nrow: int, ncol: int):
    """Bonds of one TEBD layer in application order: (site a, site b, vertical)."""
    out = []
    for start in (0, 1):
        for p in range(nrow):
            for q in range(start, ncol - 1, 2):
                out.append((p * ncol + q, p * ncol + q + 1, False))
    for start in (0, 1):
        for p in range(start, nrow - 1, 2):
            for q in range(ncol):
                out.append((p * ncol + q, (p + 1) * ncol + q, True))
    return out


def bond_index(nrow: int, ncol: int, a: int, b: int) -> int:
    """Position of the bond between sites a < b in bond order."""
    p, q = divmod(a, ncol)
    if b == a + 1:
        return p * (ncol - 1) + q
    return nrow * (ncol - 1) + p * ncol + q


def tebd_layer(sites, G, D_max, seed, unit=False, site_gates=None):
    """One-site operators on every site (if given), then G on every
    nearest-neighbour bond (Algorithm 1 each), in tebd_bonds order.

    G: one (d^2 x d^2) operator for every bond, or a list in bond order;
    site_gates: None, one (d x d) operator, or a row-major list per site."""
    nrow, ncol = len(sites), len(sites[0])
    flat = [np.asarray(T) for row in sites for T in row]
    if site_gates is not None:
        per_site = isinstance(site_gates, (list, tuple))
        flat = [apply_one_site(T, site_gates[i] if per_site else site_gates) for i, T in enumerate(flat)]
    per_bond = isinstance(G, (list, tuple))
    sig = []
    for a, b, vertical in tebd_bonds(nrow, ncol):
        g = G[bond_index(nrow, ncol, a, b)] if per_bond else G
        flat[a], flat[b], s = apply_two_site(flat[a], flat[b], g, D_max, vertical, seed, bond_stream(a, b), unit)
        sig.append(s)
    return [flat[p * ncol:(p + 1) * ncol] for p in range(nrow)], sig
