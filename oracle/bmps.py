"""Algorithms 2 and 3: boundary-MPS contraction by zip-up (oracle side).

Boundary-MPS sites are [left][vert][right]; in the two-layer form of
Sec. III-B the vertical index is the (ket, bra) pair v = u*DU + U.  The carry
of the zip-up is V [kL][t][a][h]: left bond, (ket, bra) down pair of the
previous column, right bond of the old boundary site, (ket, bra) horizontal
pair into the current column.

Algorithm 2: S <- first row (contracted over the physical index, not
truncated); for every later row, S <- ApproxApply(S, row, m); finally the
boundary (whose vertical bonds are all 1) is contracted to a scalar.
Algorithm 3 (zip-up ApproxApply): V1 <- contraction of S1 with the first
MPO site, then for each following column an einsumsvd splits (V, S_i, O_i)
into the finished site of the previous column and the next carry.

The scalar is returned as (log|v|, arg v); every einsumsvd divides its carry
by sigma_1 and the logs are summed, so no intermediate overflows.
"""
from __future__ import annotations

import numpy as np

from . import philox
from .rsvd import einsumsvd

TRIVIAL_BRA = np.ones((1, 1, 1, 1, 1))


def trivial_bra_rows(nrow: int, ncol: int):
    return [[TRIVIAL_BRA for _ in range(ncol)] for _ in range(nrow)]


def first_row_boundary(ket_row, bra_row):
    """Row one of the two-layer network, contracted over s (not truncated)."""
    out = []
    for K, Kb in zip(ket_row, bra_row):
        d, Dl, Du, Dx, De = K.shape
        _, DL, DU, DX, DE = Kb.shape
        assert Du == 1 and DU == 1, "first row must be a lattice edge"
        S = np.einsum("slxe,sLXE->lLxXeE", K[:, :, 0], np.conj(Kb[:, :, 0]))
        out.append(S.reshape(Dl * DL, Dx * DX, De * DE))
    return out


def zipup_start(S1, K, Kb):
    """V1 of Algorithm 3: first boundary site times the first MPO site."""
    d, Dl, Du, Dx, De = K.shape
    _, DL, DU, DX, DE = Kb.shape
    a, v, b = S1.shape
    assert a == 1 and Dl == 1 and DL == 1
    S4 = S1.reshape(a, Du, DU, b)
    V1 = np.einsum("uUb,suxe,sUXE->xXbeE", S4[0], K[:, 0], np.conj(Kb[:, 0]))
    return V1.reshape(1, Dx * DX, b, De * DE)


def absorb_side(row, alternate):
    """Where a row's einsumsvd steps put Sigma: into the carry ("right") on
    every row, or, with alternating canonicalisation (Sec. III-A), into the
    finished boundary site ("left") on the even rows 2, 4, ..."""
    return "left" if alternate and row % 2 == 0 else "right"


def zipup(S_sites, ket_row, bra_row, m, p, q, seed, direction, row,
          sketch_kind="gauss", rtol=None, record=None, alternate=False):
    """Algorithm 3 on one row; returns (new boundary sites, sum of logs)."""
    n = len(ket_row)
    V = zipup_start(S_sites[0], ket_row[0], bra_row[0])
    new = [None] * n
    total = 0.0
    side = absorb_side(row, alternate)
    for i in range(1, n):
        inst = philox.instance_id(direction, row, i)
        U, W, s, logs1 = einsumsvd(V, S_sites[i], ket_row[i], bra_row[i],
                                   m, p, q, seed, inst, sketch_kind, rtol, absorb=side)
        if record is not None:
            record.append(dict(row=row, col=i, sigma=s, logs1=logs1,
                               M=U.shape[0] * U.shape[1],
                               N=W.shape[1] * W.shape[2] * W.shape[3]))
        new[i - 1] = U
        V = W
        total += logs1
    k, t, b, h = V.shape
    assert b == 1 and h == 1
    new[n - 1] = V.reshape(k, t, 1)
    return new, total


def boundary_scalar(S_sites):
    """Contract a boundary MPS whose vertical bonds are all 1."""
    v = S_sites[0][:, 0, :]
    for S in S_sites[1:]:
        v = v @ S[:, 0, :]
    return complex(v[0, 0]) if np.iscomplexobj(v) else float(v[0, 0])


def sweep(ket, bra, m, p, q, seed, direction=0, upto=None, sketch_kind="gauss",
          rtol=None, record=None, alternate=False):
    """Boundaries after rows 0..r for r = 0..upto (list) and their log scales."""
    nrow = len(ket)
    if bra is None:
        bra = trivial_bra_rows(nrow, len(ket[0]))
    last = nrow - 1 if upto is None else upto
    S = first_row_boundary(ket[0], bra[0])
    bounds = [S]
    logs = [0.0]
    total = 0.0
    for r in range(1, last + 1):
        S, lg = zipup(S, ket[r], bra[r], m, p, q, seed, direction, r,
                      sketch_kind, rtol, record, alternate)
        total += lg
        bounds.append(S)
        logs.append(total)
    return bounds, logs


def contract(ket, bra, m, p, q, seed, direction=0, sketch_kind="gauss",
             rtol=None, record=None, alternate=False):
    """Algorithm 2: returns (log|v|, arg v) of the contracted network.

    ``bra=None`` is the one-layer contraction (ket sites have d = 1); for a
    norm pass ``bra=ket`` (the bra layer enters conjugated).  ``alternate``
    selects the alternating canonicalisation of Sec. III-A (absorb_side).
    """
    bounds, logs = sweep(ket, bra, m, p, q, seed, direction, None, sketch_kind,
                         rtol, record, alternate)
    v = boundary_scalar(bounds[-1])
    if v == 0:
        return float("-inf"), 0.0
    return float(np.log(abs(v)) + logs[-1]), float(np.angle(v))


def flip_vertical(sites):
    """Lattice read bottom-up: rows reversed and up/down bonds swapped."""
    return [[np.ascontiguousarray(T.transpose(0, 1, 3, 2, 4)) for T in row]
            for row in sites[::-1]]


def transpose_lattice(sites):
    """Lattice with rows and columns exchanged: left<->up, down<->right."""
    nrow, ncol = len(sites), len(sites[0])
    return [[np.ascontiguousarray(sites[p][q].transpose(0, 2, 1, 4, 3))
             for p in range(nrow)] for q in range(ncol)]
