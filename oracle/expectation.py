"""Expectation values by Eq. 6 with cached boundary environments (Sec. IV-B).

<psi|H|psi> / <psi|psi> for H = sum_t c_t O_t.  Following Sec. IV-B, two
full two-layer boundary sweeps (top-down and bottom-up) are run once and the
boundary after every row is kept; each local term is then a 3 x n strip
(upper environment, the row holding the term, lower environment) contracted
exactly.  Readings of points the paper leaves open:
  * each term is normalised by its own strip without operator,
    <O_t> = strip(O_t) / strip(1); the energy is sum_t c_t <O_t>;
  * terms on vertical bonds use the same procedure on the transposed lattice
    (the paper caches "rows (or columns)");
  * a two-site operator enters through its operator-Schmidt decomposition
    O = sum_x A_x (x) B_x, so every strip carries one-site operators only;
  * sweep directions get their own sketch streams: 0 top-down, 1 bottom-up,
    2 and 3 the same on the transposed lattice.
"""
from __future__ import annotations

import numpy as np

from . import bmps


def operator_schmidt(op: np.ndarray, d: int, tol: float = 1e-14):
    """O[(s1',s2'),(s1,s2)] = sum_x A_x[s1',s1] B_x[s2',s2]."""
    O4 = op.reshape(d, d, d, d)
    M = O4.transpose(0, 2, 1, 3).reshape(d * d, d * d)
    U, s, Vh = np.linalg.svd(M)
    keep = s > tol * s[0]
    return [(U[:, x].reshape(d, d) * s[x], Vh[x].reshape(d, d))
            for x in np.nonzero(keep)[0]]


def trivial_env(ncol: int):
    return [np.ones((1, 1, 1)) for _ in range(ncol)]


def strip_value(upper, ket_row, bra_row, lower, ops):
    """Exact contraction of (upper env) x (row with ops) x (lower env)."""
    L = np.ones((1, 1, 1, 1))            # [a][l][L][c]
    for q, (K, Kb) in enumerate(zip(ket_row, bra_row)):
        if q in ops:
            K = np.einsum("ts,sluxe->tluxe", ops[q], K)
        _, Dl, Du, Dx, De = K.shape
        _, DL, DU, DX, DE = Kb.shape
        a, _, b = upper[q].shape
        c, _, f = lower[q].shape
        T = upper[q].reshape(a, Du, DU, b)
        Bt = lower[q].reshape(c, Dx, DX, f)
        # the five-tensor product of this column as four pairwise sums
        A1 = np.einsum("alLc,auUb->lLcuUb", L, T)
        A2 = np.einsum("lLcuUb,sluxe->LcUbsxe", A1, K)
        A3 = np.einsum("LcUbsxe,sLUXE->cbexXE", A2, np.conj(Kb))
        L = np.einsum("cbexXE,cxXf->beEf", A3, Bt)
    return L.reshape(-1)[0]


def row_environments(sites, m, p, q, seed, dir_top, dir_bot, sketch_kind="gauss"):
    """upper[r], lower[r]: boundaries above and below row r."""
    nrow, ncol = len(sites), len(sites[0])
    top, _ = bmps.sweep(sites, sites, m, p, q, seed, dir_top, nrow - 2, sketch_kind) \
        if nrow > 1 else ([], [])
    flipped = bmps.flip_vertical(sites)
    bot, _ = bmps.sweep(flipped, flipped, m, p, q, seed, dir_bot, nrow - 2, sketch_kind) \
        if nrow > 1 else ([], [])
    upper = [trivial_env(ncol)] + [top[r] for r in range(nrow - 1)]
    lower = [bot[nrow - 2 - r] for r in range(nrow - 1)] + [trivial_env(ncol)]
    return upper, lower


def _term_values(sites, row_terms, m, p, q, seed, dir_top, dir_bot, sketch_kind):
    """Sum of c_t <O_t> for terms given as {row: [(col->op dict list, c)]}."""
    upper, lower = row_environments(sites, m, p, q, seed, dir_top, dir_bot, sketch_kind)
    total = 0.0
    per_term = []
    for r, tlist in sorted(row_terms.items()):
        norm = strip_value(upper[r], sites[r], sites[r], lower[r], {})
        for (components, coeff, tag) in tlist:
            val = sum(strip_value(upper[r], sites[r], sites[r], lower[r], ops)
                      for ops in components)
            e = coeff * val / norm
            per_term.append((tag, e))
            total += e
    return total, per_term


def energy(sites, terms, m, p, q, seed, sketch_kind="gauss", return_terms=False):
    """Rayleigh quotient <psi|H|psi>/<psi|psi> (Eq. 6 with Sec. IV-B caching)."""
    nrow, ncol = len(sites), len(sites[0])
    d = sites[0][0].shape[0]
    rows_h, rows_v = {}, {}
    for ti, (st, op, coeff) in enumerate(terms):
        if len(st) == 1:
            (r, c), = st
            rows_h.setdefault(r, []).append(([{c: op}], coeff, ti))
            continue
        (r0, c0), (r1, c1) = st
        comps = operator_schmidt(op, d)
        if r0 == r1 and c1 == c0 + 1:
            rows_h.setdefault(r0, []).append(
                ([{c0: A, c1: B} for A, B in comps], coeff, ti))
        elif c0 == c1 and r1 == r0 + 1:
            # on the transposed lattice the bond (r0,c)-(r0+1,c) is horizontal
            rows_v.setdefault(c0, []).append(
                ([{r0: A, r1: B} for A, B in comps], coeff, ti))
        else:
            raise ValueError("only nearest-neighbour terms (left-to-right or top-down)")
    e_h, t_h = _term_values(sites, rows_h, m, p, q, seed, 0, 1, sketch_kind)
    e_v, t_v = 0.0, []
    if rows_v:
        tsites = bmps.transpose_lattice(sites)
        e_v, t_v = _term_values(tsites, rows_v, m, p, q, seed, 2, 3, sketch_kind)
    e = e_h + e_v
    e = float(np.real(e))
    if return_terms:
        vals = dict(t_h + t_v)
        return e, [vals[i] for i in range(len(terms))]
    return e
