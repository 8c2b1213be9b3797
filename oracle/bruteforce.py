"""Exact (exponential-cost) contractions used to pin the oracle on tiny lattices.

Two independent exact methods, neither sharing code with bmps.py:
  * ``exact_scalar``: the whole one-layer network (the double layer formed
    site by site over the physical index, as the naive way of Sec. III-B)
    handed to one einsum;
  * ``transfer_scalar``: row-by-row transfer of a dense boundary vector over
    all vertical bonds, never truncated.
``statevector`` contracts the ket layer alone into the 2^n amplitude tensor
(Sec. II-A) for energy checks against a dense state vector.
"""
from __future__ import annotations

import string

import numpy as np


def double_layer(K, Kb):
    """E[(l,L)][(u,U)][(x,X)][(e,E)] = sum_s K[s,l,u,x,e] conj(Kb[s,L,U,X,E])."""
    d, Dl, Du, Dx, De = K.shape
    _, DL, DU, DX, DE = Kb.shape
    E = np.einsum("sluxe,sLUXE->lLuUxXeE", K, np.conj(Kb))
    return E.reshape(Dl * DL, Du * DU, Dx * DX, De * DE)


def _layer(ket, bra):
    nrow, ncol = len(ket), len(ket[0])
    if bra is None:
        one = np.ones((1, 1, 1, 1, 1))
        bra = [[one] * ncol for _ in range(nrow)]
    return [[double_layer(ket[p][q], bra[p][q]) for q in range(ncol)]
            for p in range(nrow)]


def exact_scalar(ket, bra):
    """Exact value of the one-layer (bra=None) or two-layer network."""
    E = _layer(ket, bra)
    nrow, ncol = len(E), len(E[0])
    letters = iter(string.ascii_letters)
    hb = {}
    vb = {}
    for p in range(nrow):
        for q in range(ncol - 1):
            hb[p, q] = next(letters)
    for p in range(nrow - 1):
        for q in range(ncol):
            vb[p, q] = next(letters)
    ops, subs = [], []
    for p in range(nrow):
        for q in range(ncol):
            T = E[p][q]
            idx = ""
            shp = []
            if q > 0:
                idx += hb[p, q - 1]; shp.append(T.shape[0])
            if p > 0:
                idx += vb[p - 1, q]; shp.append(T.shape[1])
            if p < nrow - 1:
                idx += vb[p, q]; shp.append(T.shape[2])
            if q < ncol - 1:
                idx += hb[p, q]; shp.append(T.shape[3])
            ops.append(T.reshape(shp))
            subs.append(idx)
    expr = ",".join(subs) + "->"
    return np.einsum(expr, *ops, optimize="greedy")[()]


def transfer_scalar(ket, bra):
    """Exact value by a dense row-to-row transfer vector (no truncation)."""
    E = _layer(ket, bra)
    nrow, ncol = len(E), len(E[0])
    ups = [E[0][q].shape[1] for q in range(ncol)]
    vec = np.ones(int(np.prod(ups)), dtype=E[0][0].dtype)
    for p in range(nrow):
        ups = [E[p][q].shape[1] for q in range(ncol)]
        T = vec.reshape(1, 1, int(np.prod(ups)))        # (done, h, rest)
        for q in range(ncol):
            A = E[p][q]                                 # [h][u][x][r]
            done, h, rest = T.shape
            uq = A.shape[1]
            T4 = T.reshape(done, h, uq, rest // uq)
            N = np.einsum("phur,huxs->pxsr", T4, A)
            T = N.reshape(done * A.shape[2], A.shape[3], rest // uq)
        vec = T.reshape(-1)
    return vec.reshape(())[()]


def statevector(ket):
    """Amplitudes psi[s_00, s_01, ..., s_(n-1)(n-1)] (row-major site order)."""
    nrow, ncol = len(ket), len(ket[0])
    letters = iter(string.ascii_letters)
    phys = {}
    hb, vb = {}, {}
    for p in range(nrow):
        for q in range(ncol):
            phys[p, q] = next(letters)
    for p in range(nrow):
        for q in range(ncol - 1):
            hb[p, q] = next(letters)
    for p in range(nrow - 1):
        for q in range(ncol):
            vb[p, q] = next(letters)
    ops, subs = [], []
    for p in range(nrow):
        for q in range(ncol):
            T = ket[p][q]
            idx = phys[p, q]
            shp = [T.shape[0]]
            if q > 0:
                idx += hb[p, q - 1]; shp.append(T.shape[1])
            if p > 0:
                idx += vb[p - 1, q]; shp.append(T.shape[2])
            if p < nrow - 1:
                idx += vb[p, q]; shp.append(T.shape[3])
            if q < ncol - 1:
                idx += hb[p, q]; shp.append(T.shape[4])
            ops.append(T.reshape(shp))
            subs.append(idx)
    out = "".join(phys[p, q] for p in range(nrow) for q in range(ncol))
    return np.einsum(",".join(subs) + "->" + out, *ops, optimize="greedy")


def statevector_energy(ket, terms):
    """<psi|H|psi>/<psi|psi> with H = sum_t c_t O_t applied term by term."""
    psi = statevector(ket)
    ncol = len(ket[0])
    norm = np.vdot(psi, psi)
    total = 0.0
    for sites, op, coeff in terms:
        axes = [p * ncol + q for (p, q) in sites]
        n = len(axes)
        d = psi.shape[0]
        O = op.reshape([d] * (2 * n))
        phi = np.tensordot(O, psi, axes=(list(range(n, 2 * n)), axes))
        phi = np.moveaxis(phi, list(range(n)), axes)
        total += coeff * np.vdot(psi, phi)
    return (total / norm).real
