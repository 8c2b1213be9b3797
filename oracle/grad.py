"""Central finite differences of the expectation energy (gradient checks).

E(sites) is oracle.expectation.energy with the ket and bra layers both equal
to ``sites``; every sketch is a fixed function of (seed, stream id), so the
energy is a deterministic smooth function of the site entries away from
rank decisions and the derivative is taken with the sketches held fixed.
"""
from __future__ import annotations

import numpy as np

from .expectation import energy


def _perturbed(sites, pq, idx, delta):
    out = [[T for T in row] for row in sites]
    p, q = pq
    T = sites[p][q].copy()
    T[idx] += delta
    out[p][q] = T
    return out


def fd_entry(sites, terms, pq, idx, m, p, q, seed, h=1e-6):
    ep = energy(_perturbed(sites, pq, idx, h), terms, m, p, q, seed)
    em = energy(_perturbed(sites, pq, idx, -h), terms, m, p, q, seed)
    return (ep - em) / (2 * h)


def fd_directional(sites, terms, direction, m, p, q, seed, h=1e-6):
    """d/dt E(sites + t * direction) at t = 0."""
    plus = [[sites[a][b] + h * direction[a][b] for b in range(len(sites[0]))]
            for a in range(len(sites))]
    minus = [[sites[a][b] - h * direction[a][b] for b in range(len(sites[0]))]
             for a in range(len(sites))]
    return (energy(plus, terms, m, p, q, seed) -
            energy(minus, terms, m, p, q, seed)) / (2 * h)
