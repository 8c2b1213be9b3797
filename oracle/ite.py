"""Imaginary-time evolution by TEBD (Sec. II-D), oracle side.

TEST INFRASTRUCTURE ONLY (see the package docstring).

One ITE step applies exp(-tau H_j) for every local term H_j of
H = sum_j H_j (first-order Trotter-Suzuki product): the one-site operators
on every site (Eq. 4), then the two-site operators on every
nearest-neighbour bond by Algorithm 1 (qrsvd.tebd_layer, bonds normalised by
their largest singular value so the state's scale stays bounded).  After
every step the Rayleigh quotient <psi|H|psi> / <psi|psi> is evaluated by
Eq. 6 with the cached environments of Sec. IV-B (expectation.energy).
"""
from __future__ import annotations

from . import expectation, qrsvd


def ite(sites, bond_gates, site_gates, D_max, seed, steps, terms, m, p, q, sketch_seed):
    """Returns (final sites, [energy after each step])."""
    energies = []
    for _ in range(steps):
        sites, _ = qrsvd.tebd_layer(sites, bond_gates, D_max, seed, unit=True, site_gates=site_gates)
        energies.append(expectation.energy(sites, terms, m, p, q, sketch_seed))
    return sites, energies
