"""Pins of the oracle's imaginary-time evolution (Sec. II-D):
  * on open chains (no truncation, exact contraction) every step's energy
    equals the Rayleigh quotient of the state vector evolved by the same
    operators in the same order;
  * with truncation the energy is still a Rayleigh quotient of a valid
    state: never below the exact ground-state energy (dense diagonalisation
    of the 3 x 3 transverse-field Ising Hamiltonian), and it falls from the
    random start."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, ite, qrsvd


def _dense_apply(psi, op, axes, n, d=2):
    k = len(axes)
    T = np.moveaxis(psi.reshape([d] * n), axes, list(range(k)))
    T = np.tensordot(op.reshape([d] * (2 * k)), T, axes=(list(range(k, 2 * k)), list(range(k))))
    return np.moveaxis(T, list(range(k)), axes).reshape(-1)


def _dense_energy(psi, terms, ncol, n):
    tot = 0.0
    for st, op, coeff in terms:
        axes = [p * ncol + q for p, q in st]
        tot += coeff * np.vdot(psi, _dense_apply(psi, op, axes, n))
    return (tot / np.vdot(psi, psi)).real


@pytest.mark.parametrize("shape", [(1, 4), (4, 1)])
def test_exact_ite_equals_state_vector_ite(shape):
    # open chains: every bond's Theta has at most the rank of the state across
    # that bond (2^2 on 4 sites), so D_max = 4 never truncates, and the single
    # row (or column) makes Eq. 6 exact
    nr, nc = shape
    n = nr * nc
    ket = synth.random_peps(nr, nc, 2, 2, "c64", "cgauss_scaled", 61)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    Gb, Gs = synth.tfi_ite_gates(1.0, 3.0, 0.05)
    _, energies = ite.ite(ket, Gb, Gs, 4, 5, 4, terms, 16, 8, 2, 9)
    psi = bruteforce.statevector(ket).reshape(-1)
    for e in energies:
        for i in range(n):
            psi = _dense_apply(psi, Gs, [i], n)
        for a, b, _ in qrsvd.tebd_bonds(nr, nc):
            psi = _dense_apply(psi, Gb, [a, b], n)
        assert abs(e - _dense_energy(psi, terms, nc, n)) <= 1e-10 * abs(e)


def _tfi_ground(nr, nc, J, h):
    n = nr * nc
    Z = np.diag([1.0, -1.0])
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    I = np.eye(2)

    def op(mats):
        out = np.ones((1, 1))
        for i in range(n):
            out = np.kron(out, mats.get(i, I))
        return out
    H = np.zeros((2 ** n, 2 ** n))
    for p in range(nr):
        for q in range(nc):
            i = p * nc + q
            if q + 1 < nc:
                H -= J * op({i: Z, i + 1: Z})
            if p + 1 < nr:
                H -= J * op({i: Z, i + nc: Z})
            H -= h * op({i: X})
    return np.linalg.eigvalsh(H)[0]


def test_truncated_ite_is_variational():
    nr, nc = 3, 3
    ket = synth.random_peps(nr, nc, 2, 2, "c64", "cgauss_scaled", 67)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    Gb, Gs = synth.tfi_ite_gates(1.0, 3.0, 0.1)
    start = _dense_energy(bruteforce.statevector(ket).reshape(-1), terms, nc, nr * nc)
    _, energies = ite.ite(ket, Gb, Gs, 2, 5, 6, terms, 16, 8, 2, 9)
    ground = _tfi_ground(nr, nc, 1.0, 3.0)
    assert all(e >= ground - 1e-9 * abs(ground) for e in energies)
    assert energies[-1] < start and energies[-1] < energies[0]
    assert energies[-1] - ground <= 0.05 * abs(ground)
