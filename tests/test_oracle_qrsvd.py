"""Pins of the oracle's operator application by QR-SVD (Algorithm 1) and of
one TEBD layer, against what the mathematics fixes:
  * without truncation the updated pair contracts to G applied to the old
    pair exactly (Eq. 5 holds with equality);
  * with truncation the error of the updated pair is the Eckart-Young error
    of Theta (the Q factors are isometries), and the kept singular values
    are Theta's leading ones;
  * a TEBD layer without truncation equals the gates applied one by one to
    the dense state vector in the same order; identity gates leave the
    state unchanged;
  * the gauge rule <g, u_c> real and >= 0 holds on the returned factors."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, philox, qrsvd


def _rand(rng, shape, cplx=True):
    x = rng.standard_normal(shape)
    return x + 1j * rng.standard_normal(shape) if cplx else x


def _gate(rng, d=2, cplx=True):
    return _rand(rng, (d * d, d * d), cplx)


def _pair_tensor(M1, M2, vertical):
    """The two sites contracted over their shared bond, open legs in a fixed
    order: [s1][s2][M1 outer bonds][M2 outer bonds]."""
    if vertical:
        return np.einsum("sluxe,tLxXE->stlueLXE", M1, M2)
    return np.einsum("sluxe,teUXE->stluxUXE", M1, M2)


@pytest.mark.parametrize("vertical", [False, True])
@pytest.mark.parametrize("cplx", [False, True])
def test_exact_when_not_truncated(vertical, cplx):
    rng = np.random.default_rng(1 + vertical + 2 * cplx)
    d, D = 2, 3
    M1 = _rand(rng, (d, D, D, D, D), cplx)
    M2 = _rand(rng, (d, D, D, D, D), cplx)
    G = _gate(rng, d, cplx)
    N1, N2, s = qrsvd.apply_two_site(M1, M2, G, 100, vertical, 7, qrsvd.bond_stream(0, 1))
    ref = np.einsum("abjk,jk...->ab...", G.reshape(d, d, d, d), _pair_tensor(M1, M2, vertical))
    got = _pair_tensor(N1, N2, vertical)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert N1.shape[4 if not vertical else 3] == len(s) == d * D * d


@pytest.mark.parametrize("vertical", [False, True])
def test_truncation_error_is_eckart_young(vertical):
    rng = np.random.default_rng(11)
    d, D = 2, 3
    M1 = _rand(rng, (d, D, D, D, D))
    M2 = _rand(rng, (d, D, D, D, D))
    G = _gate(rng, d)
    full = np.einsum("abjk,jk...->ab...", G.reshape(d, d, d, d), _pair_tensor(M1, M2, vertical))
    _, _, s_all = qrsvd.apply_two_site(M1, M2, G, 100, vertical, 7, 5)
    for k in (2, 4, 5):
        N1, N2, s = qrsvd.apply_two_site(M1, M2, G, k, vertical, 7, 5)
        err = np.linalg.norm(_pair_tensor(N1, N2, vertical) - full)
        assert err == pytest.approx(np.sqrt(np.sum(s_all[k:] ** 2)), rel=1e-10)
        assert np.allclose(s, s_all[:k], rtol=1e-12)


def test_gauge_rule():
    """<g, column c of the updated first site> is real and >= 0, whatever
    orthonormal basis the factorisation used (Q and -Q give the same sites)."""
    rng = np.random.default_rng(13)
    d, D = 2, 2
    M1, M2, G = _rand(rng, (d, 2, D, D, D)), _rand(rng, (d, D, D, D, 1)), _gate(rng)
    N1, N2, s = qrsvd.apply_two_site(M1, M2, G, 3, False, 9, 21)
    k = len(s)
    N1m = np.transpose(N1, (1, 2, 3, 0, 4)).reshape(-1, k)
    g = philox.gauge_vector(N1m.shape[0], 9, 21, True)
    ph = g.conj() @ N1m
    assert np.all(np.abs(ph.imag) <= 1e-10 * np.abs(ph)) and np.all(ph.real >= 0)
    real_qr = qrsvd._qr

    def flipped(A):
        Q, R = real_qr(A)
        return -Q, -R
    qrsvd._qr = flipped
    try:
        F1, F2, _ = qrsvd.apply_two_site(M1, M2, G, 3, False, 9, 21)
    finally:
        qrsvd._qr = real_qr
    assert np.allclose(F1, N1, atol=1e-12) and np.allclose(F2, N2, atol=1e-12)


def _apply_gate_dense(psi, G, a, b, n):
    d = 2
    T = psi.reshape([d] * n)
    T = np.moveaxis(T, (a, b), (0, 1))
    T = np.tensordot(G.reshape(d, d, d, d), T, axes=([2, 3], [0, 1]))
    return np.moveaxis(T, (0, 1), (a, b)).reshape(-1)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 2)])
def test_tebd_layer_equals_dense_gates(shape):
    nr, nc = shape
    rng = np.random.default_rng(17 + nr)
    ket = synth.random_peps(nr, nc, 2, 2, "c64", "cgauss_scaled", 23 + nc)
    G = _gate(rng)
    new, sig = qrsvd.tebd_layer(ket, G, 64, 3)
    psi = bruteforce.statevector(ket).reshape(-1)
    for a, b, _ in qrsvd.tebd_bonds(nr, nc):
        psi = _apply_gate_dense(psi, G, a, b, nr * nc)
    got = bruteforce.statevector(new).reshape(-1)
    assert np.linalg.norm(got - psi) <= 1e-11 * np.linalg.norm(psi)
    n_bonds = nr * (nc - 1) + (nr - 1) * nc
    assert len(qrsvd.tebd_bonds(nr, nc)) == n_bonds == len(sig)


def test_identity_gates_keep_the_state():
    ket = synth.random_peps(3, 3, 2, 2, "c64", "cgauss_scaled", 5)
    new, _ = qrsvd.tebd_layer(ket, np.eye(4), 8, 1)
    a = bruteforce.statevector(ket).reshape(-1)
    b = bruteforce.statevector(new).reshape(-1)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a)


def _apply_site_dense(psi, g, a, n):
    d = 2
    T = np.moveaxis(psi.reshape([d] * n), a, 0)
    T = np.tensordot(g, T, axes=([1], [0]))
    return np.moveaxis(T, 0, a).reshape(-1)


def test_per_bond_and_site_operators_equal_dense_application():
    """Distinct operators per bond (looked up by the pair of sites they join)
    and per site: without truncation the layer equals the site operators
    then the bond operators applied to the state vector in layer order."""
    nr, nc = 2, 3
    rng = np.random.default_rng(41)
    ket = synth.random_peps(nr, nc, 2, 2, "c64", "cgauss_scaled", 43)
    by_pair = {(a, b): _gate(rng) for a, b, _ in qrsvd.tebd_bonds(nr, nc)}
    # bond order: horizontal bonds by left site, then vertical bonds by upper site
    order = [(p * nc + q, p * nc + q + 1) for p in range(nr) for q in range(nc - 1)]
    order += [(p * nc + q, (p + 1) * nc + q) for p in range(nr - 1) for q in range(nc)]
    gates = [by_pair[ab] for ab in order]
    site_ops = [_rand(rng, (2, 2)) for _ in range(nr * nc)]
    new, _ = qrsvd.tebd_layer(ket, gates, 64, 3, site_gates=site_ops)
    psi = bruteforce.statevector(ket).reshape(-1)
    for i, g in enumerate(site_ops):
        psi = _apply_site_dense(psi, g, i, nr * nc)
    for a, b, _ in qrsvd.tebd_bonds(nr, nc):
        psi = _apply_gate_dense(psi, by_pair[(a, b)], a, b, nr * nc)
    got = bruteforce.statevector(new).reshape(-1)
    assert np.linalg.norm(got - psi) <= 1e-11 * np.linalg.norm(psi)


def test_unit_bonds_change_only_the_scale():
    """Normalised bonds: the same state up to one positive factor, and each
    bond's singular values the same up to one positive factor."""
    ket = synth.random_peps(3, 2, 2, 2, "c64", "cgauss_scaled", 47)
    G = _gate(np.random.default_rng(49))
    a, sa = qrsvd.tebd_layer(ket, G, 2, 5)
    b, sb = qrsvd.tebd_layer(ket, G, 2, 5, unit=True)
    pa = bruteforce.statevector(a).reshape(-1)
    pb = bruteforce.statevector(b).reshape(-1)
    c = np.vdot(pb, pa) / np.vdot(pb, pb)
    assert abs(c.imag) <= 1e-10 * abs(c) and c.real > 0
    assert np.linalg.norm(pa - c * pb) <= 1e-10 * np.linalg.norm(pa)
    for x, y in zip(sa, sb):
        assert np.allclose(x / x[0], y / y[0], rtol=1e-10)
