"""Pins of the oracle's boundary-MPS contraction (Algorithms 2 and 3).

In the exact regime (truncation m at or above every cut rank) the zip-up
must reproduce two independent exact contractions; away from it, the
structure of the method fixes product-state values, scaling laws, the
invariance under the transposed lattice in the exact regime, and that the
randomized SVD adds no error over a dense SVD once it has converged.
"""
import numpy as np
import pytest

import synth
from oracle import bmps, bruteforce
from oracle.implicit import ImplicitOp
from oracle import rsvd


def test_c1_one_layer_equals_bruteforce():
    cfg = synth.config("c1")
    ket = synth.peps_for(cfg)
    la, ph = bmps.contract(ket, None, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    ex = bruteforce.exact_scalar(ket, None)
    tr = bruteforce.transfer_scalar(ket, None)
    assert tr == pytest.approx(ex, rel=1e-12)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-12)
    assert np.cos(ph) == pytest.approx(np.sign(ex), abs=1e-12)


@pytest.mark.parametrize("shape,D,m", [((3, 3), 2, 16), ((2, 4), 2, 16), ((3, 2), 3, 81)])
def test_two_layer_exact_regime(shape, D, m):
    nr, nc = shape
    ket = synth.random_peps(nr, nc, 2, D, "c64", "cgauss_scaled", 31)
    la, ph = bmps.contract(ket, ket, m, 4, 1, 77)
    ex = bruteforce.exact_scalar(ket, ket)
    psi = bruteforce.statevector(ket)
    assert abs(ex - np.vdot(psi, psi)) <= 1e-12 * abs(ex)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-10)
    assert abs(np.sin(ph)) < 1e-10


def test_rank_deficient_block_zero_padding():
    """3 x 5 with m = 64: on the middle row the step at column 3 asks for
    k = 64 > cut rank 16, so 48 directions are numerically zero and must be
    padded with zeros, not kept."""
    ket = synth.random_peps(3, 5, 2, 2, "c64", "cgauss_scaled", 5)
    rec = []
    la, _ = bmps.contract(ket, ket, 64, 8, 1, 3, record=rec)
    ex = bruteforce.exact_scalar(ket, ket)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-10)
    zeros = [int(np.sum(r["sigma"] == 0)) for r in rec]
    assert max(zeros) > 0


def test_product_state_norm():
    """D = 1: the norm is the product of the local norms."""
    ket = synth.random_peps(4, 4, 2, 1, "c64", "cgauss_scaled", 8)
    la, _ = bmps.contract(ket, ket, 4, 2, 1, 1)
    ref = sum(np.log(np.vdot(T, T).real) for row in ket for T in row)
    assert la == pytest.approx(ref, abs=1e-12)


def test_site_scaling_law():
    """Scaling one site by c shifts the log-norm by 2 log|c| (truncated regime)."""
    ket = synth.random_peps(4, 4, 2, 3, "c64", "cgauss_scaled", 9)
    la, _ = bmps.contract(ket, ket, 5, 2, 1, 4)
    ket2 = [[T for T in row] for row in ket]
    c = 2.5 - 1.0j
    ket2[2][1] = ket[2][1] * c
    lb, _ = bmps.contract(ket2, ket2, 5, 2, 1, 4)
    assert lb - la == pytest.approx(2 * np.log(abs(c)), abs=1e-10)


def test_transposed_lattice_exact_regime():
    ket = synth.random_peps(3, 3, 2, 2, "c64", "cgauss_scaled", 12)
    la, _ = bmps.contract(ket, ket, 16, 4, 1, 2)
    lt, _ = bmps.contract(bmps.transpose_lattice(ket), bmps.transpose_lattice(ket), 16, 4, 1, 2)
    lf, _ = bmps.contract(bmps.flip_vertical(ket), bmps.flip_vertical(ket), 16, 4, 1, 2)
    assert lt == pytest.approx(la, abs=1e-10)
    assert lf == pytest.approx(la, abs=1e-10)


def _dense_einsumsvd(V, S, K, Kb, m, *args, absorb="right", **kw):
    """Naive einsumsvd: form A explicitly and take LAPACK's truncated SVD."""
    op = ImplicitOp(V, S, K, Kb)
    A = op.dense()
    k = min(m, op.M, op.N)
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    U, s, Vh = U[:, :k], s[:k], Vh[:k]
    W = s[:, None] * Vh / s[0]
    Dx, DX, b, De, DE = op.col_shape
    return (U.reshape(op.dims["kL"], op.dims["t"], k),
            W.reshape(k, Dx * DX, b, De * DE), s, float(np.log(s[0])))


def test_no_additional_error_versus_dense_svd(monkeypatch):
    """With enough power iterations the implicit rSVD contraction matches the
    contraction that uses a dense truncated SVD (the accuracy claim of the
    randomized-SVD experiments): both truncate to the same m."""
    ket = synth.random_peps(4, 4, 2, 3, "c64", "cgauss_scaled", 21)
    la, _ = bmps.contract(ket, ket, 6, 10, 12, 5)
    monkeypatch.setattr(bmps, "einsumsvd", _dense_einsumsvd)
    ld, _ = bmps.contract(ket, ket, 6, 10, 12, 5)
    assert la == pytest.approx(ld, abs=1e-8)


def test_truncated_regime_close_to_exact():
    ket = synth.random_peps(4, 4, 2, 2, "c64", "cgauss_scaled", 13)
    ex = np.log(abs(bruteforce.exact_scalar(ket, ket)))
    errs = [abs(bmps.contract(ket, ket, m, 4, 2, 6)[0] - ex) for m in (2, 8, 16)]
    assert errs[1] < errs[0]
    assert errs[2] < 1e-10          # m = 16 is the largest cut rank: exact


def test_left_absorption_is_the_same_factorisation():
    """absorb="left" (Sigma into the finished site) factorises the same
    truncated matrix: U W is unchanged, the carry's rows are orthonormal
    (V^H), U's column norms are sigma_c / sigma_1, the log-scale is the same,
    and the gauge phases (<g, u_c> real and >= 0) still hold."""
    rng = np.random.default_rng(4)
    cplx = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)   # noqa: E731
    V, S, K, Kb = cplx(3, 4, 5, 4), cplx(5, 4, 3), cplx(2, 2, 2, 2, 2), cplx(2, 2, 2, 2, 2)
    Ur, Wr, sr, lr = rsvd.einsumsvd(V, S, K, Kb, 6, 4, 2, 11, 3)
    Ul, Wl, sl, ll = rsvd.einsumsvd(V, S, K, Kb, 6, 4, 2, 11, 3, absorb="left")
    k = len(sr)
    assert np.array_equal(sr, sl) and lr == ll
    UWr = Ur.reshape(-1, k) @ Wr.reshape(k, -1)
    UWl = Ul.reshape(-1, k) @ Wl.reshape(k, -1)
    assert np.linalg.norm(UWl - UWr) <= 1e-12 * np.linalg.norm(UWr)
    Wm = Wl.reshape(k, -1)
    assert np.allclose(Wm @ Wm.conj().T, np.eye(k), atol=1e-12)
    assert np.allclose(np.linalg.norm(Ul.reshape(-1, k), axis=0), sl / sl[0], atol=1e-12)
    g = rsvd.philox.gauge_vector(Ul.reshape(-1, k).shape[0], 11, 3, True)
    ph = g.conj() @ Ul.reshape(-1, k)
    assert np.all(np.abs(ph.imag) <= 1e-12 * np.abs(ph)) and np.all(ph.real >= 0)


@pytest.mark.parametrize("shape,D,m", [((3, 3), 2, 16), ((4, 3), 2, 16)])
def test_alternating_canonicalisation_exact_regime(shape, D, m):
    """Alternating where Sigma goes (Sec. III-A) changes no exact contraction."""
    nr, nc = shape
    ket = synth.random_peps(nr, nc, 2, D, "c64", "cgauss_scaled", 41)
    la, ph = bmps.contract(ket, ket, m, 4, 1, 77, alternate=True)
    ex = bruteforce.exact_scalar(ket, ket)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-10)
    assert abs(np.sin(ph)) < 1e-10
    assert [bmps.absorb_side(r, True) for r in (1, 2, 3, 4)] == ["right", "left", "right", "left"]


def test_alternating_canonicalisation_truncated_regime():
    """Truncated: a different (still valid) approximation of the same norm,
    as close to the exact value as the right-absorbing sweep at each m."""
    ket = synth.random_peps(4, 4, 2, 2, "c64", "cgauss_scaled", 43)
    ex = np.log(abs(bruteforce.exact_scalar(ket, ket)))
    for m in (3, 6):
        lr = bmps.contract(ket, ket, m, 4, 2, 6)[0]
        la = bmps.contract(ket, ket, m, 4, 2, 6, alternate=True)[0]
        assert la != lr
        assert abs(la - ex) < 5 * abs(lr - ex) + 1e-6
