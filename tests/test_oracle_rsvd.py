"""Pins of the oracle's implicit operator (Sec. IV-A) and Algorithm 4.

The implicit products are checked against the explicitly formed matrix and
the adjoint identity; the randomized SVD against LAPACK's dense SVD in the
exact regime, Ritz interlacing, the Eckart-Young bound and orthogonality.
"""
import numpy as np
import pytest

from oracle import philox
from oracle.implicit import ImplicitOp
from oracle.rsvd import einsumsvd, orthogonalize, rsvd_implicit, block_sizes


def _rand(rng, shape, cplx):
    x = rng.standard_normal(shape)
    if cplx:
        x = x + 1j * rng.standard_normal(shape)
    return x


def make_op(rng, kL=3, t=4, a=5, b=3, d=2, D=(2, 2, 2, 2), DB=(2, 2, 2, 2), cplx=True):
    Dl, Du, Dx, De = D
    DL, DU, DX, DE = DB
    V = _rand(rng, (kL, t, a, Dl * DL), cplx)
    S = _rand(rng, (a, Du * DU, b), cplx)
    K = _rand(rng, (d, Dl, Du, Dx, De), cplx)
    Kb = _rand(rng, (d, DL, DU, DX, DE), cplx)
    return ImplicitOp(V, S, K, Kb)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("dims", [
    dict(kL=3, t=4, a=5, b=3, d=2, D=(2, 2, 2, 2), DB=(2, 2, 2, 2)),
    dict(kL=1, t=4, a=2, b=1, d=3, D=(1, 2, 2, 1), DB=(1, 2, 2, 1)),
    dict(kL=2, t=3, a=4, b=2, d=2, D=(2, 3, 1, 2), DB=(3, 1, 2, 1)),
])
def test_implicit_products_match_dense(cplx, dims):
    rng = np.random.default_rng(1)
    op = make_op(rng, cplx=cplx, **dims)
    A = op.dense()
    X = _rand(rng, (op.N, 5), cplx)
    Y = _rand(rng, (op.M, 5), cplx)
    np.testing.assert_allclose(op.matvec(X), A @ X, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(op.rmatvec(Y), A.conj().T @ Y, rtol=1e-12, atol=1e-12)
    # adjoint identity <Y, A X> = <A^H Y, X>
    lhs = np.vdot(Y, op.matvec(X))
    rhs = np.vdot(op.rmatvec(Y), X)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_dense_matrix_entry_by_definition():
    """One entry of A summed by explicit loops over every contracted index."""
    rng = np.random.default_rng(2)
    op = make_op(rng, kL=2, t=2, a=2, b=2, d=2, D=(2, 1, 2, 1), DB=(1, 2, 1, 2))
    A = op.dense()
    k, t, x, X, b, e, E = 1, 1, 1, 0, 1, 0, 1
    g = op.dims
    tot = 0
    for a in range(g["a"]):
        for l in range(g["Dl"]):
            for L in range(g["DL"]):
                for u in range(g["Du"]):
                    for U in range(g["DU"]):
                        for s in range(g["d"]):
                            tot += (op.V[k, t, a, l * g["DL"] + L]
                                    * op.S[a, u * g["DU"] + U, b]
                                    * op.K[s, l, u, x, e]
                                    * np.conj(op.Kb[s, L, U, X, E]))
    col = (((x * g["DX"] + X) * g["b"] + b) * g["De"] + e) * g["DE"] + E
    assert A[k * g["t"] + t, col] == pytest.approx(tot, rel=1e-13)


def test_product_macs_table2():
    """Per-product multiply-adds reproduce Table 2's two-layer terms:
    l*(2 b d D^6 + a b D^4 + kL a D^4) for a uniform bond D, t = h = D^2."""
    rng = np.random.default_rng(3)
    D, d, m, ell = 3, 2, 4, 6
    op = make_op(rng, kL=m, t=D * D, a=m, b=m, d=d, D=(D,) * 4, DB=(D,) * 4, cplx=False)
    assert op.product_macs(ell) == ell * (2 * m * d * D ** 6 + m * m * D ** 4 + m * m * D ** 4)


def test_orthogonalize_rank_deficient():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((30, 3)) + 1j * rng.standard_normal((30, 3))
    Y = B @ (rng.standard_normal((3, 6)) + 0j)
    Q = orthogonalize(Y, 1e-12)
    nz = np.linalg.norm(Q, axis=0) > 0.5
    assert nz.sum() == 3
    Qn = Q[:, nz]
    np.testing.assert_allclose(Qn.conj().T @ Qn, np.eye(3), atol=1e-13)
    # same range as Y
    np.testing.assert_allclose(Qn @ (Qn.conj().T @ Y), Y, atol=1e-11)


@pytest.mark.parametrize("cplx", [False, True])
def test_exact_regime_equals_dense_svd(cplx):
    """l >= rank(A): Algorithm 4 returns the truncated SVD exactly."""
    rng = np.random.default_rng(5)
    op = make_op(rng, kL=2, t=4, a=3, b=2, d=2, cplx=cplx)   # M = 8
    A = op.dense()
    k, ell = block_sizes(6, 4, op.M, op.N)
    assert ell == op.M
    om = philox.sketch(op.N, ell, 3, 1, cplx)
    P, Ut, s, Vh = rsvd_implicit(op, k, ell, 1, om, 1e-13)
    sref = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(s, sref[:k], rtol=1e-12)
    Ur, sr, Vr = np.linalg.svd(A, full_matrices=False)
    Ak = (Ur[:, :k] * sr[:k]) @ Vr[:k]
    np.testing.assert_allclose((P @ Ut) @ (s[:, None] * Vh), Ak, atol=1e-11 * sr[0])


def test_interlacing_eckart_young_and_power_iterations():
    rng = np.random.default_rng(6)
    op = make_op(rng, kL=4, t=9, a=6, b=5, d=2, D=(3, 3, 3, 3), DB=(3, 3, 3, 3))
    A = op.dense()
    sref = np.linalg.svd(A, compute_uv=False)
    k, ell = block_sizes(10, 4, op.M, op.N)
    tail = np.sqrt(np.sum(sref[k:] ** 2))
    errs = []
    for q in (0, 1, 3):
        om = philox.sketch(op.N, ell, 11, 2, True)
        P, Ut, s, Vh = rsvd_implicit(op, k, ell, q, om, 1e-13)
        # P orthonormal
        np.testing.assert_allclose(P.conj().T @ P, np.eye(ell), atol=1e-13)
        # Ritz values interlace: sigma_i(P^H A) <= sigma_i(A)
        assert np.all(s <= sref[:k] * (1 + 1e-12))
        err = np.linalg.norm(A - (P @ Ut) @ (s[:, None] * Vh))
        assert err >= tail * (1 - 1e-12)          # Eckart-Young
        errs.append(err)
    assert errs[2] <= errs[0]
    assert errs[2] <= tail * 1.05                 # converges to the optimum


def test_einsumsvd_gauge_scale_and_shapes():
    rng = np.random.default_rng(7)
    op = make_op(rng, kL=3, t=4, a=5, b=3, d=2)
    U, W, s, l1 = einsumsvd(op.V, op.S, op.K, op.Kb, 4, 2, 2, 5, 9)
    k = 4
    assert U.shape == (3, 4, k) and W.shape == (k, 4, 3, 4)
    g = philox.gauge_vector(op.M, 5, 9, True)
    phi = g.conj() @ U.reshape(op.M, k)
    assert np.all(np.abs(phi.imag) < 1e-12) and np.all(phi.real > 0)
    assert np.linalg.norm(W.reshape(k, -1)[0]) == pytest.approx(1.0, rel=1e-12)
    # scale equivariance: A -> c A shifts log sigma_1 by log|c|, factors unchanged
    U2, W2, s2, l2 = einsumsvd(op.V * 3.0, op.S, op.K, op.Kb, 4, 2, 2, 5, 9)
    assert l2 - l1 == pytest.approx(np.log(3.0), abs=1e-12)
    np.testing.assert_allclose(U2, U, atol=1e-11)
    np.testing.assert_allclose(W2, W, atol=1e-11)
    np.testing.assert_allclose(s2, 3 * s, rtol=1e-11)
