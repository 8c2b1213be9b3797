"""The einsumsvd adjoint on the GPU against central finite differences of the
FP64 oracle's einsumsvd (the sketch held fixed): directional derivatives of
    L = <U_bar, U> + <W_bar, W> + l_bar log sigma_1
along random directions in all four operands (V, S, ket, bra)."""
import numpy as np
import pytest
import torch

import synth
from oracle import rsvd
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import TORCH_DT, tensor

pytestmark = pytest.mark.gpu


def _case(rng, kL, t, a, b, d, D, dtype):
    R = D * D

    def r(shape):
        return synth.round_to(rng.standard_normal(shape), dtype)
    return r((kL, t, a, R)), r((a, R, b)), r((d, D, D, D, D)), r((d, D, D, D, D))


def _loss(ops, Ub, Wb, lb, m, p, q, seed):
    U, W, s, l1 = rsvd.einsumsvd(*ops, m, p, q, seed, 0)
    return np.sum(Ub * U) + np.sum(Wb * W) + lb * l1


@pytest.mark.parametrize("dtype,shape,m,q,tol", [
    ("f64", (3, 4, 5, 3, 2, 2), 4, 1, 1e-6),
    ("f32", (3, 4, 5, 3, 2, 2), 4, 1, 1e-4),
    ("f64", (6, 9, 7, 5, 2, 3), 9, 2, 1e-6),
    # a middle step of the 6 x 6, D = 3, m = 18 sweep: l = 26 singular values whose close pairs
    # enter the SVD adjoint as 1 / (s_j^2 - s_i^2); the single-precision forward (bases,
    # Jacobi vectors) moves the directional derivatives by up to ~1.2e-4 relative
    ("f32", (18, 9, 18, 18, 2, 3), 18, 2, 2e-4),
])
def test_einsumsvd_adjoint_matches_finite_differences(dtype, shape, m, q, tol):
    rng = np.random.default_rng(11)
    kL, t, a, b, d, D = shape
    ops = _case(rng, kL, t, a, b, d, D, dtype)
    p, seed = 4, 7
    U, W, s, l1 = rsvd.einsumsvd(*ops, m, p, q, seed, 0)
    Ub = rng.standard_normal(U.shape)
    Wb = rng.standard_normal(W.shape)
    lb = 0.3
    dev = [tensor(x, dtype) for x in ops]
    (gU, gW, gs, gl), grads = libpeps.einsumsvd_grad(*dev, m, p, q, seed, tensor(Ub, dtype), tensor(Wb, dtype), lb)
    # forward parity first
    assert np.max(np.abs(gs.cpu().numpy() - s)) <= (1e-10 if dtype == "f64" else 1e-5) * s[0]
    g = [x.cpu().numpy().astype(np.float64) for x in grads]
    for trial in range(3):
        dirs = [rng.standard_normal(x.shape) for x in ops]
        eps = 1e-6
        plus = [x + eps * dx for x, dx in zip(ops, dirs)]
        minus = [x - eps * dx for x, dx in zip(ops, dirs)]
        fd = (_loss(plus, Ub, Wb, lb, m, p, q, seed) - _loss(minus, Ub, Wb, lb, m, p, q, seed)) / (2 * eps)
        ad = sum(np.sum(gx * dx) for gx, dx in zip(g, dirs))
        assert abs(ad - fd) <= tol * max(1.0, abs(fd)), (trial, ad, fd)
