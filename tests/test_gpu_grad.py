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


# ---- energy gradient through the whole network (peps_grad) ----

from oracle import expectation, grad  # noqa: E402
from tests.gpu_util import to_dev  # noqa: E402


@pytest.mark.parametrize("dtype,shape,D,m,dist,tol", [
    ("f64", (3, 3), 2, 3, "normal", 1e-6),
    ("f32", (3, 4), 2, 4, "normal", 1e-4),
])
def test_energy_gradient_small(dtype, shape, D, m, dist, tol):
    """Truncated environments (m below the exact boundary bond): E and dE/d(site)
    against the oracle's energy and its central differences along random
    directions."""
    nr, nc = shape
    ket = synth.random_peps(nr, nc, 2, D, dtype, dist, 5)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    p, q, seed = 2, 1, 9
    e, g = libpeps.energy_grad(to_dev(ket, dtype), terms, m, p, q, seed)
    ref = expectation.energy(ket, terms, m, p, q, seed)
    assert abs(e - ref) <= (1e-10 if dtype == "f64" else 1e-5) * max(1.0, abs(ref)), (e, ref)
    g = [[x.cpu().numpy().astype(np.float64) for x in row] for row in g]
    rng = np.random.default_rng(3)
    for trial in range(2):
        dirs = [[rng.standard_normal(T.shape) for T in row] for row in ket]
        fd = grad.fd_directional(ket, terms, dirs, m, p, q, seed)
        ad = sum(np.sum(g[a][b] * dirs[a][b]) for a in range(nr) for b in range(nc))
        assert abs(ad - fd) <= tol * max(1.0, abs(fd)), (trial, ad, fd)


def test_c4_energy_gradient():
    """The 6 x 6 transverse-field Ising workload (D = 3, m = 18, real).

    The energy as computed (truncated environments, fixed sketches) is smooth
    only on a small neighbourhood of these sites: a central difference with
    step 1e-5 crosses a kink (a gauge / ordering decision of a near-degenerate
    truncation: the difference quotient jumps to -127), and step 1e-6 is
    still contaminated at 1e-4.  The FD reference therefore uses step 1e-7.
      * FP64 network: directional derivatives within 1e-5 of the FP64 oracle's
        central differences (measured 1.1e-6);
      * FP32 network (the workload's precision): energy within 1e-5 and the
        whole gradient within 1e-4 normwise of the FD-checked FP64 gradient
        (measured 5.5e-5)."""
    cfg = synth.config("c4")
    ket = synth.peps_for(cfg)
    terms = synth.tfi_terms(cfg.nrow, cfg.ncol, cfg.extra["J"], cfg.extra["h"])
    args = (cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    e64, g64 = libpeps.energy_grad(to_dev(ket, "f64"), terms, *args)
    e32, g32 = libpeps.energy_grad(to_dev(ket, "f32"), terms, *args)
    ref = expectation.energy(ket, terms, *args)
    assert abs(e64 - ref) <= 1e-10 * abs(ref), (e64, ref)
    assert abs(e32 - ref) <= 1e-5 * abs(ref), (e32, ref)
    g64 = [[x.cpu().numpy() for x in row] for row in g64]
    g32 = [[x.cpu().numpy().astype(np.float64) for x in row] for row in g32]
    rng = np.random.default_rng(4)
    for trial in range(2):
        dirs = [[rng.standard_normal(T.shape) for T in row] for row in ket]
        fd = grad.fd_directional(ket, terms, dirs, *args, h=1e-7)
        ad = sum(np.sum(g64[a][b] * dirs[a][b]) for a in range(cfg.nrow) for b in range(cfg.ncol))
        assert abs(ad - fd) <= 1e-5 * max(1.0, abs(fd)), (trial, ad, fd)
    num = np.sqrt(sum(np.sum((g32[a][b] - g64[a][b]) ** 2) for a in range(cfg.nrow) for b in range(cfg.ncol)))
    den = np.sqrt(sum(np.sum(g64[a][b] ** 2) for a in range(cfg.nrow) for b in range(cfg.ncol)))
    assert num <= 1e-4 * den, num / den


def test_autograd_function_backward():
    """The torch.autograd entry gives peps_grad's gradient, scaled by the
    incoming cotangent."""
    ket = synth.random_peps(3, 3, 2, 2, "f64", "normal", 8)
    terms = synth.tfi_terms(3, 3, 1.0, 3.0)
    k = to_dev(ket, "f64")
    flat = [t.clone().requires_grad_(True) for row in k for t in row]
    E = libpeps.peps_energy(terms, 3, 2, 1, 9, 3, 3, *flat)
    (2.5 * E).backward()
    e, g = libpeps.energy_grad(k, terms, 3, 2, 1, 9)
    assert float(E) == pytest.approx(e, abs=1e-12)
    for x, gr in zip(flat, [t for row in g for t in row]):
        assert torch.allclose(x.grad, 2.5 * gr, rtol=1e-12, atol=1e-14)


def test_autograd_function_forward_only():
    """With no input requiring a gradient the autograd entry runs the
    expectation value alone (no reverse sweep) and returns the same energy."""
    ket = synth.random_peps(3, 3, 2, 2, "f64", "normal", 8)
    terms = synth.tfi_terms(3, 3, 1.0, 3.0)
    k = to_dev(ket, "f64")
    flat = [t for row in k for t in row]
    with torch.no_grad():
        E = libpeps.peps_energy(terms, 3, 2, 1, 9, 3, 3, *flat)
    e, _ = libpeps.energy_grad(k, terms, 3, 2, 1, 9)
    assert not E.requires_grad
    assert float(E) == pytest.approx(e, abs=1e-12)
