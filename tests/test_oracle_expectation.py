"""Pins of the oracle's cached-environment expectation (Eq. 6, Sec. IV-B) and
of its finite-difference gradient.

Product states have a closed form; in the exact regime the energy must equal
the dense state-vector Rayleigh quotient, and the finite-difference gradient
must equal torch autograd through that dense energy (a library routine).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import bruteforce, expectation, grad


def test_product_state_closed_form():
    ket = synth.random_peps(3, 3, 2, 1, "c64", "cgauss_scaled", 3)
    terms = synth.tfi_terms(3, 3, 1.0, 3.0)
    e = expectation.energy(ket, terms, 2, 2, 1, 5)
    z, x = {}, {}
    for p in range(3):
        for q in range(3):
            v = ket[p][q].reshape(2)
            n = np.vdot(v, v).real
            z[p, q] = (abs(v[0]) ** 2 - abs(v[1]) ** 2) / n
            x[p, q] = 2 * np.real(np.conj(v[0]) * v[1]) / n
    ref = 0.0
    for sites, op, c in terms:
        if len(sites) == 2:
            ref += c * z[sites[0]] * z[sites[1]]
        else:
            ref += c * x[sites[0]]
    assert e == pytest.approx(ref, abs=1e-12)


@pytest.mark.parametrize("shape,dtype", [((3, 3), "c64"), ((2, 3), "f32"), ((3, 2), "f32")])
def test_exact_regime_equals_statevector(shape, dtype):
    nr, nc = shape
    dist = "cgauss_scaled" if dtype == "c64" else "normal"
    ket = synth.random_peps(nr, nc, 2, 2, dtype, dist, 17)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    e, per = expectation.energy(ket, terms, 16, 4, 1, 2, return_terms=True)
    ref = bruteforce.statevector_energy(ket, terms)
    assert e == pytest.approx(ref, abs=1e-10)
    # per-term values against the state vector as well
    psi = bruteforce.statevector(ket)
    norm = np.vdot(psi, psi)
    for (sites, op, c), val in zip(terms[:4], per[:4]):
        one = bruteforce.statevector_energy(ket, [(sites, op, c)])
        assert val == pytest.approx(one, abs=1e-10)


def test_operator_schmidt_roundtrip():
    rng = np.random.default_rng(0)
    op = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    comps = expectation.operator_schmidt(op, 2)
    rebuilt = sum(np.kron(A, B) for A, B in comps)
    np.testing.assert_allclose(rebuilt, op, atol=1e-12)


def _torch_energy(tensors, shape, terms):
    nr, nc = shape
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    it = iter(letters)
    phys = {(p, q): next(it) for p in range(nr) for q in range(nc)}
    hb = {(p, q): next(it) for p in range(nr) for q in range(nc - 1)}
    vb = {(p, q): next(it) for p in range(nr - 1) for q in range(nc)}
    subs, ops = [], []
    for p in range(nr):
        for q in range(nc):
            T = tensors[p * nc + q]
            idx, shp = phys[p, q], [T.shape[0]]
            if q > 0:
                idx += hb[p, q - 1]; shp.append(T.shape[1])
            if p > 0:
                idx += vb[p - 1, q]; shp.append(T.shape[2])
            if p < nr - 1:
                idx += vb[p, q]; shp.append(T.shape[3])
            if q < nc - 1:
                idx += hb[p, q]; shp.append(T.shape[4])
            subs.append(idx)
            ops.append(T.reshape(shp))
    out = "".join(phys[p, q] for p in range(nr) for q in range(nc))
    psi = torch.einsum(",".join(subs) + "->" + out, *ops)
    num = 0.0
    for sites, op, c in terms:
        axes = [p * nc + q for (p, q) in sites]
        n = len(axes)
        O = torch.tensor(np.real(op), dtype=torch.float64).reshape([2] * (2 * n))
        phi = torch.tensordot(O, psi, dims=(list(range(n, 2 * n)), axes))
        phi = torch.movedim(phi, list(range(n)), axes)
        num = num + c * torch.sum(psi * phi)
    return num / torch.sum(psi * psi)


def test_fd_gradient_equals_autograd_exact_regime():
    nr, nc = 2, 3
    ket = synth.random_peps(nr, nc, 2, 2, "f32", "normal", 23)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    ts = [torch.tensor(ket[p][q], dtype=torch.float64, requires_grad=True)
          for p in range(nr) for q in range(nc)]
    e = _torch_energy(ts, (nr, nc), terms)
    e.backward()
    assert float(e.detach()) == pytest.approx(expectation.energy(ket, terms, 16, 4, 1, 2), abs=1e-10)
    rng = np.random.default_rng(1)
    for _ in range(6):
        p, q = int(rng.integers(nr)), int(rng.integers(nc))
        idx = tuple(int(rng.integers(s)) for s in ket[p][q].shape)
        fd = grad.fd_entry(ket, terms, (p, q), idx, 16, 4, 1, 2)
        ag = float(ts[p * nc + q].grad[idx])
        assert fd == pytest.approx(ag, rel=1e-5, abs=1e-7)
