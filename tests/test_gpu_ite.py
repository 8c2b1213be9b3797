"""Imaginary-time evolution on the GPU (Sec. II-D) against the oracle:
  * one TEBD layer with a different two-site operator on every bond and a
    one-site operator on every site (Eq. 4), normalised bonds or not, site
    for site against oracle.qrsvd.tebd_layer (FP64 1e-10, single precision
    1e-4: the bars of the plain TEBD layer);
  * ITE steps (layer of exp(-tau H_j), then the Rayleigh quotient by Eq. 6)
    of the transverse-field Ising model against oracle.ite.ite: every step's
    energy within 1e-9 (FP64) / 1e-6 (FP32; measured 3e-8) relative, and the
    final sites within 1e-9 / 1e-5 (measured 3e-7) after four steps."""
import numpy as np
import pytest
import torch

import synth
from oracle import ite, qrsvd
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _rand(rng, shape, cplx):
    x = rng.standard_normal(shape)
    return x + 1j * rng.standard_normal(shape) if cplx else x


def _round(a, dtype):
    if dtype == "c64":
        return a.astype(np.complex64).astype(np.complex128)
    if dtype == "f32":
        return a.astype(np.float32).astype(np.float64)
    return a


def _worst(k, ref):
    return max(np.linalg.norm(k[p][q].cpu().numpy() - ref[p][q]) / np.linalg.norm(ref[p][q])
               for p in range(len(ref)) for q in range(len(ref[0])))


@pytest.mark.parametrize("shape,D,dtype,tol,unit", [((3, 3), 2, "c128", 1e-10, False),
                                                    ((4, 3), 3, "f64", 1e-10, True),
                                                    ((3, 4), 2, "c64", 1e-4, True),
                                                    ((4, 4), 3, "f32", 1e-4, False)])
def test_per_bond_and_site_operators_match_oracle(shape, D, dtype, tol, unit):
    nr, nc = shape
    cplx = dtype.startswith("c")
    rng = np.random.default_rng(5 + nr + D)
    ket = synth.random_peps(nr, nc, 2, D, "c64" if cplx else "f64", "cgauss_scaled" if cplx else "normal", 3 + D)
    ket = [[_round(np.asarray(T), dtype) for T in row] for row in ket]
    nb = nr * (nc - 1) + (nr - 1) * nc
    gates = [_round(_rand(rng, (4, 4), cplx), dtype) for _ in range(nb)]
    sops = [_round(_rand(rng, (2, 2), cplx), dtype) for _ in range(nr * nc)]
    ref, _ = qrsvd.tebd_layer(ket, gates, D, 13, unit=unit, site_gates=sops)
    k = to_dev(ket, dtype)
    libpeps.tebd_layer(k, gates, 13, unit=unit, site_gates=sops)
    torch.cuda.synchronize()
    worst = _worst(k, ref)
    print(f"{shape} D={D} {dtype} unit={unit}: worst site error {worst:.2e}")
    assert worst <= tol


@pytest.mark.parametrize("dtype,etol,stol", [("c128", 1e-9, 1e-9), ("f32", 1e-6, 1e-5)])
def test_ite_energies_match_oracle(dtype, etol, stol):
    nr, nc, D = 3, 3, 2
    cplx = dtype.startswith("c")
    ket = synth.random_peps(nr, nc, 2, D, "c64" if cplx else "f64", "cgauss_scaled" if cplx else "normal", 71)
    ket = [[_round(np.asarray(T), dtype) for T in row] for row in ket]
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    Gb, Gs = synth.tfi_ite_gates(1.0, 3.0, 0.1)
    Gb, Gs = _round(Gb, dtype), _round(Gs, dtype)
    m, p, q, sseed, seed, steps = 16, 8, 2, 9, 5, 4
    ref_sites, ref_e = ite.ite(ket, Gb, Gs, D, seed, steps, terms, m, p, q, sseed)
    k = to_dev(ket, dtype)
    drv = libpeps.IteDriver(k, Gb, Gs, terms, libpeps.make_opts(m, p, q, sseed), seed)
    got = drv.run(steps)
    rel = [abs(a - b) / abs(b) for a, b in zip(got, ref_e)]
    print(f"ITE {dtype}: energies {got}, oracle {ref_e}, worst relative {max(rel):.2e}")
    assert max(rel) <= etol
    assert got[-1] < got[0]
    worst = _worst(k, ref_sites)
    print(f"ITE {dtype}: worst final site error {worst:.2e}")
    assert worst <= stol


def test_captured_ite_step_replays_the_eager_steps():
    """One ITE step captured as a CUDA graph (both plans, the expectation's
    sweeps on parallel branches) and replayed gives the eager steps' energies
    and sites."""
    nr, nc, D = 3, 4, 2
    ket = synth.random_peps(nr, nc, 2, D, "c64", "cgauss_scaled", 73)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    Gb, Gs = synth.tfi_ite_gates(1.0, 3.0, 0.1)
    opts = libpeps.make_opts(16, 8, 2, 9)
    k1, k2 = to_dev(ket, "c128"), to_dev(ket, "c128")
    eager = libpeps.IteDriver(k1, Gb, Gs, terms, opts, 5).run(4)
    drv = libpeps.IteDriver(k2, Gb, Gs, terms, opts, 5)
    first = drv.run(1)
    drv.capture()                     # the second step
    got = first + [drv.expect.result()[0]] + drv.run(2)
    assert np.allclose(got, eager, rtol=1e-12, atol=0)
    assert _worst(k2, [[T.cpu().numpy() for T in row] for row in k1]) <= 1e-12
