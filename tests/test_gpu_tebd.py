"""One TEBD layer (Algorithm 1 on every bond) on the GPU against the oracle's
tebd_layer on identical inputs: every updated site tensor, normwise relative
1e-10 in FP64 and 1e-4 in single precision (CholeskyQR2 and the gate
contraction in single precision, the small SVD in FP64; the bar leaves
room for singular vectors of close singular values), real and complex, and
the identity gate leaving the state's amplitudes unchanged."""
import numpy as np
import pytest
import torch

import synth
from oracle import bruteforce, qrsvd
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _gate(seed, cplx):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((4, 4))
    if cplx:
        g = g + 1j * rng.standard_normal((4, 4))
    return g


@pytest.mark.parametrize("shape,D,dtype,tol", [((3, 3), 2, "c128", 1e-10), ((5, 3), 2, "f64", 1e-10),
                                               ((4, 4), 3, "c64", 1e-4), ((3, 5), 4, "f32", 1e-4),
                                               ((6, 6), 4, "c64", 1e-4)])
def test_tebd_layer_matches_oracle(shape, D, dtype, tol):
    nr, nc = shape
    cplx = dtype.startswith("c")
    store = "c64" if cplx else ("f64" if dtype == "f64" else "f32")
    ket = synth.random_peps(nr, nc, 2, D, "c64" if cplx else "f64", "cgauss_scaled" if cplx else "normal", 7 + D)
    ket = [[synth.round_to(T, store if dtype in ("c64", "f32") else ("c128" if cplx else "f64")) for T in row]
           for row in ket]
    G = _gate(3 + nr, cplx)
    if dtype == "f32":
        G = G.astype(np.float32).astype(np.float64)
    elif dtype == "c64":
        G = G.astype(np.complex64).astype(np.complex128)
    ref, _ = qrsvd.tebd_layer(ket, G, D, 11)
    k = to_dev(ket, dtype)
    libpeps.tebd_layer(k, G, 11)
    torch.cuda.synchronize()
    worst = 0.0
    for p in range(nr):
        for q in range(nc):
            got = k[p][q].cpu().numpy()
            r = ref[p][q]
            assert got.shape == r.shape
            worst = max(worst, np.linalg.norm(got - r) / np.linalg.norm(r))
    print(f"{shape} D={D} {dtype}: worst site error {worst:.2e}")
    assert worst <= tol


def test_identity_gate_keeps_amplitudes():
    ket = synth.random_peps(3, 3, 2, 2, "c64", "cgauss_scaled", 5)
    k = to_dev(ket, "c128")
    libpeps.tebd_layer(k, np.eye(4), 1)
    new = [[T.cpu().numpy() for T in row] for row in k]
    a = bruteforce.statevector(ket).reshape(-1)
    b = bruteforce.statevector(new).reshape(-1)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


def test_status_word_of_the_layer():
    """A clean layer leaves the plan's status word at zero; a NaN in one site
    tensor sets STATUS_NONFINITE (the layer has no result call: peps_poll is
    its report)."""
    ket = synth.random_peps(3, 3, 2, 2, "c64", "cgauss_scaled", 5)
    k = to_dev(ket, "c64")
    plan = libpeps.TebdPlan(k, np.eye(4), 1)
    plan.execute()
    r, word = plan.poll()
    assert r == 0 and word == 0
    k[1][1][0, 0, 0, 0, 0] = float("nan")
    plan.execute()
    r, word = plan.poll()
    assert word & libpeps.STATUS_NONFINITE
