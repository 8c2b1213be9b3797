"""GPU parity of the boundary-MPS contraction (Algorithms 2-4) through the
C ABI against the CPU oracle on identical seeded inputs.

Tolerances: FP64 data, 1e-9 on log|v| (the FP64 path reproduces the oracle up
to rounding order); single-precision data, 1e-5 relative on log|v|.  The
singular values of every step of a whole sweep are compared normwise
(against sigma_1) at SWEEP_SIGMA_TOL = 1e-4: a step's inputs (the boundary
left by earlier rows) already differ from the oracle's by single-precision
rounding, and truncating at a flat spectrum amplifies such differences (the
FP64 oracle moves late-row singular values by up to 5e-6 when its inputs are
perturbed by 1e-7 relative).  With identical inputs a single einsumsvd step
matches at 1e-5 (tests/test_gpu_einsumsvd.py; measured ~2e-7).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import bmps, bruteforce
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import sigma_errors, to_dev

pytestmark = pytest.mark.gpu

SWEEP_SIGMA_TOL = 1e-4


def _run(ket, bra, dtype, m, p, q, seed, **kw):
    kt = to_dev(ket, dtype)
    bt = None if bra is None else (kt if bra is ket else to_dev(bra, dtype))
    return libpeps.boundary_contract(kt, bt, m, p, q, seed, with_sigma=True, **kw)


def test_c1_one_layer_fp64_matches_oracle_and_bruteforce():
    cfg = synth.config("c1")
    ket = synth.peps_for(cfg)
    rec = []
    la, ph, sig = _run(ket, None, "f64", cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    ra, rp = bmps.contract(ket, None, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec)
    ex = bruteforce.exact_scalar(ket, None)
    assert la == pytest.approx(ra, abs=1e-9)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-9)
    assert np.cos(ph) == pytest.approx(np.sign(ex), abs=1e-9)
    assert sigma_errors(sig, rec).max() < 1e-10


@pytest.mark.parametrize("shape,D,m,dtype", [((3, 3), 2, 16, "c128"), ((3, 5), 2, 64, "c128"),
                                             ((2, 4), 2, 16, "f64")])
def test_two_layer_exact_regime_fp64(shape, D, m, dtype):
    nr, nc = shape
    dist = "cgauss_scaled" if dtype.startswith("c") else "normal"
    ket = synth.random_peps(nr, nc, 2, D, "c64" if dtype.startswith("c") else "f64", dist, 31)
    la, ph, _ = _run(ket, ket, dtype, m, 8, 1, 77)
    ex = bruteforce.exact_scalar(ket, ket)
    assert la == pytest.approx(np.log(abs(ex)), abs=1e-9)
    assert abs(np.sin(ph)) < 1e-9


@pytest.mark.parametrize("shape,D,m,p,q", [((4, 4), 3, 6, 4, 2), ((5, 3), 2, 5, 3, 1),
                                           ((3, 6), 3, 9, 2, 0)])
def test_two_layer_truncated_complex64(shape, D, m, p, q):
    nr, nc = shape
    ket = synth.random_peps(nr, nc, 2, D, "c64", "cgauss_scaled", 101 + nr)
    rec = []
    la, ph, sig = _run(ket, ket, "c64", m, p, q, 5)
    ra, rp = bmps.contract(ket, ket, m, p, q, 5, record=rec)
    assert abs(la - ra) <= 1e-5 * abs(ra)
    assert sigma_errors(sig, rec).max() <= SWEEP_SIGMA_TOL


def test_c2_norm_8x8_complex64():
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    rec = []
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec)
    assert abs(la - ra) <= 1e-5 * abs(ra)
    assert sigma_errors(sig, rec).max() <= SWEEP_SIGMA_TOL


def test_real_f32_norm_6x6_and_uniform_sketch():
    cfg = synth.config("c4")
    ket = synth.peps_for(cfg)
    for sketch, kind in ((libpeps.SKETCH_GAUSS, "gauss"), (libpeps.SKETCH_UNIFORM, "uniform")):
        rec = []
        la, ph, sig = _run(ket, ket, "f32", cfg.m, cfg.p, cfg.q, cfg.omega_seed, sketch=sketch)
        ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, sketch_kind=kind,
                               record=rec)
        assert abs(la - ra) <= 1e-5 * abs(ra)
        assert sigma_errors(sig, rec).max() <= SWEEP_SIGMA_TOL


def test_direction_changes_streams_and_replay_is_deterministic():
    ket = synth.random_peps(4, 4, 2, 2, "c64", "cgauss_scaled", 3)
    kt = to_dev(ket, "c64")
    opts = libpeps.make_opts(3, 2, 1, 9)
    plan = libpeps.ContractPlan(kt, kt, opts, direction=1)
    plan.execute()
    a = plan.result(with_sigma=True)
    plan.execute()
    b = plan.result(with_sigma=True)
    assert a[0] == b[0] and np.array_equal(a[2], b[2])
    ra, _ = bmps.contract(ket, ket, 3, 2, 1, 9, direction=1)
    assert abs(a[0] - ra) <= 1e-5 * abs(ra)


def test_single_row_and_single_column():
    for shape in ((1, 4), (4, 1)):
        ket = synth.random_peps(*shape, 2, 2, "c64", "cgauss_scaled", 17)
        la, _, _ = _run(ket, ket, "c128", 4, 2, 1, 3)
        ex = bruteforce.exact_scalar(ket, ket)
        assert la == pytest.approx(np.log(abs(ex)), abs=1e-9)


def test_c2_mixed_precision():
    """Tensor-core products: the log-norm stays within 1e-5 of the FP64
    oracle and the first row's einsumsvd steps (identical inputs) keep their
    singular values within 1e-5 normwise."""
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    rec = []
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=libpeps.PREC_MIXED)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec)
    assert abs(la - ra) <= 1e-5 * abs(ra)
    errs = sigma_errors(sig, rec)
    row1 = [i for i, r in enumerate(rec) if r["row"] == 1]
    assert errs[row1].max() <= 1e-5


def test_c2_fast_precision_log_norm():
    """PEPS_PREC_FAST (plain TF32 for the early power-iteration products): the
    contracted scalar stays within 1e-5 of the FP64 oracle."""
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=libpeps.PREC_FAST)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    assert abs(la - ra) <= 1e-5 * abs(ra)


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_c2_fp64_small_factorisations(prec):
    """PEPS_FLAG_FP64_SMALL (CholeskyQR2's Cholesky factorisations and the
    Jacobi SVD in FP64 on single-precision data): the 8x8 log-norm stays
    within 1e-5 of the FP64 oracle and the first row's steps (identical
    inputs) keep their singular values within 1e-5 normwise."""
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    rec = []
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec,
                       flags=libpeps.FLAG_FP64_SMALL)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec)
    assert abs(la - ra) <= 1e-5 * abs(ra)
    errs = sigma_errors(sig, rec)
    row1 = [i for i, r in enumerate(rec) if r["row"] == 1]
    assert errs[row1].max() <= 1e-5
