"""GPU parity of the boundary-MPS contraction (Algorithms 2-4) through the
C ABI against the CPU oracle on identical seeded inputs.

Tolerances: FP64 data, 1e-9 on log|v| (the FP64 path reproduces the oracle up
to rounding order); single-precision data, 1e-5 relative on log|v|.

Singular values of a whole single-precision sweep: a step's inputs (the
boundary left by earlier rows) already differ from the oracle's by rounding,
and truncation at a flat spectrum amplifies such differences row by row.  The
8 x 8 norm workload's bar is therefore per row, from the oracle replayed in
emulated single precision (tests/golden/make_c2_envelope.py: products,
sketch, QR and small SVD in complex64, every step's U and W rounded, four
rounding realizations): every step of row r is held to SWEEP_ENVELOPE_FACTOR
times the largest envelope of rows 1..r.  Measured on the GPU: at most 2.1 times
the envelope on the plain and mixed paths, with and without FP64 small
factorisations.  The smaller workloads below keep SWEEP_SIGMA_TOL = 1e-4, the
largest row envelope of the 8 x 8 sweep (4.5e-5) with room for their own
rows.  A row's envelope is taken cumulatively over the rows above it.  With identical inputs a single einsumsvd step matches at 1e-5
(tests/test_gpu_einsumsvd.py; measured ~2e-7).
"""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import bmps, bruteforce
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import sigma_errors, to_dev

pytestmark = pytest.mark.gpu

SWEEP_SIGMA_TOL = 1e-4
SWEEP_ENVELOPE_FACTOR = 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _row_bars(name):
    """Per-step bar of the 8 x 8 sweep: the factor times the envelope of its
    row, taken cumulatively over the rows above it (a row inherits all their
    rounding; a smaller maximum in a later row is the sampling of four
    realizations, not a smaller sensitivity)."""
    env = json.load(open(os.path.join(GOLDEN, name)))
    rows = np.array([s["row"] for s in env["steps"]])
    e = np.array([s["envelope"] for s in env["steps"]])
    per_row = np.maximum.accumulate([e[rows == r].max() for r in range(1, rows.max() + 1)])
    return SWEEP_ENVELOPE_FACTOR * per_row[rows - 1], rows, env


def _c2_row_bars():
    bars, _, env = _row_bars("c2_envelope.json")
    return bars, env


def _c2_against_golden(sig, la, prec_name):
    """Every step's singular values against the stored FP64 sweep and the
    log-norm: relative 1e-5 on log|v|, and |d log v| within ten times the
    largest single-precision replay's (reported with the relative error on v)."""
    gold = json.load(open(os.path.join(GOLDEN, "c2_sweep.json")))
    bars, env = _c2_row_bars()
    pos, errs = 0, []
    for st in gold["steps"]:
        ref = np.asarray(st["sigma"])
        errs.append(np.max(np.abs(sig[pos:pos + len(ref)] - ref)) / ref[0])
        pos += len(ref)
    errs = np.array(errs)
    bad = [(gold["steps"][i]["row"], gold["steps"][i]["col"], "%.2e > %.2e" % (errs[i], bars[i]))
           for i in np.nonzero(errs > bars)[0]]
    assert not bad, (prec_name, bad)
    dlog = abs(la - gold["log_norm"])
    print(f"{prec_name}: max step sigma error {errs.max():.2e}, |d log v| {dlog:.2e} "
          f"(relative on v {np.expm1(dlog):.2e}, on log v {dlog / abs(gold['log_norm']):.2e})")
    assert dlog <= 1e-5 * abs(gold["log_norm"])
    assert dlog <= 10 * max(abs(x) for x in env["dlog"])


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


def test_one_layer_8x8_truncated_matches_oracle():
    """One-layer zip-up with truncation (the contraction bond equal to the
    initial bond, D = m = 4, 8 x 8 without physical index) against the oracle:
    every step's singular values and log|v| in FP64; the single-precision
    mixed path of the same network within 1e-5 relative on log|v|."""
    ket = synth.random_peps(8, 8, 1, 4, "f64", "normal_half", 91)
    rec = []
    la, ph, sig = _run(ket, None, "f64", 4, 4, 2, 13)
    ra, rp = bmps.contract(ket, None, 4, 4, 2, 13, record=rec)
    assert la == pytest.approx(ra, abs=1e-9 * max(1.0, abs(ra)))
    assert sigma_errors(sig, rec).max() < 1e-10
    lm, _, _ = _run(ket, None, "f32", 4, 4, 2, 13, prec=libpeps.PREC_MIXED)
    assert abs(lm - ra) <= 1e-5 * abs(ra)


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


@pytest.mark.parametrize("prec,flags", [(libpeps.PREC_PLAIN, 0), (libpeps.PREC_MIXED, 0),
                                        (libpeps.PREC_PLAIN, libpeps.FLAG_FP64_SMALL),
                                        (libpeps.PREC_MIXED, libpeps.FLAG_FP64_SMALL)])
def test_c2_norm_8x8_complex64_every_step(prec, flags):
    """The 8 x 8 norm on every path against the stored FP64 sweep: every
    step of every row at the row's envelope bar, and the log-norm."""
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec, flags=flags)
    _c2_against_golden(sig, la, f"prec {prec} flags {flags}")


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


def test_c2_fast_precision_log_norm():
    """PEPS_PREC_FAST (plain TF32 for the early power-iteration products): the
    contracted scalar stays within 1e-5 of the FP64 oracle."""
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=libpeps.PREC_FAST)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    assert abs(la - ra) <= 1e-5 * abs(ra)


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_alternating_canonicalisation(prec):
    """PEPS_FLAG_ALTERNATE (Sigma into the finished site on even rows,
    Sec. III-A) against the oracle's alternating sweep: the exact regime in
    FP64 against brute force, and the truncated 8 x 8 workload in complex64:
    log-norm at 1e-5 relative on log|v|, every step's singular values at 3x
    its row's single-precision envelope (tests/golden/
    c2_envelope_alternate.json: the carry V^H gives the small singular
    directions unit weight, so rounding moves late rows far more than in the
    default sweep, up to 8.5e-4 in row 6)."""
    ket = synth.random_peps(4, 3, 2, 2, "c64", "cgauss_scaled", 41)
    la, ph, _ = _run(ket, ket, "c128", 16, 4, 1, 77, prec=libpeps.PREC_PLAIN, flags=libpeps.FLAG_ALTERNATE)
    assert la == pytest.approx(np.log(abs(bruteforce.exact_scalar(ket, ket))), abs=1e-9)
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    rec = []
    la, ph, sig = _run(ket, ket, "c64", cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec, flags=libpeps.FLAG_ALTERNATE)
    ra, rp = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec, alternate=True)
    assert abs(la - ra) <= 1e-5 * abs(ra)
    bars, rows, env = _row_bars("c2_envelope_alternate.json")
    errs = sigma_errors(sig, rec)
    print(f"prec {prec}: per-row max", ["%.1e" % errs[rows == r].max() for r in range(1, 8)],
          "bars", ["%.1e" % bars[rows == r].max() for r in range(1, 8)], f"|d log v| {abs(la - ra):.2e}")
    assert np.all(errs <= bars), [(int(rows[i]), "%.2e" % errs[i]) for i in np.nonzero(errs > bars)[0]]
    plain, _ = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    assert ra != plain
