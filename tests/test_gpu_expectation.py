"""GPU expectation values (Eq. 6 with the cached environments of Sec. IV-B)
against the oracle: the 6 x 6 transverse-field Ising energy of the workload
(real FP32 sites, m = 18), the exact regime against the state vector, the
uncached schedule against the cached one, and a complex lattice."""
import numpy as np
import pytest

import synth
from oracle import bmps, bruteforce, expectation
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _oracle_log_norm(ket, m, p, q, seed):
    """log <psi|psi> the way the GPU reads it: row 0's strip and the scales of
    the bottom-up sweep below it."""
    nrow, ncol = len(ket), len(ket[0])
    fl = bmps.flip_vertical(ket)
    bot, logs = bmps.sweep(fl, fl, m, p, q, seed, 1, nrow - 2)
    v = expectation.strip_value(expectation.trivial_env(ncol), ket[0], ket[0], bot[nrow - 2], {})
    return float(np.log(abs(v)) + logs[nrow - 2])


def test_c4_tfi_energy_matches_oracle():
    cfg = synth.config("c4")
    ket = synth.peps_for(cfg)
    terms = synth.tfi_terms(cfg.nrow, cfg.ncol, cfg.extra["J"], cfg.extra["h"])
    e, ln, tv = libpeps.expectation(to_dev(ket, "f32"), terms, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    ref, ref_t = expectation.energy(ket, terms, cfg.m, cfg.p, cfg.q, cfg.omega_seed, return_terms=True)
    assert abs(e - ref) <= 1e-5 * abs(ref), (e, ref)
    ref_t = np.asarray(ref_t)
    assert np.max(np.abs(tv - ref_t)) <= 1e-5 * np.max(np.abs(ref_t))
    rl = _oracle_log_norm(ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    assert abs(ln - rl) <= 1e-5 * abs(rl), (ln, rl)


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5), ("f64", 1e-9)])
def test_exact_regime_equals_statevector(dtype, tol):
    ket = synth.random_peps(3, 3, 2, 2, dtype, "normal", 23)
    terms = synth.tfi_terms(3, 3, 1.0, 3.0)
    e, ln, tv = libpeps.expectation(to_dev(ket, dtype), terms, 16, 4, 1, 2)
    ref = bruteforce.statevector_energy(ket, terms)
    assert e == pytest.approx(ref, abs=tol * max(1.0, abs(ref)))
    psi = bruteforce.statevector(ket)
    assert ln == pytest.approx(float(np.log(np.vdot(psi, psi).real)), abs=tol * 10)


def test_uncached_schedule_gives_the_cached_values():
    cfg = synth.config("c4")
    ket = synth.random_peps(4, 4, 2, 3, "f32", "normal_tenth", 31)
    terms = synth.tfi_terms(4, 4, 1.0, 3.0)
    k = to_dev(ket, "f32")
    a = libpeps.expectation(k, terms, 9, 8, 2, 5, use_cache=True)
    b = libpeps.expectation(k, terms, 9, 8, 2, 5, use_cache=False)
    assert a[0] == b[0] and a[1] == b[1]
    assert np.array_equal(a[2], b[2])
    ref = expectation.energy(ket, terms, 9, 8, 2, 5)
    assert abs(a[0] - ref) <= 1e-5 * abs(ref)


def test_complex_lattice_matches_oracle():
    ket = synth.random_peps(4, 3, 2, 2, "c64", "cgauss_scaled", 41)
    terms = synth.tfi_terms(4, 3, 0.7, 1.3)
    e, ln, tv = libpeps.expectation(to_dev(ket, "c64"), terms, 4, 4, 2, 3)
    ref, ref_t = expectation.energy(ket, terms, 4, 4, 2, 3, return_terms=True)
    assert abs(e - ref) <= 1e-5 * max(1.0, abs(ref)), (e, ref)
    # <O_t> from truncated environments may carry a small imaginary part; the
    # library reports Re(strip(O) / strip(1)) per term
    ref_t = np.real(np.asarray(ref_t))
    assert np.max(np.abs(tv - ref_t)) <= 1e-5 * max(1.0, np.max(np.abs(ref_t)))


@pytest.mark.parametrize("dtype,prec", [("f64", libpeps.PREC_PLAIN), ("c64", libpeps.PREC_MIXED)])
def test_two_part_split_gives_the_single_plan_values(dtype, prec):
    """The two-GPU split of the cached expectation emulated with two plans on
    one GPU: plan A runs the top-down sweeps (part 0), plan B the bottom-up
    ones (part 1), each copies the other's region (what the all-gather does
    between ranks), both run the strips (part 2).  Every value equals the
    single plan's; so does one plan running the three parts in turn."""
    import torch
    cplx = dtype.startswith("c")
    ket = synth.random_peps(4, 3, 2, 2, "c64" if cplx else "f64", "cgauss_scaled" if cplx else "normal", 43)
    terms = synth.tfi_terms(4, 3, 0.7, 1.3)
    k = to_dev(ket, dtype)
    opts = libpeps.make_opts(4, 4, 2, 3, prec=prec)
    ref = libpeps.ExpectationPlan(k, terms, opts)
    ref.execute()
    r = ref.result()
    a = libpeps.ExpectationPlan(k, terms, opts)
    b = libpeps.ExpectationPlan(k, terms, opts)
    assert a.env_region(0) == b.env_region(0) and a.env_region(1) == b.env_region(1)
    a.execute_part(0)
    b.execute_part(1)
    torch.cuda.synchronize()
    a.env_view(1).copy_(b.env_view(1))
    b.env_view(0).copy_(a.env_view(0))
    a.execute_part(2)
    b.execute_part(2)
    one = libpeps.ExpectationPlan(k, terms, opts)
    for part in (0, 1, 2):
        one.execute_part(part)
    for got in (a.result(), b.result(), one.result()):
        assert got[0] == pytest.approx(r[0], rel=1e-12, abs=1e-12)
        assert got[1] == pytest.approx(r[1], rel=1e-12, abs=1e-12)
        assert np.allclose(got[2], r[2], rtol=1e-12, atol=1e-12)
