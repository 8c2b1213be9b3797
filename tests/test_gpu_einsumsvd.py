"""GPU parity of batched einsumsvd (Algorithm 3's einsumsvd line with
Algorithm 4 applied implicitly) against the oracle, instance by instance.

Checked per instance: singular values (normwise 1e-5 against sigma_1 for
single precision, 1e-10 for FP64), the factors U and W after the shared gauge
rule, and log(sigma_1).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import rsvd
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import TORCH_DT, tensor

pytestmark = pytest.mark.gpu


def _operands(rng, kL, t, a, b, d, Dk, Db, dtype):
    cplx = dtype.startswith("c")

    def r(shape):
        x = rng.standard_normal(shape)
        if cplx:
            x = x + 1j * rng.standard_normal(shape)
        return synth.round_to(x, dtype)
    Dl, Du, Dx, De = Dk
    DL, DU, DX, DE = Db
    return (r((kL, t, a, Dl * DL)), r((a, Du * DU, b)), r((d, Dl, Du, Dx, De)),
            r((d, DL, DU, DX, DE)))


def _run_batch(cases, dtype, m, p, q, seed, prec=libpeps.PREC_PLAIN, ranks=None, flags=0):
    shapes, ios, outs = [], [], []
    for i, (V, S, K, Kb) in enumerate(cases):
        kL, t, a, h = V.shape
        _, v, b = S.shape
        d, Dl, Du, Dx, De = K.shape
        _, DL, DU, DX, DE = Kb.shape
        shapes.append((kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE, ranks[i] if ranks else 0))
    plan = libpeps.EinsumsvdPlan(TORCH_DT[dtype], shapes, libpeps.make_opts(m, p, q, seed, prec=prec, flags=flags),
                                 instance_ids=list(range(100, 100 + len(cases))))
    for i, (V, S, K, Kb) in enumerate(cases):
        k = plan.ranks[i]
        kL, t = V.shape[:2]
        d, Dl, Du, Dx, De = K.shape
        _, DL, DU, DX, DE = Kb.shape
        b = S.shape[2]
        U = torch.zeros((kL, t, k), dtype=TORCH_DT[dtype], device="cuda")
        W = torch.zeros((k, Dx * DX, b, De * DE), dtype=TORCH_DT[dtype], device="cuda")
        sg = torch.zeros(k, dtype=torch.float64, device="cuda")
        lg = torch.zeros(1, dtype=torch.float64, device="cuda")
        io = (tensor(V, dtype), tensor(S, dtype), tensor(K, dtype), tensor(Kb, dtype), U, W, sg, lg)
        ios.append(io)
        outs.append((U, W, sg, lg))
    plan.execute(ios)
    torch.cuda.synchronize()
    return [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy(), float(o[3].cpu()[0]))
            for o in outs]


def _check(case, out, m, p, q, seed, inst, dtype, ftol=None):
    V, S, K, Kb = case
    U, W, s, l1 = rsvd.einsumsvd(V, S, K, Kb, m, p, q, seed, inst)
    gU, gW, gs, gl = out
    tol = 1e-10 if dtype in ("f64", "c128") else 1e-5
    assert np.max(np.abs(gs - s)) <= tol * s[0]
    assert gl == pytest.approx(l1, abs=tol)
    # factors: the product U W (gauge independent) and each factor (gauge fixed)
    k = len(s)
    UW = U.reshape(-1, k) @ W.reshape(k, -1)
    gUW = gU.reshape(-1, k) @ gW.reshape(k, -1)
    assert np.linalg.norm(gUW - UW) <= 10 * tol * np.linalg.norm(UW)
    if ftol is None:
        ftol = 1e-8 if dtype in ("f64", "c128") else 2e-3
    assert np.max(np.abs(gU - U)) <= ftol
    assert np.max(np.abs(gW - W)) <= ftol * np.max(np.abs(W))


@pytest.mark.parametrize("dtype", ["c64", "f32", "c128", "f64"])
def test_single_instance_ragged_tiles(dtype):
    rng = np.random.default_rng(3)
    # M = 20*9 = 180, N = 9*17*9 = 1377: several 64-wide tiles plus ragged tails
    case = _operands(rng, 20, 9, 20, 17, 2, (3, 3, 3, 3), (3, 3, 3, 3), dtype)
    out = _run_batch([case], dtype, 16, 8, 2, 42)
    _check(case, out[0], 16, 8, 2, 42, 100, dtype)


def test_batched_uneven_instances():
    rng = np.random.default_rng(4)
    cases = [
        _operands(rng, 4, 4, 6, 5, 2, (2, 2, 2, 2), (2, 2, 2, 2), "c64"),
        _operands(rng, 1, 9, 9, 9, 2, (3, 1, 3, 3), (3, 1, 3, 3), "c64"),     # kL = 1 row start
        _operands(rng, 16, 16, 16, 1, 2, (4, 4, 4, 1), (4, 4, 4, 1), "c64"),  # last column: b = e = 1
        _operands(rng, 12, 4, 7, 3, 3, (2, 2, 2, 2), (2, 1, 2, 2), "c64"),    # uneven ket/bra bonds
    ]
    outs = _run_batch(cases, "c64", 8, 4, 2, 9)
    for i, (c, o) in enumerate(zip(cases, outs)):
        _check(c, o, 8, 4, 2, 9, 100 + i, "c64")


def test_exact_regime_l_equals_m():
    """l = min(k+p, M, N) = M: the sketch spans the whole row space."""
    rng = np.random.default_rng(5)
    case = _operands(rng, 2, 4, 3, 4, 2, (2, 2, 2, 2), (2, 2, 2, 2), "c128")
    out = _run_batch([case], "c128", 50, 8, 1, 1)
    _check(case, out[0], 50, 8, 1, 1, 100, "c128")


def test_c3_sample_instances_full_size():
    """A sample of the batched workload's instances at their full sizes."""
    cfg = synth.config("c3")
    dims = synth.batched_dims(cfg)
    pick = [0, 1, int(np.argmax([m * D ** 4 for m, D in dims[:16]]))]
    cases, ms = [], []
    for i in pick:
        mm, D = dims[i]
        inst = synth.batched_instance(cfg, i, mm, D)
        cases.append((inst["V"], inst["S"], inst["ket"], inst["bra"]))
        ms.append(mm)
    # one plan per rank (k = m per instance)
    for c, mm, i in zip(cases, ms, pick):
        out = _run_batch([c], "f32", mm, cfg.p, cfg.q, cfg.omega_seed)
        _check(c, out[0], mm, cfg.p, cfg.q, cfg.omega_seed, 100, "f32")


@pytest.mark.parametrize("dtype", ["c64", "f32"])
def test_mixed_precision_tensor_core_step(dtype):
    """PEPS_PREC_MIXED: tensor-core products (TF32 for the early power-iteration
    products, 3xTF32 from the last A Q on).  Singular values stay within 1e-5
    of the FP64 oracle (normwise); the factors within the looser bound that
    single-precision singular vectors allow."""
    rng = np.random.default_rng(8)
    # every contracted extent even (complex) / a multiple of 4 (real): TMA rows
    D = 4 if dtype == "c64" else 4
    case = _operands(rng, 20, D * D, 20, 17 if dtype == "c64" else 16, 2, (D,) * 4, (D,) * 4, dtype)
    out = _run_batch([case], dtype, 16, 8, 2, 42, prec=libpeps.PREC_MIXED)
    V, S, K, Kb = case
    U, W, s, l1 = rsvd.einsumsvd(V, S, K, Kb, 16, 8, 2, 42, 100)
    gU, gW, gs, gl = out[0]
    assert np.max(np.abs(gs - s)) <= 1e-5 * s[0]
    assert gl == pytest.approx(l1, abs=1e-5)
    k = len(s)
    UW = U.reshape(-1, k) @ W.reshape(k, -1)
    gUW = gU.reshape(-1, k) @ gW.reshape(k, -1)
    assert np.linalg.norm(gUW - UW) <= 1e-4 * np.linalg.norm(UW)


@pytest.mark.parametrize("dtype,prec", [("c64", libpeps.PREC_PLAIN), ("c64", libpeps.PREC_MIXED),
                                        ("f32", libpeps.PREC_PLAIN), ("c128", libpeps.PREC_PLAIN)])
def test_wide_sketch_cluster_factorisations(dtype, prec):
    """l = 264: the l x l Cholesky and Jacobi no longer fit one CTA's shared
    memory and run as 8-CTA clusters (rows / columns in distributed shared
    memory; the Jacobi block-cyclic for single precision, a column window for
    FP64 complex, with a ragged last column block); FP64 data take the
    global-memory Cholesky.  Same parity bar."""
    rng = np.random.default_rng(21)
    D = 4
    # a * D^2 = 320 >= l: A has full rank 288 (no directions below rounding level)
    case = _operands(rng, 18, D * D, 20, 18, 2, (D,) * 4, (D,) * 4, dtype)
    out = _run_batch([case], dtype, 256, 8, 2, 77, prec=prec)
    _check(case, out[0], 256, 8, 2, 77, 100, dtype)


def test_block_cyclic_jacobi_fp64_complex():
    """l = 168 in complex FP64: the Jacobi runs on the block-cyclic cluster
    kernel (16 column blocks of 11, two per CTA) rather than the column-window
    one that l = 264 takes in FP64 complex."""
    rng = np.random.default_rng(23)
    D = 4
    case = _operands(rng, 18, D * D, 20, 18, 2, (D,) * 4, (D,) * 4, "c128")
    out = _run_batch([case], "c128", 160, 8, 2, 78, prec=libpeps.PREC_PLAIN)
    _check(case, out[0], 160, 8, 2, 78, 100, "c128")


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_c3_batch_with_per_instance_ranks(prec):
    """Twelve instances of the batched workload in ONE plan, each with its own
    rank k = m (grouped launches for the small kernels, tensor-core stages
    instance by instance where the extents allow)."""
    cfg = synth.config("c3")
    dims = synth.batched_dims(cfg)[:12]
    cases, ms = [], []
    for i, (mm, D) in enumerate(dims):
        inst = synth.batched_instance(cfg, i, mm, D)
        cases.append((inst["V"], inst["S"], inst["ket"], inst["bra"]))
        ms.append(mm)
    out = _run_batch(cases, "f32", 128, cfg.p, cfg.q, cfg.omega_seed, prec=prec, ranks=ms)
    for i, (c, mm) in enumerate(zip(cases, ms)):
        # singular values, log sigma_1 and U W at the single-precision bar;
        # the individual factors of the m = 80, D = 5 instance move by 3.4e-3
        # (close singular values at its truncation edge: single-precision
        # singular vectors move by ~u sigma_1 / gap), so they get 1e-2
        _check(c, out[i], mm, cfg.p, cfg.q, cfg.omega_seed, 100 + i, "f32", ftol=1e-2)


@pytest.mark.parametrize("dtype", ["f32", "c64"])
def test_padded_copy_on_tensor_cores(dtype):
    """Instances whose contracted extents break the TMA row alignment (odd
    bonds, t and a not multiples of 4) run on the tensor cores through a
    zero-padded copy: the padded operator is the original one with zero rows
    and columns added, the sketch and gauge vector are drawn at the original
    element numbering, so every singular value, U and W match the oracle on
    the original operands.  Several such instances share one plan (their
    chains run as concurrent graph branches)."""
    rng = np.random.default_rng(29)
    cases = [_operands(rng, 6, 9, 7, 5, 2, (3, 3, 3, 3), (3, 3, 3, 3), dtype),
             _operands(rng, 10, 25, 13, 6, 2, (5, 5, 5, 5), (5, 5, 5, 5), dtype),
             _operands(rng, 12, 6, 10, 9, 2, (2, 3, 3, 2), (3, 2, 2, 3), dtype)]
    out = _run_batch(cases, dtype, 24, 8, 2, 81, prec=libpeps.PREC_MIXED)
    for i, c in enumerate(cases):
        _check(c, out[i], 24, 8, 2, 81, 100 + i, dtype, ftol=1e-2)


@pytest.mark.parametrize("dtype,prec", [("c64", libpeps.PREC_PLAIN), ("c64", libpeps.PREC_MIXED),
                                        ("f32", libpeps.PREC_PLAIN), ("f32", libpeps.PREC_MIXED)])
@pytest.mark.parametrize("ell_case", ["one_cta", "cluster"])
def test_fp64_small_factorisations(dtype, prec, ell_case):
    """PEPS_FLAG_FP64_SMALL: the CholeskyQR2 factorisations and the Jacobi SVD
    run in FP64 on single-precision data (one-CTA kernels at l = 40, 8-CTA
    cluster kernels at l = 264); same parity bar as the default."""
    rng = np.random.default_rng(31)
    D = 4
    if ell_case == "one_cta":
        case = _operands(rng, 6, D * D, 8, 6, 2, (D,) * 4, (D,) * 4, dtype)
        m = 32
    else:
        case = _operands(rng, 18, D * D, 20, 18, 2, (D,) * 4, (D,) * 4, dtype)
        m = 256
    out = _run_batch([case], dtype, m, 8, 2, 79, prec=prec, flags=libpeps.FLAG_FP64_SMALL)
    _check(case, out[0], m, 8, 2, 79, 100, dtype)


def test_branch_count_changes_no_result():
    """Dealing the tensor-core chains to 1 or to 64 side streams (parallel
    graph branches, per-branch scratch) runs the same kernels on the same
    operands: bit-identical outputs."""
    cfg = synth.config("c3")
    dims = synth.batched_dims(cfg)[:24]
    shapes, host = [], []
    for i, (mm, D) in enumerate(dims):
        inst = synth.batched_instance(cfg, i, mm, D)
        host.append([inst[k] for k in ("V", "S", "ket", "bra")])
        R = D * D
        shapes.append((mm, R, mm, mm, cfg.d, D, D, D, D, D, D, D, D, mm))
    plan = libpeps.EinsumsvdPlan(torch.float32, shapes,
                                 libpeps.make_opts(128, cfg.p, cfg.q, cfg.omega_seed, prec=libpeps.PREC_MIXED))
    outs = []
    for nb in (1, 64):
        plan.set_branches(nb)
        ios = []
        for (V, S, K, Kb), sh, k in zip(host, shapes, plan.ranks):
            mm, R = sh[0], sh[1]
            ios.append((tensor(V, "f32"), tensor(S, "f32"), tensor(K, "f32"), tensor(Kb, "f32"),
                        torch.zeros((mm * R, k), device="cuda"), torch.zeros((k, R * mm * R), device="cuda"),
                        torch.zeros(k, dtype=torch.float64, device="cuda"),
                        torch.zeros(1, dtype=torch.float64, device="cuda")))
        plan.execute(ios)
        torch.cuda.synchronize()
        outs.append([[t.cpu().numpy() for t in io[4:]] for io in ios])
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
