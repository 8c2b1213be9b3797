"""Host-side bounds check of every launch descriptor (no GPU needed).

peps_plan_validate rebuilds a plan's launch schedule for concrete (fake)
addresses and checks that each kernel's reachable byte range lies inside the
workspace or a caller tensor of the planned shape.  Every shape the GPU tests
and the benchmark use is checked here before it ever reaches a GPU.
"""
import ctypes as C

import pytest

import synth

L = pytest.importorskip("paper_2006_15234_gb300.libpeps")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_15234_gb300 import build
    build.build_library()
    return L.load()


class FakeHeap:
    """Disjoint, page-aligned fake device addresses with guard gaps."""

    def __init__(self):
        self.top = 1 << 40

    def __call__(self, nbytes):
        p = self.top
        self.top += ((int(nbytes) + 4095) // 4096 + 16) * 4096
        return p


ES = {0: 4, 1: 8, 2: 8, 3: 16}


def _einsumsvd_ok(lib, dt, shapes, m, p, q, prec=0):
    heap = FakeHeap()
    n = len(shapes)
    arr = (L.EinsumsvdShape * n)(*[L.EinsumsvdShape(*s) for s in shapes])
    plan, ws = C.c_void_p(), C.c_size_t()
    opts = L.make_opts(m, p, q, 1, prec=prec)
    assert lib.peps_einsumsvd_plan(C.byref(plan), dt, n, arr, None, C.byref(opts), C.byref(ws)) == 0
    es = ES[dt]
    io = (L.EinsumsvdIO * n)()
    for i, s in enumerate(shapes):
        kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE = s[:13]
        k = C.c_int32()
        lib.peps_einsumsvd_rank(plan, i, C.byref(k))
        M, N = kL * t, Dx * DX * b * De * DE
        io[i] = L.EinsumsvdIO(heap(es * kL * t * a * Dl * DL), heap(es * a * Du * DU * b),
                              heap(es * d * Dl * Du * Dx * De), heap(es * d * DL * DU * DX * DE),
                              heap(es * M * k.value), heap(es * k.value * N), heap(8 * k.value), heap(8))
    wsp = heap(ws.value)
    r = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, io)
    msg = lib.peps_last_error().decode()
    # one byte less of workspace must be refused
    r2 = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value - 1, io)
    lib.peps_plan_destroy(plan)
    return r, msg, r2


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dt", [0, 1, 2, 3])
def test_einsumsvd_test_shapes(lib, dt, prec):
    shapes = [(20, 9, 20, 17, 2, 3, 3, 3, 3, 3, 3, 3, 3), (4, 4, 6, 5, 2, 2, 2, 2, 2, 2, 2, 2, 2),
              (1, 9, 9, 9, 2, 3, 1, 3, 3, 3, 1, 3, 3), (16, 16, 16, 1, 2, 4, 4, 4, 1, 4, 4, 4, 1),
              (12, 4, 7, 3, 3, 2, 2, 2, 2, 2, 1, 2, 2), (2, 4, 3, 4, 2, 2, 2, 2, 2, 2, 2, 2, 2)]
    r, msg, r2 = _einsumsvd_ok(lib, dt, shapes, 8, 4, 2, prec)
    assert r == 0, msg
    assert r2 != 0


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_workload_sample(lib, prec):
    cfg = synth.config("c3")
    dims = synth.batched_dims(cfg)[:64]
    # per-instance rank k = m (the shape's rank field)
    shapes = [(m, D * D, m, m, 2, D, D, D, D, D, D, D, D, m) for m, D in dims]
    r, msg, _ = _einsumsvd_ok(lib, 0, shapes, 128, cfg.p, cfg.q, prec)
    assert r == 0, msg


def _net(heap, sites_shape, dt):
    nrow, ncol = len(sites_shape), len(sites_shape[0])
    es = ES[dt]
    bh = (C.c_int32 * max(1, nrow * (ncol - 1)))()
    bv = (C.c_int32 * max(1, (nrow - 1) * ncol))()
    for p in range(nrow):
        for q in range(ncol - 1):
            bh[p * (ncol - 1) + q] = sites_shape[p][q][4]
    for p in range(nrow - 1):
        for q in range(ncol):
            bv[p * ncol + q] = sites_shape[p][q][3]
    ptrs = (C.c_void_p * (nrow * ncol))()
    for p in range(nrow):
        for q in range(ncol):
            s = sites_shape[p][q]
            ptrs[p * ncol + q] = heap(es * s[0] * s[1] * s[2] * s[3] * s[4])
    net = L.Network(nrow, ncol, sites_shape[0][0][0], dt, C.cast(bh, C.POINTER(C.c_int32)),
                    C.cast(bv, C.POINTER(C.c_int32)), C.cast(ptrs, C.POINTER(C.c_void_p)))
    return net, (bh, bv, ptrs)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key,dt,two", [("c1", 2, False), ("c2", 1, True), ("c4", 0, True),
                                        ("c5", 1, True)])
def test_contract_workloads(lib, key, dt, two, prec):
    cfg = synth.config(key)
    shp = [[synth.site_shape(cfg.nrow, cfg.ncol, p, q, cfg.d, cfg.D) for q in range(cfg.ncol)]
           for p in range(cfg.nrow)]
    heap = FakeHeap()
    net, keep = _net(heap, shp, dt)
    plan, ws = C.c_void_p(), C.c_size_t()
    opts = L.make_opts(cfg.m, cfg.p, cfg.q, 1, prec=prec)
    assert lib.peps_contract_plan(C.byref(plan), C.byref(net), C.byref(net) if two else None,
                                  C.byref(opts), 0, C.byref(ws)) == 0, lib.peps_last_error()
    wsp = heap(ws.value)
    r = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, None)
    assert r == 0, lib.peps_last_error().decode()
    lib.peps_plan_destroy(plan)


@pytest.mark.parametrize("shape,D,m", [((3, 3), 2, 16), ((3, 5), 2, 64), ((1, 4), 2, 4),
                                       ((4, 1), 2, 4), ((5, 3), 2, 5), ((3, 6), 3, 9)])
def test_contract_test_shapes(lib, shape, D, m):
    nr, nc = shape
    shp = [[synth.site_shape(nr, nc, p, q, 2, D) for q in range(nc)] for p in range(nr)]
    for dt in (1, 3):
        heap = FakeHeap()
        net, keep = _net(heap, shp, dt)
        plan, ws = C.c_void_p(), C.c_size_t()
        opts = L.make_opts(m, 8, 1, 1, prec=1 if dt == 1 else 0)
        assert lib.peps_contract_plan(C.byref(plan), C.byref(net), C.byref(net), C.byref(opts), 0,
                                      C.byref(ws)) == 0
        wsp = heap(ws.value)
        assert lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, None) == 0, lib.peps_last_error()
        lib.peps_plan_destroy(plan)


def _term_array(terms, ncol, cplx):
    import numpy as np
    arr = (L.Term * len(terms))()
    keep = []
    for i, (st, op, coeff) in enumerate(terms):
        a = np.ascontiguousarray(np.asarray(op, dtype=np.complex128 if cplx else np.float64))
        if cplx:
            a = np.ascontiguousarray(a.view(np.float64))
        keep.append(a)
        arr[i].nsite = len(st)
        for k, (p, q) in enumerate(st):
            arr[i].site[k] = p * ncol + q
        arr[i].op = a.ctypes.data_as(C.POINTER(C.c_double))
        arr[i].coeff = coeff
    return arr, keep


@pytest.mark.parametrize("use_cache", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key,dt,shape", [("c4", 0, None), ("c4", 2, (3, 4)), ("c2", 1, (3, 3))])
def test_expectation_plans(lib, key, dt, shape, prec, use_cache):
    """Cached and uncached expectation plans (lattice copies, four sweeps,
    strips) stay inside the workspace and the network."""
    cfg = synth.config(key)
    nr, nc = shape if shape else (cfg.nrow, cfg.ncol)
    D = cfg.D if key == "c4" else 2
    shp = [[synth.site_shape(nr, nc, p, q, cfg.d, D) for q in range(nc)] for p in range(nr)]
    heap = FakeHeap()
    net, keep = _net(heap, shp, dt)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    arr, tkeep = _term_array(terms, nc, dt in (1, 3))
    plan, ws = C.c_void_p(), C.c_size_t()
    opts = L.make_opts(cfg.m if key == "c4" else 8, 8, 2, 1, prec=prec)
    assert lib.peps_expectation_plan(C.byref(plan), C.byref(net), arr, len(terms), C.byref(opts), use_cache,
                                     C.byref(ws)) == 0, lib.peps_last_error()
    wsp = heap(ws.value)
    r = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, None)
    assert r == 0, lib.peps_last_error().decode()
    # the two-GPU split: each sweep part's environments in one region of the
    # workspace, the two regions disjoint (cached schedule only)
    off, n = [C.c_size_t(), C.c_size_t()], [C.c_size_t(), C.c_size_t()]
    rs = [lib.peps_expectation_env_region(plan, part, C.byref(off[part]), C.byref(n[part])) for part in (0, 1)]
    if use_cache:
        assert rs == [0, 0], lib.peps_last_error()
        assert 0 < n[0].value and 0 < n[1].value
        assert off[0].value + n[0].value <= off[1].value and off[1].value + n[1].value <= ws.value
    else:
        assert rs == [3, 3]
    lib.peps_plan_destroy(plan)


def test_expectation_rejects_long_range_terms(lib):
    import numpy as np
    shp = [[synth.site_shape(3, 3, p, q, 2, 2) for q in range(3)] for p in range(3)]
    net, keep = _net(FakeHeap(), shp, 0)
    zz = np.kron(np.diag([1.0, -1.0]), np.diag([1.0, -1.0]))
    arr, tkeep = _term_array([(((0, 0), (0, 2)), zz, 1.0)], 3, False)
    plan, ws = C.c_void_p(), C.c_size_t()
    opts = L.make_opts(4, 2, 1, 1)
    assert lib.peps_expectation_plan(C.byref(plan), C.byref(net), arr, 1, C.byref(opts), 1, C.byref(ws)) == 3
    assert b"nearest-neighbour" in lib.peps_last_error()


def test_per_instance_rank(lib):
    """The shape's rank field overrides opts.m for that instance only."""
    shapes = [(16, 9, 16, 16, 2, 3, 3, 3, 3, 3, 3, 3, 3, 5), (16, 9, 16, 16, 2, 3, 3, 3, 3, 3, 3, 3, 3, 0)]
    arr = (L.EinsumsvdShape * 2)(*[L.EinsumsvdShape(*s) for s in shapes])
    plan, ws = C.c_void_p(), C.c_size_t()
    opts = L.make_opts(12, 4, 1, 1)
    assert lib.peps_einsumsvd_plan(C.byref(plan), 0, 2, arr, None, C.byref(opts), C.byref(ws)) == 0
    k = C.c_int32()
    lib.peps_einsumsvd_rank(plan, 0, C.byref(k))
    assert k.value == 5
    lib.peps_einsumsvd_rank(plan, 1, C.byref(k))
    assert k.value == 12
    lib.peps_plan_destroy(plan)


@pytest.mark.parametrize("dt", [0, 2])
@pytest.mark.parametrize("shape,m,q", [((3, 4, 5, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2), 4, 1),
                                       ((18, 9, 18, 18, 2, 3, 3, 3, 3, 3, 3, 3, 3), 18, 2)])
def test_einsumsvd_adjoint_plan(lib, dt, shape, m, q):
    """The adjoint's forward-with-saving and reverse sweep stay inside the
    workspace, the operands, the cotangents and the gradient buffers."""
    heap = FakeHeap()
    es = ES[dt]
    kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE = shape
    sh = L.EinsumsvdShape(*shape, m)
    plan, ws = C.c_void_p(), C.c_size_t()
    assert lib.peps_einsumsvd_grad_plan(C.byref(plan), dt, C.byref(sh), C.byref(L.make_opts(m, 8, q, 1)),
                                        C.byref(ws)) == 0, lib.peps_last_error()
    k = C.c_int32()
    lib.peps_einsumsvd_rank(plan, 0, C.byref(k))
    M, N = kL * t, Dx * DX * b * De * DE
    sizes = (es * kL * t * a * Dl * DL, es * a * Du * DU * b, es * d * Dl * Du * Dx * De, es * d * DL * DU * DX * DE)
    io = L.EinsumsvdIO(*[heap(x) for x in sizes], heap(es * M * k.value), heap(es * k.value * N),
                       heap(8 * k.value), heap(8))
    ct = L.Cotangent(heap(es * M * k.value), heap(es * k.value * N), heap(8))
    gr = L.Grads(*[heap(x) for x in sizes])
    assert lib.peps_einsumsvd_grad_bind(plan, C.byref(ct), C.byref(gr)) == 0
    wsp = heap(ws.value)
    r = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, C.byref(io))
    assert r == 0, lib.peps_last_error().decode()
    lib.peps_plan_destroy(plan)


@pytest.mark.parametrize("dt,shape,D,m", [(0, (3, 3), 2, 4), (2, (3, 4), 2, 6), (0, (6, 6), 3, 18)])
def test_energy_gradient_plans(lib, dt, shape, D, m):
    """The gradient plan (sweeps keeping every step, strips, reverse sweep,
    lattice adjoints) stays inside the workspace and the network."""
    nr, nc = shape
    shp = [[synth.site_shape(nr, nc, p, q, 2, D) for q in range(nc)] for p in range(nr)]
    heap = FakeHeap()
    net, keep = _net(heap, shp, dt)
    terms = synth.tfi_terms(nr, nc, 1.0, 3.0)
    arr, tkeep = _term_array(terms, nc, False)
    plan, ws = C.c_void_p(), C.c_size_t()
    assert lib.peps_grad_plan(C.byref(plan), C.byref(net), arr, len(terms), C.byref(L.make_opts(m, 8, 2, 1)),
                              C.byref(ws)) == 0, lib.peps_last_error()
    wsp = heap(ws.value)
    r = lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, None)
    assert r == 0, lib.peps_last_error().decode()
    lib.peps_plan_destroy(plan)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dt", [0, 1])
def test_random_single_instance_shapes(lib, dt, prec):
    """Seeded random zip-up step shapes, one instance per plan, each validated
    against its workspace with the workspace one byte short refused.  Half of
    them are drawn with bond and boundary sizes that meet the tensor-core
    path's alignment (the mixed path's schedule for single instances: B
    pre-expansion scratch, tensor-core CholeskyQR apply, or its SIMT fallback
    where M > N, Grams split over K); the mixed plans must use the tensor
    cores for those."""
    import numpy as np
    rng = np.random.default_rng(20200619 + 10 * dt + prec)
    tc_plans = tall = 0
    for i in range(16):
        if i % 2:
            D = [int(x) for x in rng.choice([2, 4], size=8)]
            kL, a, b = (4 * int(x) for x in rng.integers(1, 12, size=3))
            t = int(rng.choice([4, 16]))
            d = 2
        else:
            D = [int(x) for x in rng.integers(1, 5, size=8)]
            kL, a, b = (int(x) for x in rng.integers(1, 40, size=3))
            t = int(rng.integers(1, 17))
            d = int(rng.integers(1, 3))
        m = int(rng.integers(2, 48))
        shape = (kL, t, a, b, d) + tuple(D)
        r, msg, r2 = _einsumsvd_ok(lib, dt, [shape], m, 4, int(rng.integers(0, 3)), prec)
        assert r == 0, (shape, m, msg)
        assert r2 != 0, shape
        arr = (L.EinsumsvdShape * 1)(L.EinsumsvdShape(*shape))
        plan, ws = C.c_void_p(), C.c_size_t()
        assert lib.peps_einsumsvd_plan(C.byref(plan), dt, 1, arr, None, C.byref(L.make_opts(m, 4, 1, 1, prec=prec)),
                                       C.byref(ws)) == 0
        n = C.c_int64()
        lib.peps_plan_launch_count(plan, C.byref(n))
        kinds = set()
        for j in range(n.value):
            kk = C.c_char_p()
            lib.peps_plan_launch_kernel(plan, j, C.byref(kk))
            kinds.add(kk.value.decode())
        lib.peps_plan_destroy(plan)
        if "tc_gemm" in kinds:
            tc_plans += 1
            M, N = kL * t, D[2] * D[6] * b * D[3] * D[7]
            tall += M > N
    if prec == 1:
        assert tc_plans >= 4, tc_plans
    else:
        assert tc_plans == 0


def _stage_flops(lib, dt, shape, m, p, q, prec):
    arr = (L.EinsumsvdShape * 1)(L.EinsumsvdShape(*shape))
    plan, ws = C.c_void_p(), C.c_size_t()
    assert lib.peps_einsumsvd_plan(C.byref(plan), dt, 1, arr, None, C.byref(L.make_opts(m, p, q, 1, prec=prec)),
                                   C.byref(ws)) == 0
    n = C.c_int64()
    lib.peps_plan_launch_count(plan, C.byref(n))
    agg = {}
    for i in range(n.value):
        tag, fl, by = C.c_char_p(), C.c_double(), C.c_double()
        lib.peps_plan_launch_info(plan, i, C.byref(tag), C.byref(fl), C.byref(by))
        agg[tag.value.decode()] = agg.get(tag.value.decode(), 0.0) + fl.value
    k = C.c_int32()
    lib.peps_einsumsvd_rank(plan, 0, C.byref(k))
    lib.peps_plan_destroy(plan)
    return agg, k.value


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,m,q", [((32, 16, 32, 32, 2, 4, 4, 4, 4, 4, 4, 4, 4), 32, 2),
                                       ((256, 64, 256, 256, 2) + (8,) * 8, 256, 2),
                                       ((20, 9, 20, 17, 2, 3, 3, 3, 3, 3, 3, 3, 3), 8, 1)])
def test_product_flops_follow_table_2(lib, shape, m, q, prec):
    """The planner's flop accounting of the implicit products (what the
    benchmark's TFLOP/s and roofline rest on) equals Table 2's two-layer
    terms: per product of c columns, c (b d (P1 Q1 Q2 + P1 Q2 P2) + a b h v
    + M a h) complex MACs (the four contraction stages), q + 1 products A X
    and q + 1 products A^H Y of l columns; W is one more implicit product of k
    columns on the tensor-core path and a k x l x N GEMM on the plain path."""
    kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE = shape
    P1, Q1, P2, Q2 = Dl * Du, Dx * De, DL * DU, DX * DE
    h, v = Dl * DL, Du * DU
    M, N = kL * t, Dx * DX * b * De * DE
    p = 8
    agg, k = _stage_flops(lib, 1, shape, m, p, q, prec)
    ell = min(k + p, M, N)

    def prod(c):
        return 8.0 * c * (b * d * (P1 * Q1 * Q2 + P1 * Q2 * P2) + a * b * h * v + M * a * h)

    fwd = sum(v_ for t_, v_ in agg.items() if t_.startswith("product_"))
    adj = sum(v_ for t_, v_ in agg.items() if t_.startswith("adjoint_"))
    assert fwd == pytest.approx((q + 1) * prod(ell), rel=1e-12)
    if "svd_gram" in agg:                      # tensor-core path
        assert adj + agg["epilogue_w"] == pytest.approx((q + 1) * prod(ell) + prod(k), rel=1e-12)
    else:
        assert adj == pytest.approx((q + 1) * prod(ell), rel=1e-12)
        assert agg["epilogue_w"] == pytest.approx(8.0 * k * ell * N, rel=1e-12)


@pytest.mark.parametrize("shape,D,dt,per_bond,nsite,flags",
                         [((3, 3), 2, 3, False, 0, 0), ((4, 4), 3, 1, True, 1, 8), ((5, 3), 4, 0, False, 15, 8),
                          ((16, 16), 8, 1, False, 1, 8), ((2, 5), 2, 2, True, 10, 0), ((1, 4), 2, 1, False, 0, 0)])
def test_tebd_layer_plans(lib, shape, D, dt, per_bond, nsite, flags):
    """The TEBD layer's launches (one-site operators, site matrices,
    CholeskyQR2, Theta, its SVD, N = Q R~, gauge phases, sites written back
    in place) stay inside the workspace and the site tensors, with one or
    per-bond operators and none, one or per-site one-site operators; one
    byte less of workspace is refused."""
    nr, nc = shape
    shp = [[synth.site_shape(nr, nc, p, q, 2, D) for q in range(nc)] for p in range(nr)]
    heap = FakeHeap()
    net, keep = _net(heap, shp, dt)
    nb = nr * (nc - 1) + (nr - 1) * nc
    ng = nb if per_bond else 1
    gate = (C.c_double * (32 * ng))(*([0.5] * (32 * ng)))
    sg = (C.c_double * max(1, 8 * nsite))(*([0.25] * max(1, 8 * nsite)))
    plan, ws = C.c_void_p(), C.c_size_t()
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, ng, sg if nsite else None, nsite,
                              C.byref(L.make_opts(1, 0, 0, 3, flags=flags)), C.byref(ws)) == 0, lib.peps_last_error()
    wsp = heap(ws.value)
    assert lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value, None) == 0, lib.peps_last_error().decode()
    assert lib.peps_plan_validate(plan, C.c_void_p(wsp), ws.value - 1, None) != 0
    lib.peps_plan_destroy(plan)


def test_tebd_refuses_unsupported(lib):
    heap = FakeHeap()
    shp = [[synth.site_shape(3, 3, p, q, 2, 2) for q in range(3)] for p in range(3)]
    net, keep = _net(heap, shp, 1)
    gate = (C.c_double * 32)(*([0.5] * 32))
    plan, ws = C.c_void_p(), C.c_size_t()
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, 1, None, 0,
                              C.byref(L.make_opts(1, 0, 0, 3, prec=1)), C.byref(ws)) == 3
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), None, 1, None, 0, C.byref(L.make_opts(1, 0, 0, 3)),
                              C.byref(ws)) == 1
    # operator counts: 1 or the number of bonds (12 on 3 x 3); 0, 1 or 9 one-site operators
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, 2, None, 0, C.byref(L.make_opts(1, 0, 0, 3)),
                              C.byref(ws)) == 1
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, 1, gate, 4, C.byref(L.make_opts(1, 0, 0, 3)),
                              C.byref(ws)) == 1
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, 1, None, 1, C.byref(L.make_opts(1, 0, 0, 3)),
                              C.byref(ws)) == 1
    # flags other than PEPS_FLAG_UNIT_BOND are refused, and UNIT_BOND elsewhere
    assert lib.peps_tebd_plan(C.byref(plan), C.byref(net), gate, 1, None, 0,
                              C.byref(L.make_opts(1, 0, 0, 3, flags=L.FLAG_ALTERNATE)), C.byref(ws)) == 3
    assert lib.peps_contract_plan(C.byref(plan), C.byref(net), None,
                                  C.byref(L.make_opts(4, 2, 1, 3, flags=L.FLAG_UNIT_BOND)), 0, C.byref(ws)) == 3
