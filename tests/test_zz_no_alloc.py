"""peps_boundary_contract_static: the contraction for callers that cannot
allocate device memory (a plugin given only its buffers by a host application
that keeps the allocators, a process whose memory another framework's caching
allocator already holds, a loop that cannot pay for cudaMalloc's device-wide
synchronisation).  It runs in the library's fixed 32 MiB device scratch array.

The GPU test checks it against peps_boundary_contract (caller-provided
workspace) on two calls in a row, the second one starting from the scratch
the first one left behind, and checks that the second call changes neither
the device's free memory nor any allocation count of PyTorch's caching
allocator.  The file is named to be collected last.
"""
import ctypes as C

import pytest

import synth
from paper_2006_15234_gb300 import libpeps

LOG_TOL = 1e-5      # relative log-norm tolerance of the contraction tests


def _shapes(nrow, ncol, d, D):
    return [[synth.site_shape(nrow, ncol, p, q, d, D) for q in range(ncol)] for p in range(nrow)]


def test_oversize_rejected_before_any_gpu_work():
    """A 16 x 16, D = 8, m = 256 norm needs far more than the static array:
    refused with PEPS_ERR_WORKSPACE while planning (no device is touched)."""
    from paper_2006_15234_gb300 import build
    build.build_library()
    lib = libpeps.load()
    shp = _shapes(16, 16, 2, 8)
    bh = (C.c_int32 * (16 * 15))(*([8] * (16 * 15)))
    bv = (C.c_int32 * (15 * 16))(*([8] * (15 * 16)))
    ptrs = (C.c_void_p * 256)(*[(1 << 40) + (i << 24) for i in range(256)])
    assert shp[5][5] == (2, 8, 8, 8, 8)
    net = libpeps.Network(16, 16, 2, 1, C.cast(bh, C.POINTER(C.c_int32)), C.cast(bv, C.POINTER(C.c_int32)),
                          C.cast(ptrs, C.POINTER(C.c_void_p)))
    opts = libpeps.make_opts(256, 16, 2, 1)
    need = C.c_size_t()
    assert lib.peps_boundary_workspace(C.byref(net), C.byref(net), C.byref(opts), C.byref(need)) == 0
    assert need.value > libpeps.STATIC_SCRATCH_BYTES
    la, ph = C.c_double(), C.c_double()
    r = lib.peps_boundary_contract_static(C.byref(net), C.byref(net), C.byref(opts), None,
                                          C.byref(la), C.byref(ph))
    assert r == 5
    msg = lib.peps_last_error().decode()
    assert str(need.value) in msg and str(libpeps.STATIC_SCRATCH_BYTES) in msg


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["4x4_D3_m6_plain", "8x8_D4_m32_mixed"])
def test_static_scratch_matches_caller_workspace(case):
    import torch
    from tests.gpu_util import to_dev
    if case.startswith("4x4"):
        ket = synth.random_peps(4, 4, 2, 3, "c64", "cgauss_scaled", 31)
        m, p, q, seed, prec = 6, 4, 1, 5, libpeps.PREC_PLAIN
    else:
        cfg = synth.config("c2")
        ket = synth.peps_for(cfg)
        m, p, q, seed, prec = cfg.m, cfg.p, cfg.q, cfg.omega_seed, libpeps.PREC_MIXED
    k = to_dev(ket, "c64")
    ref_la, ref_ph = libpeps.boundary_contract(k, k, m, p, q, seed, prec=prec)
    torch.cuda.synchronize()
    keys = ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current")
    for call in range(2):
        if call == 1:
            free0 = torch.cuda.mem_get_info()[0]
            st0 = torch.cuda.memory_stats()
        la, ph = libpeps.boundary_contract_static(k, k, m, p, q, seed, prec=prec)
        assert abs(la - ref_la) <= LOG_TOL * abs(ref_la), (call, la, ref_la)
        assert abs(ph - ref_ph) <= 1e-5, (call, ph, ref_ph)
    torch.cuda.synchronize()
    st1 = torch.cuda.memory_stats()
    assert torch.cuda.mem_get_info()[0] == free0
    assert [st1.get(x, 0) for x in keys] == [st0.get(x, 0) for x in keys]
