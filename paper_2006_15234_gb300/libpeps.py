"""ctypes binding of libpeps (argument marshalling only).

Every function here forwards to an ``extern "C"`` entry point declared in
``include/libpeps.h``; tensors are PyTorch CUDA tensors passed by pointer,
streams are ``torch.cuda.Stream`` handles.  Importing this module does not
need a GPU; calling into the library does.  There is no CPU fallback: if
the shared library is missing the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

__all__ = [
    "PepsError", "load", "lib_path", "RsvdOpts", "EinsumsvdShape", "EinsumsvdIO",
    "Network", "ContractPlan", "EinsumsvdPlan", "boundary_contract", "dtype_code",
    "EXPORTED_SYMBOLS", "PREC_PLAIN", "PREC_MIXED", "PREC_FAST", "SKETCH_GAUSS", "SKETCH_UNIFORM",
    "debug_tc_gemm", "FLAG_ORTH_Q", "boundary_contract_static", "STATIC_SCRATCH_BYTES",
    "Term", "ExpectationPlan", "expectation", "Cotangent", "Grads", "einsumsvd_grad", "GradPlan",
    "energy_grad", "peps_energy", "STATUS_NONFINITE", "STATUS_JACOBI_NOCONV", "STATUS_TIMEOUT",
    "ERR_NUMERIC", "ERR_TIMEOUT", "FLAG_FP64_SMALL", "FLAG_ALTERNATE", "FLAG_UNIT_BOND",
]

PREC_PLAIN, PREC_MIXED, PREC_FAST = 0, 1, 2
SKETCH_GAUSS, SKETCH_UNIFORM = 0, 1

EXPORTED_SYMBOLS = [
    "peps_status_string", "peps_last_error", "peps_version",
    "peps_einsumsvd_plan", "peps_einsumsvd_rank", "peps_einsumsvd_execute", "peps_plan_destroy",
    "peps_contract_plan", "peps_contract_execute", "peps_contract_result",
    "peps_contract_sigma_count", "peps_boundary_contract", "peps_boundary_workspace",
    "peps_plan_launch_count", "peps_plan_launch_info", "peps_plan_profile", "peps_plan_validate",
    "peps_debug_tc_gemm", "peps_boundary_contract_static",
    "peps_expectation_plan", "peps_expectation_execute", "peps_expectation_result",
    "peps_expectation_workspace", "peps_expectation", "peps_plan_launch_kernel",
    "peps_plan_kernel_launches", "peps_einsumsvd_grad_plan", "peps_einsumsvd_grad_bind",
    "peps_einsumsvd_grad_execute", "peps_grad_plan", "peps_grad_execute", "peps_grad",
    "peps_poll", "peps_plan_set_wait_limit", "peps_debug_sketch",
    "peps_plan_autotune", "peps_plan_tune_table", "peps_plan_set_tune_table", "peps_einsumsvd_set_branches",
    "peps_tebd_plan", "peps_tebd_execute", "peps_expectation_env_region", "peps_expectation_execute_part",
]

# Bits of a plan's device status word (peps_poll).
STATUS_NONFINITE, STATUS_JACOBI_NOCONV, STATUS_TIMEOUT = 1, 2, 4
# Status codes the synchronising calls return for them.
ERR_NUMERIC, ERR_TIMEOUT = 6, 7

# Size of the library's fixed device scratch used by boundary_contract_static.
STATIC_SCRATCH_BYTES = 32 << 20

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.environ.get("LIBPEPS_PATH", os.path.join(_HERE, "_build", "libpeps.so"))


class PepsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class RsvdOpts(C.Structure):
    _fields_ = [("m", C.c_int32), ("p", C.c_int32), ("q", C.c_int32), ("seed", C.c_uint64),
                ("sketch", C.c_int32), ("prec", C.c_int32), ("flags", C.c_uint32)]


class EinsumsvdShape(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("kL", "t", "a", "b", "d", "Dl", "Du", "Dx", "De", "DL", "DU", "DX", "DE", "m")]


class EinsumsvdIO(C.Structure):
    _fields_ = [("V", C.c_void_p), ("S", C.c_void_p), ("ket", C.c_void_p), ("bra", C.c_void_p),
                ("U", C.c_void_p), ("W", C.c_void_p), ("sigma", C.c_void_p),
                ("log_scale", C.c_void_p)]


class Network(C.Structure):
    _fields_ = [("nrow", C.c_int32), ("ncol", C.c_int32), ("d", C.c_int32), ("dtype", C.c_int32),
                ("bond_h", C.POINTER(C.c_int32)), ("bond_v", C.POINTER(C.c_int32)),
                ("site", C.POINTER(C.c_void_p))]


class Cotangent(C.Structure):
    _fields_ = [("U_bar", C.c_void_p), ("W_bar", C.c_void_p), ("log_scale_bar", C.c_void_p)]


class Grads(C.Structure):
    _fields_ = [("V_bar", C.c_void_p), ("S_bar", C.c_void_p), ("ket_bar", C.c_void_p), ("bra_bar", C.c_void_p)]


class Term(C.Structure):
    _fields_ = [("nsite", C.c_int32), ("site", C.c_int32 * 2), ("op", C.POINTER(C.c_double)),
                ("coeff", C.c_double)]


_lib = None


def load():
    """Load libpeps.so (built in-tree by ``build.build_library``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise PepsError(-1, f"libpeps.so not found at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    st = C.c_int32
    vp = C.c_void_p
    lib.peps_status_string.restype = C.c_char_p
    lib.peps_status_string.argtypes = [st]
    lib.peps_last_error.restype = C.c_char_p
    lib.peps_version.restype = C.c_char_p
    lib.peps_einsumsvd_plan.restype = st
    lib.peps_einsumsvd_plan.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32, C.POINTER(EinsumsvdShape),
                                        C.POINTER(C.c_uint64), C.POINTER(RsvdOpts), C.POINTER(C.c_size_t)]
    lib.peps_einsumsvd_rank.restype = st
    lib.peps_einsumsvd_rank.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    lib.peps_einsumsvd_execute.restype = st
    lib.peps_einsumsvd_execute.argtypes = [vp, C.POINTER(EinsumsvdIO), vp, C.c_size_t, vp]
    lib.peps_plan_destroy.restype = st
    lib.peps_plan_destroy.argtypes = [vp]
    lib.peps_contract_plan.restype = st
    lib.peps_contract_plan.argtypes = [C.POINTER(vp), C.POINTER(Network), C.POINTER(Network),
                                       C.POINTER(RsvdOpts), C.c_int32, C.POINTER(C.c_size_t)]
    lib.peps_contract_execute.restype = st
    lib.peps_contract_execute.argtypes = [vp, vp, C.c_size_t, vp]
    lib.peps_contract_result.restype = st
    lib.peps_contract_result.argtypes = [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]
    lib.peps_contract_sigma_count.restype = st
    lib.peps_contract_sigma_count.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.peps_boundary_contract.restype = st
    lib.peps_boundary_contract.argtypes = [C.POINTER(Network), C.POINTER(Network), C.POINTER(RsvdOpts),
                                           vp, C.c_size_t, vp, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]
    lib.peps_boundary_workspace.restype = st
    lib.peps_boundary_workspace.argtypes = [C.POINTER(Network), C.POINTER(Network), C.POINTER(RsvdOpts),
                                            C.POINTER(C.c_size_t)]
    lib.peps_plan_launch_count.restype = st
    lib.peps_plan_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.peps_plan_launch_info.restype = st
    lib.peps_plan_launch_info.argtypes = [vp, C.c_int64, C.POINTER(C.c_char_p),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.peps_plan_kernel_launches.restype = st
    lib.peps_plan_kernel_launches.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.peps_plan_launch_kernel.restype = st
    lib.peps_plan_launch_kernel.argtypes = [vp, C.c_int64, C.POINTER(C.c_char_p)]
    lib.peps_plan_profile.restype = st
    lib.peps_plan_profile.argtypes = [vp, vp, C.c_size_t, vp, C.POINTER(C.c_double)]
    lib.peps_debug_tc_gemm.restype = st
    lib.peps_debug_tc_gemm.argtypes = [C.c_int32] * 7 + [vp, vp, vp, vp, vp]
    lib.peps_plan_validate.restype = st
    lib.peps_plan_validate.argtypes = [vp, vp, C.c_size_t, C.POINTER(EinsumsvdIO)]
    lib.peps_grad_plan.restype = st
    lib.peps_grad_plan.argtypes = [C.POINTER(vp), C.POINTER(Network), C.POINTER(Term), C.c_int32,
                                   C.POINTER(RsvdOpts), C.POINTER(C.c_size_t)]
    lib.peps_grad_execute.restype = st
    lib.peps_grad_execute.argtypes = [vp, C.POINTER(vp), vp, C.c_size_t, vp, C.POINTER(C.c_double)]
    lib.peps_grad.restype = st
    lib.peps_grad.argtypes = [C.POINTER(Network), C.POINTER(Term), C.c_int32, C.POINTER(RsvdOpts), C.POINTER(vp),
                              vp, C.c_size_t, vp, C.POINTER(C.c_double)]
    lib.peps_einsumsvd_grad_plan.restype = st
    lib.peps_einsumsvd_grad_plan.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(EinsumsvdShape),
                                             C.POINTER(RsvdOpts), C.POINTER(C.c_size_t)]
    lib.peps_einsumsvd_grad_bind.restype = st
    lib.peps_einsumsvd_grad_bind.argtypes = [vp, C.POINTER(Cotangent), C.POINTER(Grads)]
    lib.peps_einsumsvd_grad_execute.restype = st
    lib.peps_einsumsvd_grad_execute.argtypes = [vp, C.POINTER(EinsumsvdIO), C.POINTER(Cotangent),
                                                C.POINTER(Grads), vp, C.c_size_t, vp]
    lib.peps_expectation_plan.restype = st
    lib.peps_expectation_plan.argtypes = [C.POINTER(vp), C.POINTER(Network), C.POINTER(Term), C.c_int32,
                                          C.POINTER(RsvdOpts), C.c_int32, C.POINTER(C.c_size_t)]
    lib.peps_expectation_execute.restype = st
    lib.peps_expectation_execute.argtypes = [vp, vp, C.c_size_t, vp]
    lib.peps_expectation_result.restype = st
    lib.peps_expectation_result.argtypes = [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
    lib.peps_expectation_workspace.restype = st
    lib.peps_expectation_workspace.argtypes = [C.POINTER(Network), C.POINTER(Term), C.c_int32,
                                               C.POINTER(RsvdOpts), C.c_int32, C.POINTER(C.c_size_t)]
    lib.peps_expectation.restype = st
    lib.peps_expectation.argtypes = [C.POINTER(Network), C.POINTER(Term), C.c_int32, C.POINTER(RsvdOpts),
                                     C.c_int32, vp, C.c_size_t, vp, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]
    lib.peps_boundary_contract_static.restype = st
    lib.peps_boundary_contract_static.argtypes = [C.POINTER(Network), C.POINTER(Network),
                                                  C.POINTER(RsvdOpts), vp, C.POINTER(C.c_double),
                                                  C.POINTER(C.c_double)]
    lib.peps_debug_sketch.restype = st
    lib.peps_debug_sketch.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_uint64, C.c_uint64, C.c_int32,
                                      C.c_int32, vp, vp, vp]
    lib.peps_expectation_env_region.restype = st
    lib.peps_expectation_env_region.argtypes = [vp, C.c_int32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    lib.peps_expectation_execute_part.restype = st
    lib.peps_expectation_execute_part.argtypes = [vp, vp, C.c_size_t, vp, C.c_int32]
    lib.peps_tebd_plan.restype = st
    lib.peps_tebd_plan.argtypes = [C.POINTER(vp), C.POINTER(Network), C.POINTER(C.c_double), C.c_int64,
                                   C.POINTER(C.c_double), C.c_int64, C.POINTER(RsvdOpts), C.POINTER(C.c_size_t)]
    lib.peps_tebd_execute.restype = st
    lib.peps_tebd_execute.argtypes = [vp, vp, C.c_size_t, vp]
    lib.peps_einsumsvd_set_branches.restype = st
    lib.peps_einsumsvd_set_branches.argtypes = [vp, C.c_int32, C.POINTER(C.c_size_t)]
    lib.peps_plan_autotune.restype = st
    lib.peps_plan_autotune.argtypes = [vp, vp, C.c_size_t, vp, C.c_int32]
    lib.peps_plan_tune_table.restype = st
    lib.peps_plan_tune_table.argtypes = [vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
    lib.peps_plan_set_tune_table.restype = st
    lib.peps_plan_set_tune_table.argtypes = [vp, C.c_char_p]
    lib.peps_poll.restype = st
    lib.peps_poll.argtypes = [vp, vp, vp, C.POINTER(C.c_uint32)]
    lib.peps_plan_set_wait_limit.restype = st
    lib.peps_plan_set_wait_limit.argtypes = [vp, C.c_uint64]
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        lib = load()
        raise PepsError(status, f"{lib.peps_status_string(status).decode()}: "
                                f"{lib.peps_last_error().decode()}")


def dtype_code(dtype) -> int:
    import torch
    return {torch.float32: 0, torch.complex64: 1, torch.float64: 2, torch.complex128: 3}[dtype]


FLAG_ORTH_Q = 1
FLAG_FP64_SMALL = 2
FLAG_ALTERNATE = 4
FLAG_UNIT_BOND = 8


def make_opts(m, p, q, seed, sketch=SKETCH_GAUSS, prec=PREC_PLAIN, flags=0) -> RsvdOpts:
    return RsvdOpts(int(m), int(p), int(q), int(seed) & (2 ** 64 - 1), int(sketch), int(prec), int(flags))


__all__.append("make_opts")


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _workspace(nbytes: int, device):
    import torch
    buf = torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


@dataclass
class _NetHolder:
    net: Network
    keep: list


def _network(sites, d=None) -> _NetHolder:
    """sites: list of rows of CUDA tensors [d][left][up][down][right]."""
    nrow, ncol = len(sites), len(sites[0])
    t0 = sites[0][0]
    dt = dtype_code(t0.dtype)
    for row in sites:
        for t in row:
            if not t.is_cuda or not t.is_contiguous() or t.dim() != 5 or t.dtype != t0.dtype:
                raise PepsError(1, "site tensors must be contiguous 5-d CUDA tensors of one dtype")
    bh = (C.c_int32 * max(1, nrow * (ncol - 1)))()
    bv = (C.c_int32 * max(1, (nrow - 1) * ncol))()
    for p in range(nrow):
        for q in range(ncol - 1):
            bh[p * (ncol - 1) + q] = sites[p][q].shape[4]
    for p in range(nrow - 1):
        for q in range(ncol):
            bv[p * ncol + q] = sites[p][q].shape[3]
    ptrs = (C.c_void_p * (nrow * ncol))(*[sites[p][q].data_ptr() for p in range(nrow)
                                          for q in range(ncol)])
    net = Network(nrow, ncol, int(t0.shape[0] if d is None else d), dt,
                  C.cast(bh, C.POINTER(C.c_int32)), C.cast(bv, C.POINTER(C.c_int32)),
                  C.cast(ptrs, C.POINTER(C.c_void_p)))
    return _NetHolder(net, [bh, bv, ptrs, sites])


class _Ledger:
    def poll(self, stream=None):
        """(status code, status word) of the last execute, after a synchronisation."""
        w = C.c_uint32()
        r = self._lib.peps_poll(self._plan, C.c_void_p(self._ws), _stream_handle(stream), C.byref(w))
        return r, w.value

    def autotune(self, reps: int = 3, stream=None):
        """Time every candidate MMA width per tensor-core GEMM shape and keep
        the fastest (execute the plan once before, and once more before a
        graph capture)."""
        _check(self._lib.peps_plan_autotune(self._plan, C.c_void_p(self._ws), C.c_size_t(self.workspace_bytes),
                                            _stream_handle(stream), int(reps)))

    def tune_table(self) -> str:
        n = C.c_size_t()
        _check(self._lib.peps_plan_tune_table(self._plan, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self._lib.peps_plan_tune_table(self._plan, buf, n.value, C.byref(n)))
        return buf.value.decode()

    def set_tune_table(self, text: str):
        _check(self._lib.peps_plan_set_tune_table(self._plan, text.encode()))

    def set_wait_limit(self, ns: int):
        """Limit (ns) of one tensor-core pipeline wait for later executes; 0: default."""
        _check(self._lib.peps_plan_set_wait_limit(self._plan, int(ns)))

    def launch_count(self) -> int:
        n = C.c_int64()
        _check(self._lib.peps_plan_launch_count(self._plan, C.byref(n)))
        return n.value

    def launches(self):
        """[(stage tag, algorithmic flops, algorithmic bytes)] per kernel launch."""
        out = []
        for i in range(self.launch_count()):
            tag, fl, by = C.c_char_p(), C.c_double(), C.c_double()
            _check(self._lib.peps_plan_launch_info(self._plan, i, C.byref(tag), C.byref(fl),
                                                   C.byref(by)))
            out.append((tag.value.decode(), fl.value, by.value))
        return out

    def kernel_launches(self):
        """CUDA kernel launches of one execute."""
        n = C.c_int64()
        _check(self._lib.peps_plan_kernel_launches(self._plan, C.byref(n)))
        return n.value

    def kernels(self):
        """Kernel family of every launch ("tc_gemm", "chol", ...)."""
        out = []
        for i in range(self.launch_count()):
            k = C.c_char_p()
            _check(self._lib.peps_plan_launch_kernel(self._plan, i, C.byref(k)))
            out.append(k.value.decode())
        return out

    def profile(self, stream=None):
        """Device time (ms) of every launch of one more execute."""
        import numpy as np
        n = self.launch_count()
        ms = np.zeros(max(n, 1), dtype=np.float64)
        _check(self._lib.peps_plan_profile(self._plan, C.c_void_p(self._ws),
                                           C.c_size_t(self.workspace_bytes), _stream_handle(stream),
                                           ms.ctypes.data_as(C.POINTER(C.c_double))))
        return ms[:n]


class ContractPlan(_Ledger):
    """Boundary-MPS contraction plan (Algorithms 2 and 3) with its workspace."""

    def __init__(self, ket, bra, opts: RsvdOpts, direction: int = 0):
        import torch
        self._lib = load()
        self._ket = _network(ket)
        self._bra = _network(bra) if bra is not None else None
        self._opts = opts
        plan = C.c_void_p()
        ws = C.c_size_t()
        _check(self._lib.peps_contract_plan(C.byref(plan), C.byref(self._ket.net),
                                            C.byref(self._bra.net) if self._bra else None,
                                            C.byref(opts), int(direction), C.byref(ws)))
        self._plan = plan
        self.workspace_bytes = ws.value
        self._buf, self._ws = _workspace(ws.value, ket[0][0].device)
        n = C.c_int64()
        _check(self._lib.peps_contract_sigma_count(plan, C.byref(n)))
        self.sigma_count = n.value

    def execute(self, stream=None):
        _check(self._lib.peps_contract_execute(self._plan, C.c_void_p(self._ws),
                                               C.c_size_t(self.workspace_bytes),
                                               _stream_handle(stream)))

    def result(self, stream=None, with_sigma=False):
        import numpy as np
        la, ph = C.c_double(), C.c_double()
        sig = np.zeros(max(1, self.sigma_count), dtype=np.float64) if with_sigma else None
        _check(self._lib.peps_contract_result(
            self._plan, C.c_void_p(self._ws), _stream_handle(stream), C.byref(la), C.byref(ph),
            sig.ctypes.data_as(C.POINTER(C.c_double)) if with_sigma else None))
        if with_sigma:
            return la.value, ph.value, sig[: self.sigma_count]
        return la.value, ph.value

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                self._lib.peps_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass


class EinsumsvdPlan(_Ledger):
    """Batched einsumsvd plan (one zip-up step per instance)."""

    def __init__(self, dtype, shapes, opts: RsvdOpts, instance_ids=None, device="cuda"):
        self._lib = load()
        n = len(shapes)
        arr = (EinsumsvdShape * n)(*[EinsumsvdShape(*s) for s in shapes])
        ids = None
        if instance_ids is not None:
            ids = (C.c_uint64 * n)(*[int(x) for x in instance_ids])
        plan = C.c_void_p()
        ws = C.c_size_t()
        _check(self._lib.peps_einsumsvd_plan(C.byref(plan), dtype_code(dtype), n, arr, ids,
                                             C.byref(opts), C.byref(ws)))
        self._plan = plan
        self.batch = n
        self.workspace_bytes = ws.value
        self._buf, self._ws = _workspace(ws.value, device)
        self.ranks = []
        for i in range(n):
            k = C.c_int32()
            _check(self._lib.peps_einsumsvd_rank(plan, i, C.byref(k)))
            self.ranks.append(k.value)

    def set_branches(self, n: int, device="cuda"):
        """Side streams of the tensor-core chains; reallocates the workspace."""
        ws = C.c_size_t()
        _check(self._lib.peps_einsumsvd_set_branches(self._plan, int(n), C.byref(ws)))
        self.workspace_bytes = ws.value
        self._buf = None
        self._buf, self._ws = _workspace(ws.value, device)

    def execute(self, io_list, stream=None):
        """io_list: per instance (V, S, ket, bra, U, W, sigma, log_scale) tensors."""
        arr = (EinsumsvdIO * self.batch)()
        for i, io in enumerate(io_list):
            arr[i] = EinsumsvdIO(*[t.data_ptr() if t is not None else None for t in io])
        self._keep = (arr, io_list)
        _check(self._lib.peps_einsumsvd_execute(self._plan, arr, C.c_void_p(self._ws),
                                                C.c_size_t(self.workspace_bytes),
                                                _stream_handle(stream)))

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                self._lib.peps_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass


class TebdPlan(_Ledger):
    """One TEBD layer (one-site operators by Eq. 4, then Algorithm 1 on every
    bond) applied in place to the PEPS `sites` (CUDA tensors).

    gates: one (d^2, d^2) host array for every bond, or a list in bond order
    (horizontal bonds by left site, then vertical bonds by upper site, both
    row-major); site_gates: None, one (d, d) array, or a row-major list per
    site; unit: normalise every new bond by its largest singular value."""

    def __init__(self, sites, gates, seed, unit=False, site_gates=None):
        import numpy as np
        self._lib = load()
        self._net = _network(sites)
        cplx = sites[0][0].is_complex()
        dt = np.complex128 if cplx else np.float64

        def pack(ops):
            a = np.ascontiguousarray(np.stack([np.asarray(o, dtype=dt) for o in ops]))
            return np.ascontiguousarray(a.view(np.float64)) if cplx else a
        glist = list(gates) if isinstance(gates, (list, tuple)) else [gates]
        self._gate = pack(glist)
        slist = [] if site_gates is None else (list(site_gates) if isinstance(site_gates, (list, tuple))
                                               else [site_gates])
        self._site_gate = pack(slist) if slist else None
        sp = (self._site_gate.ctypes.data_as(C.POINTER(C.c_double)) if slist
              else C.cast(None, C.POINTER(C.c_double)))
        plan = C.c_void_p()
        ws = C.c_size_t()
        _check(self._lib.peps_tebd_plan(C.byref(plan), C.byref(self._net.net),
                                        self._gate.ctypes.data_as(C.POINTER(C.c_double)), len(glist),
                                        sp, len(slist),
                                        C.byref(make_opts(1, 0, 0, seed, flags=FLAG_UNIT_BOND if unit else 0)),
                                        C.byref(ws)))
        self._plan = plan
        self.workspace_bytes = ws.value
        self._buf, self._ws = _workspace(ws.value, sites[0][0].device)

    def execute(self, stream=None):
        _check(self._lib.peps_tebd_execute(self._plan, C.c_void_p(self._ws), C.c_size_t(self.workspace_bytes),
                                           _stream_handle(stream)))

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                self._lib.peps_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass


def tebd_layer(sites, gates, seed, stream=None, unit=False, site_gates=None):
    """Apply the one-site operators, then the two-site operators to every
    bond of the PEPS, in place."""
    plan = TebdPlan(sites, gates, seed, unit, site_gates)
    plan.execute(stream)
    return plan


def cuda_graph(fn):
    """Capture fn() -- enqueue-only calls of plans that have executed once
    already (so their descriptors are resident) -- into a CUDA graph on a side
    stream; graph.replay() re-enqueues the whole recorded work with one launch
    on the current stream."""
    import torch
    g = torch.cuda.CUDAGraph()
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            fn()
    cur.wait_stream(side)
    return g


__all__.append("cuda_graph")


def exchange_env_regions(plan_views, group=None):
    """The collective of the two-GPU expectation split: rank r (0 or 1) has
    filled its own part's region (plan_views[r], a uint8 tensor); after the
    call both regions hold the owners' bytes on every rank.  One broadcast
    per part from its owner; nothing else crosses ranks."""
    import torch.distributed as dist
    for part, view in enumerate(plan_views):
        dist.broadcast(view, src=part, group=group)


__all__.append("exchange_env_regions")


def expectation_split(plan, rank, group=None, stream=None):
    """Cached expectation on two ranks (one GPU each, identical plans): rank
    r runs the sweeps of part r, the regions are exchanged, both run the
    strips; returns the result on every rank."""
    plan.execute_part(rank, stream)
    import torch
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    exchange_env_regions([plan.env_view(0), plan.env_view(1)], group)
    plan.execute_part(2, stream)
    return plan.result(stream)


__all__.append("expectation_split")


class IteDriver:
    """Imaginary-time evolution (Sec. II-D) of the PEPS `sites` in place:
    every step is one TEBD layer of exp(-tau H_j) (bond_gates, site_gates;
    bonds normalised by their largest singular value) followed by the
    Rayleigh quotient of `terms` (Eq. 6, cached environments) with the
    contraction options `opts`.  Both plans are built once: the layer keeps
    every bond dimension, so the expectation plan reads the updated sites."""

    def __init__(self, sites, bond_gates, site_gates, terms, opts: RsvdOpts, seed):
        self.tebd = TebdPlan(sites, bond_gates, seed, unit=True, site_gates=site_gates)
        self.expect = ExpectationPlan(sites, terms, opts)

        self.graph = None

    def step(self, stream=None):
        """Enqueue one ITE step (no synchronisation); after capture(), one
        replay of the captured step."""
        if self.graph is not None:
            self.graph.replay()
            return
        self.tebd.execute(stream)
        self.expect.execute(stream)

    def capture(self):
        """Record one step as a CUDA graph (runs one plain step first so the
        descriptors are resident); later steps replay it."""
        import torch
        self.step()
        torch.cuda.synchronize()
        self.graph = cuda_graph(lambda: (self.tebd.execute(), self.expect.execute()))
        return self.graph

    def run(self, steps, stream=None, every=1):
        """Energy after every `every`-th of `steps` steps and after the last
        (Sec. II-D evaluates it for the final state only: every = steps);
        synchronises once per evaluation."""
        out = []
        for i in range(steps):
            if self.graph is None and (i + 1) % every != 0 and i + 1 != steps:
                self.tebd.execute(stream)       # evolution only
                continue
            self.step(stream)
            out.append(self.expect.result(stream)[0])
        return out


__all__ += ["TebdPlan", "tebd_layer", "IteDriver"]


def boundary_contract(ket, bra, m, p, q, seed, sketch=SKETCH_GAUSS, prec=PREC_PLAIN,
                      direction=0, with_sigma=False, stream=None, flags=0):
    """Contract <bra|ket> (or the one-layer ket when bra is None) on the GPU.

    Returns (log|v|, arg v) [and the per-step singular values]."""
    plan = ContractPlan(ket, bra, make_opts(m, p, q, seed, sketch, prec, flags), direction)
    plan.execute(stream)
    return plan.result(stream, with_sigma)


class ExpectationPlan(_Ledger):
    """<psi|H|psi>/<psi|psi> with cached environments (Eq. 6, Sec. IV-B).

    terms: [(sites, op, coeff)]; sites = ((p, q),) or ((p0, q0), (p1, q1)) on a
    nearest-neighbour bond; op a (d^n x d^n) array (host)."""

    def __init__(self, ket, terms, opts: RsvdOpts, use_cache=True):
        import numpy as np
        self._lib = load()
        self._ket = _network(ket)
        ncol = len(ket[0])
        cplx = ket[0][0].is_complex()
        n = len(terms)
        self._tarr = (Term * max(1, n))()
        self._keep = []
        for i, (st, op, coeff) in enumerate(terms):
            a = np.ascontiguousarray(np.asarray(op, dtype=np.complex128 if cplx else np.float64))
            if cplx:
                a = np.ascontiguousarray(a.view(np.float64))
            self._keep.append(a)
            t = self._tarr[i]
            t.nsite = len(st)
            for k, (p, q) in enumerate(st):
                t.site[k] = p * ncol + q
            t.op = a.ctypes.data_as(C.POINTER(C.c_double))
            t.coeff = float(coeff)
        self.nterms = n
        plan = C.c_void_p()
        ws = C.c_size_t()
        _check(self._lib.peps_expectation_plan(C.byref(plan), C.byref(self._ket.net), self._tarr, n,
                                               C.byref(opts), int(bool(use_cache)), C.byref(ws)))
        self._plan = plan
        self.workspace_bytes = ws.value
        self._buf, self._ws = _workspace(ws.value, ket[0][0].device)

    def execute(self, stream=None):
        _check(self._lib.peps_expectation_execute(self._plan, C.c_void_p(self._ws),
                                                  C.c_size_t(self.workspace_bytes), _stream_handle(stream)))

    def execute_part(self, part, stream=None):
        """Enqueue one part of the two-GPU split: 0 top-down sweeps, 1
        bottom-up sweeps, 2 strips (needs both parts' environments)."""
        _check(self._lib.peps_expectation_execute_part(self._plan, C.c_void_p(self._ws),
                                                       C.c_size_t(self.workspace_bytes), _stream_handle(stream),
                                                       int(part)))

    def env_region(self, part):
        """(byte offset, bytes) of a sweep part's environments in the workspace."""
        off, n = C.c_size_t(), C.c_size_t()
        _check(self._lib.peps_expectation_env_region(self._plan, int(part), C.byref(off), C.byref(n)))
        return off.value, n.value

    def env_view(self, part):
        """uint8 CUDA tensor over a sweep part's region of the workspace (for
        the exchange between ranks)."""
        off, n = self.env_region(part)
        return self._buf.narrow(0, (self._ws - self._buf.data_ptr()) + off, n)

    def result(self, stream=None):
        """(energy, log <psi|psi>, per-term coeff_t <O_t>)."""
        import numpy as np
        e, ln = C.c_double(), C.c_double()
        tv = np.zeros(max(1, self.nterms), dtype=np.float64)
        _check(self._lib.peps_expectation_result(self._plan, C.c_void_p(self._ws), _stream_handle(stream),
                                                 C.byref(e), C.byref(ln),
                                                 tv.ctypes.data_as(C.POINTER(C.c_double))))
        return e.value, ln.value, tv[: self.nterms]

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                self._lib.peps_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass


class GradPlan(_Ledger):
    """Energy and its gradient with respect to every site tensor (real
    networks): terms as for ExpectationPlan."""

    def __init__(self, ket, terms, opts: RsvdOpts):
        import numpy as np
        self._lib = load()
        self._ket = _network(ket)
        self._sites = ket
        ncol = len(ket[0])
        n = len(terms)
        self._tarr = (Term * max(1, n))()
        self._keep = []
        for i, (st, op, coeff) in enumerate(terms):
            a = np.ascontiguousarray(np.asarray(op, dtype=np.float64))
            self._keep.append(a)
            t = self._tarr[i]
            t.nsite = len(st)
            for k, (p_, q_) in enumerate(st):
                t.site[k] = p_ * ncol + q_
            t.op = a.ctypes.data_as(C.POINTER(C.c_double))
            t.coeff = float(coeff)
        plan = C.c_void_p()
        ws = C.c_size_t()
        _check(self._lib.peps_grad_plan(C.byref(plan), C.byref(self._ket.net), self._tarr, n, C.byref(opts),
                                        C.byref(ws)))
        self._plan = plan
        self.workspace_bytes = ws.value
        self._buf, self._ws = _workspace(ws.value, ket[0][0].device)

    def execute(self, stream=None):
        """(energy, [[dE/d site]]) with gradients shaped like the sites."""
        import torch
        grads = [[torch.empty_like(t) for t in row] for row in self._sites]
        ptrs = (C.c_void_p * sum(len(r) for r in grads))(*[g.data_ptr() for r in grads for g in r])
        e = C.c_double()
        _check(self._lib.peps_grad_execute(self._plan, ptrs, C.c_void_p(self._ws), C.c_size_t(self.workspace_bytes),
                                           _stream_handle(stream), C.byref(e)))
        return e.value, grads

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                self._lib.peps_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass


def peps_energy(terms, m, p, q, seed, nrow, ncol, *sites):
    """torch.autograd entry: the energy of H = sum coeff * op for a real PEPS
    whose nrow x ncol site tensors are passed in row-major order; E.backward()
    returns dE/d(site) from the library's hand-written adjoint (peps_grad)."""
    return _PepsEnergy.apply(terms, m, p, q, seed, nrow, ncol, *sites)


def _make_energy_function():
    import torch

    class PepsEnergyFunction(torch.autograd.Function):
        @staticmethod
        def forward(ctx, terms, m, p, q, seed, nrow, ncol, *flat):
            sites = [[flat[r * ncol + c].contiguous() for c in range(ncol)] for r in range(nrow)]
            if not any(ctx.needs_input_grad[7:]):
                # no gradient wanted: the expectation value alone (no reverse sweep)
                e, _, _ = expectation(sites, terms, m, p, q, seed)
                return torch.tensor(e, dtype=torch.float64, device=flat[0].device)
            e, g = energy_grad(sites, terms, m, p, q, seed)
            ctx.save_for_backward(*[x for row in g for x in row])
            return torch.tensor(e, dtype=torch.float64, device=flat[0].device)

        @staticmethod
        def backward(ctx, gout):
            grads = ctx.saved_tensors
            scale = gout.to(grads[0].dtype)
            return (None, None, None, None, None, None, None) + tuple(g * scale for g in grads)

    return PepsEnergyFunction


class _LazyFunction:
    _f = None

    def apply(self, *args):
        if _LazyFunction._f is None:
            _LazyFunction._f = _make_energy_function()
        return _LazyFunction._f.apply(*args)


_PepsEnergy = _LazyFunction()


def energy_grad(ket, terms, m, p, q, seed, stream=None):
    """Energy of H = sum coeff * op and dE/d(site) on the GPU (real network)."""
    plan = GradPlan(ket, terms, make_opts(m, p, q, seed))
    return plan.execute(stream)


def expectation(ket, terms, m, p, q, seed, sketch=SKETCH_GAUSS, prec=PREC_PLAIN, use_cache=True,
                stream=None, flags=0):
    """Energy <psi|H|psi>/<psi|psi> of H = sum coeff * op on the GPU; returns
    (energy, log <psi|psi>, per-term values)."""
    plan = ExpectationPlan(ket, terms, make_opts(m, p, q, seed, sketch, prec, flags), use_cache)
    plan.execute(stream)
    return plan.result(stream)


def einsumsvd_grad(V, S, ket, bra, m, p, q, seed, U_bar, W_bar, log_scale_bar=0.0, stream=None):
    """One einsumsvd (real data) and its adjoint: returns (U, W, sigma,
    log sigma_1) and the cotangents (V_bar, S_bar, ket_bar, bra_bar) of
    L = <U_bar, U> + <W_bar, W> + log_scale_bar * log sigma_1."""
    import torch
    lib = load()
    kL, t, a, h = V.shape
    _, v, b = S.shape
    d, Dl, Du, Dx, De = ket.shape
    _, DL, DU, DX, DE = bra.shape
    shape = EinsumsvdShape(kL, t, a, b, d, Dl, Du, Dx, De, DL, DU, DX, DE, m)
    plan = C.c_void_p()
    ws = C.c_size_t()
    _check(lib.peps_einsumsvd_grad_plan(C.byref(plan), dtype_code(V.dtype), C.byref(shape),
                                        C.byref(make_opts(m, p, q, seed)), C.byref(ws)))
    try:
        k = C.c_int32()
        _check(lib.peps_einsumsvd_rank(plan, 0, C.byref(k)))
        k = k.value
        dev = V.device
        U = torch.empty((kL, t, k), dtype=V.dtype, device=dev)
        W = torch.empty((k, Dx * DX, b, De * DE), dtype=V.dtype, device=dev)
        sg = torch.empty(k, dtype=torch.float64, device=dev)
        lg = torch.empty(1, dtype=torch.float64, device=dev)
        lb = torch.tensor([float(log_scale_bar)], dtype=torch.float64, device=dev)
        gV, gS, gK, gKb = (torch.empty_like(x) for x in (V, S, ket, bra))
        buf, wsp = _workspace(ws.value, dev)
        io = EinsumsvdIO(V.data_ptr(), S.data_ptr(), ket.data_ptr(), bra.data_ptr(), U.data_ptr(),
                         W.data_ptr(), sg.data_ptr(), lg.data_ptr())
        ct = Cotangent(U_bar.data_ptr(), W_bar.data_ptr(), lb.data_ptr())
        gr = Grads(gV.data_ptr(), gS.data_ptr(), gK.data_ptr(), gKb.data_ptr())
        _check(lib.peps_einsumsvd_grad_execute(plan, C.byref(io), C.byref(ct), C.byref(gr), C.c_void_p(wsp),
                                               ws, _stream_handle(stream)))
        torch.cuda.synchronize(dev)
        return (U, W, sg, lg), (gV, gS, gK, gKb)
    finally:
        lib.peps_plan_destroy(plan)


def boundary_contract_static(ket, bra, m, p, q, seed, sketch=SKETCH_GAUSS, prec=PREC_PLAIN,
                             stream=None, flags=0):
    """boundary_contract without any device allocation: the workspace is the
    library's own fixed scratch array (STATIC_SCRATCH_BYTES per device), for
    callers that cannot allocate device memory.  Contractions needing more
    raise.  Calls on one device share the array, so calls that may overlap on
    the GPU must be serialised.  Returns (log|v|, arg v)."""
    lib = load()
    k = _network(ket)
    b = _network(bra) if bra is not None else None
    opts = make_opts(m, p, q, seed, sketch, prec, flags)
    la, ph = C.c_double(), C.c_double()
    _check(lib.peps_boundary_contract_static(C.byref(k.net), C.byref(b.net) if b else None, C.byref(opts),
                                             _stream_handle(stream), C.byref(la), C.byref(ph)))
    return la.value, ph.value


def debug_sketch(N, ell, seed, instance, dtype, tag=0, kind=SKETCH_GAUSS, device="cuda", stream=None):
    """The GPU's (instance, tag) Philox stream as an (ell, N) tensor of dtype
    (row j holds elements j*N .. j*N + N - 1)."""
    import torch
    lib = load()
    X = torch.empty((int(ell), int(N)), dtype=dtype, device=device)
    scratch = torch.empty(256, dtype=torch.uint8, device=device)
    _check(lib.peps_debug_sketch(dtype_code(dtype), int(N), int(ell), int(seed) & (2 ** 64 - 1),
                                 int(instance) & (2 ** 64 - 1), int(tag), int(kind), X.data_ptr(),
                                 scratch.data_ptr(), _stream_handle(stream)))
    return X


__all__.append("debug_sketch")


def debug_tc_gemm(A, B, conjA=False, conjB=False, split3=False, stream=None):
    """C = opA(A) @ opB(B)^T on the tensor-core GEMM (A: M x K, B: N x K).
    split3: False / 0 plain TF32, True / 1 3xTF32, 2 3xTF32 with B expanded
    and split beforehand (scratch allocated here)."""
    import torch
    lib = load()
    cplx = A.is_complex()
    M, K = A.shape
    N = B.shape[0]
    C_ = torch.empty((M, N), dtype=A.dtype, device=A.device)
    mode = int(split3)
    scratch = None
    if mode == 2:
        scratch = torch.empty((32 if cplx else 8) * N * K, dtype=torch.uint8, device=A.device)
    _check(lib.peps_debug_tc_gemm(int(cplx), int(conjA), int(conjB), mode, M, N, K,
                                  C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                  C.c_void_p(C_.data_ptr()),
                                  C.c_void_p(scratch.data_ptr() if scratch is not None else None),
                                  _stream_handle(stream)))
    if scratch is not None:
        torch.cuda.synchronize(A.device)     # scratch is released on return
    return C_
