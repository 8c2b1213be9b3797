"""Seeded synthetic PEPS workloads (no contraction arithmetic lives here).

Site tensors use the layout ``[d][left][up][down][right]`` (physical index
first, then the four bonds; edge bonds have dimension 1), which follows the
shared-bond pattern of the two-site update (Sec. II-C, Eq. 5) and the index
order of the zip-up start contraction (Algorithm 3).  Every array is drawn in
float64, then rounded to the storage precision of the GPU path; the returned
values are the rounded ones, widened again, so the oracle and the CUDA path
read bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "WorkloadConfig", "CONFIGS", "config", "site_shape", "random_peps",
    "round_to", "storage_numpy_dtype", "batched_instance", "batched_dims",
    "tfi_terms", "PAULI",
]

# Pauli matrices: inputs for the transverse-field Ising Hamiltonian terms.
PAULI = {
    "I": np.array([[1.0, 0.0], [0.0, 1.0]]),
    "X": np.array([[0.0, 1.0], [1.0, 0.0]]),
    "Y": np.array([[0.0, -1.0j], [1.0j, 0.0]]),
    "Z": np.array([[1.0, 0.0], [0.0, -1.0]]),
}


@dataclass(frozen=True)
class WorkloadConfig:
    name: str
    nrow: int
    ncol: int
    d: int
    D: int
    dtype: str            # storage/compute type of the GPU path: f32, f64, c64
    two_layer: bool       # True: norm <psi|psi>; False: one-layer scalar
    m: int                # boundary bond (truncation rank)
    p: int                # oversampling
    q: int                # power iterations
    dist: str             # value distribution (see _draw)
    seed: int
    omega_seed: int
    extra: dict = field(default_factory=dict)


_BASE_SEED = 20200615

CONFIGS = {
    # 4x4 one-layer scalar, physical index fixed (d=1), bond 2, N(0,1)/2.
    "c1": WorkloadConfig("c1_4x4_onelayer_D2_m4", 4, 4, 1, 2, "f64", False,
                         4, 4, 1, "normal_half", _BASE_SEED + 0, _BASE_SEED + 1),
    # 8x8 norm, complex64, d=2, bond 4, complex Gaussian / sqrt(2 d D^4).
    "c2": WorkloadConfig("c2_8x8_norm_c64_D4_m32", 8, 8, 2, 4, "c64", True,
                         32, 8, 2, "cgauss_scaled", _BASE_SEED + 1, _BASE_SEED + 2),
    # 512 independent einsumsvd instances (see batched_instance).
    "c3": WorkloadConfig("c3_batched512_f32", 0, 0, 2, 0, "f32", True,
                         0, 8, 2, "normal", _BASE_SEED + 2, _BASE_SEED + 3,
                         {"count": 512, "m_range": (16, 128), "D_range": (2, 6)}),
    # 6x6 TFI energy, real, d=2, bond 3, N(0,1)*0.1.
    "c4": WorkloadConfig("c4_6x6_tfi_f32_D3_m18", 6, 6, 2, 3, "f32", True,
                         18, 8, 2, "normal_tenth", _BASE_SEED + 3, _BASE_SEED + 4,
                         {"J": 1.0, "h": 3.0}),
    # 12x12 TFI expectation value, complex64, d=2, bond 4 (the cache-on /
    # cache-off study's shape, Sec. IV-B); boundary bond 16 = D^2.
    "f2": WorkloadConfig("f2_12x12_tfi_expectation_c64_D4_m16", 12, 12, 2, 4, "c64", True,
                         16, 8, 2, "cgauss_scaled", _BASE_SEED + 5, _BASE_SEED + 6,
                         {"J": 1.0, "h": 3.0}),
    # One TEBD layer (QR-SVD on every bond) of an imaginary-time TFI gate on a
    # 16x16, D=8 complex64 PEPS (the lattice of the 16x16 norm workload).
    "f1": WorkloadConfig("f1_16x16_tebd_layer_c64_D8", 16, 16, 2, 8, "c64", True,
                         8, 0, 0, "cgauss_fro", _BASE_SEED + 7, _BASE_SEED + 8,
                         {"J": 1.0, "h": 3.0, "tau": 0.01}),
    # Imaginary-time evolution of the transverse-field Ising model on an
    # 8x8, D=4 complex64 PEPS: one TEBD layer of exp(-tau H_j) then the
    # energy (m = 16 = D^2) per step.
    "f3": WorkloadConfig("f3_8x8_tfi_ite_c64_D4_m16", 8, 8, 2, 4, "c64", True,
                         16, 8, 2, "cgauss_scaled", _BASE_SEED + 9, _BASE_SEED + 10,
                         {"J": 1.0, "h": 3.0, "tau": 0.05}),
    # One-layer contraction of an 8x8 PEPS without physical index (d = 1), the
    # contraction bond equal to the initial bond (D = m; run for D = 2, 4, 8).
    "f4": WorkloadConfig("f4_8x8_onelayer_f32_D_eq_m", 8, 8, 1, 8, "f32", False,
                         8, 4, 2, "normal_half", _BASE_SEED + 11, _BASE_SEED + 12),
    # 16x16 norm, complex64, d=2, bond 8, per-tensor Frobenius-normalised.
    "c5": WorkloadConfig("c5_16x16_norm_c64_D8_m256", 16, 16, 2, 8, "c64", True,
                         256, 16, 2, "cgauss_fro", _BASE_SEED + 4, _BASE_SEED + 5),
}


def config(key: str) -> WorkloadConfig:
    return CONFIGS[key]


def storage_numpy_dtype(dtype: str):
    return {"f32": np.float32, "f64": np.float64,
            "c64": np.complex64, "c128": np.complex128}[dtype]


def round_to(a: np.ndarray, dtype: str) -> np.ndarray:
    """Round ``a`` to the storage precision ``dtype`` and widen it back to
    float64/complex128 so both sides see identical values."""
    r = np.asarray(a).astype(storage_numpy_dtype(dtype))
    return r.astype(np.complex128 if np.iscomplexobj(r) else np.float64)


def site_shape(nrow: int, ncol: int, p: int, q: int, d: int, D) -> tuple:
    """Shape [d][left][up][down][right] of site (p, q); edge bonds are 1.

    ``D`` is either one bond dimension for the whole lattice or a callable
    ``D(kind, p, q)`` giving the bond to the right ('h') or below ('v').
    """
    if callable(D):
        dl = D("h", p, q - 1) if q > 0 else 1
        dr = D("h", p, q) if q < ncol - 1 else 1
        du = D("v", p - 1, q) if p > 0 else 1
        dd = D("v", p, q) if p < nrow - 1 else 1
    else:
        dl = D if q > 0 else 1
        dr = D if q < ncol - 1 else 1
        du = D if p > 0 else 1
        dd = D if p < nrow - 1 else 1
    return (d, dl, du, dd, dr)


def _draw(rng: np.random.Generator, shape, dist: str, d: int, D: int) -> np.ndarray:
    if dist == "normal_half":
        return rng.standard_normal(shape) / 2.0
    if dist == "normal":
        return rng.standard_normal(shape)
    if dist == "normal_tenth":
        return rng.standard_normal(shape) * 0.1
    if dist == "cgauss_scaled":
        s = 1.0 / math.sqrt(2.0 * d * D ** 4)
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        return (re + 1j * im) * s
    if dist == "cgauss_fro":
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        z = re + 1j * im
        return z / np.linalg.norm(z.ravel())
    raise ValueError(dist)


def random_peps(nrow: int, ncol: int, d: int, D, dtype: str, dist: str,
                seed: int) -> list:
    """Site tensors ``sites[p][q]`` of an nrow x ncol PEPS.

    Each site is drawn from its own stream ``default_rng([seed, p, q])`` so a
    sub-lattice or a single site can be regenerated without the rest.
    """
    Dn = D if not callable(D) else 1
    out = []
    for p in range(nrow):
        row = []
        for q in range(ncol):
            rng = np.random.default_rng([seed, p, q])
            shp = site_shape(nrow, ncol, p, q, d, D)
            row.append(round_to(_draw(rng, shp, dist, d, Dn), dtype))
        out.append(row)
    return out


def peps_for(cfg: WorkloadConfig) -> list:
    return random_peps(cfg.nrow, cfg.ncol, cfg.d, cfg.D, cfg.dtype, cfg.dist,
                       cfg.seed)


__all__.append("peps_for")


def batched_dims(cfg: WorkloadConfig, count: int | None = None) -> list:
    """(m, D) of each batched einsumsvd instance: m ~ U{16..128}, D ~ U{2..6}
    (inclusive), drawn from one seeded stream."""
    n = cfg.extra["count"] if count is None else count
    rng = np.random.default_rng([cfg.seed, 0xB47C])
    lo, hi = cfg.extra["m_range"]
    dlo, dhi = cfg.extra["D_range"]
    ms = rng.integers(lo, hi + 1, size=cfg.extra["count"])
    Ds = rng.integers(dlo, dhi + 1, size=cfg.extra["count"])
    return [(int(ms[i]), int(Ds[i])) for i in range(n)]


def batched_instance(cfg: WorkloadConfig, i: int, m: int, D: int) -> dict:
    """One zip-up step operand set (Algorithm 3, einsumsvd line) of size m, D.

    carry V [m][D^2][m][D^2] (left, down pair of the previous column, old
    boundary bond, horizontal pair), old boundary site S [m][D^2][m],
    ket and bra [d][D][D][D][D]; real N(0,1) entries.
    """
    rng = np.random.default_rng([cfg.seed, 1, i])
    d = cfg.d
    R = D * D
    V = rng.standard_normal((m, R, m, R))
    S = rng.standard_normal((m, R, m))
    ket = rng.standard_normal((d, D, D, D, D))
    bra = rng.standard_normal((d, D, D, D, D))
    return {"V": round_to(V, cfg.dtype), "S": round_to(S, cfg.dtype),
            "ket": round_to(ket, cfg.dtype), "bra": round_to(bra, cfg.dtype),
            "m": m, "D": D, "d": d}


def tfi_terms(nrow: int, ncol: int, J: float, h: float) -> list:
    """Local terms of H = -J sum_<ij> Z_i Z_j - h sum_i X_i (open boundaries).

    Each term is (sites, op, coeff) with sites a tuple of (p, q) and op a
    d^n x d^n matrix whose row index is the outgoing physical pair.
    """
    Z, X = PAULI["Z"], PAULI["X"]
    ZZ = np.kron(Z, Z)
    terms = []
    for p in range(nrow):
        for q in range(ncol):
            if q + 1 < ncol:
                terms.append((((p, q), (p, q + 1)), ZZ, -J))
            if p + 1 < nrow:
                terms.append((((p, q), (p + 1, q)), ZZ, -J))
    for p in range(nrow):
        for q in range(ncol):
            terms.append((((p, q),), X, -h))
    return terms


def tfi_bond_gate(J: float, h: float, tau: float) -> np.ndarray:
    """exp(-tau h_ij) of one bond's share of the transverse-field Ising
    Hamiltonian, h_ij = -J Z_i Z_j - (h / 4) (X_i + X_j) (each site's field
    split over its four bonds): the two-site operator of one imaginary-time
    TEBD step, a 4 x 4 matrix [out pair][in pair] (an input, computed with
    scipy's matrix exponential)."""
    from scipy.linalg import expm
    Z, X, I = PAULI["Z"], PAULI["X"], PAULI["I"]
    hij = -J * np.kron(Z, Z) - (h / 4.0) * (np.kron(X, I) + np.kron(I, X))
    return expm(-tau * hij)


__all__.append("tfi_bond_gate")


def tfi_ite_gates(J: float, h: float, tau: float):
    """exp(-tau H_j) for the two kinds of local term of the transverse-field
    Ising Hamiltonian H = -J sum_<ij> Z_i Z_j - h sum_i X_i: the bond
    operator exp(tau J Z Z) (4 x 4, [out pair][in pair]) and the site
    operator exp(tau h X) (2 x 2), by scipy's matrix exponential (inputs)."""
    from scipy.linalg import expm
    Z, X = PAULI["Z"], PAULI["X"]
    return expm(tau * J * np.kron(Z, Z)), expm(tau * h * X)


__all__.append("tfi_ite_gates")
