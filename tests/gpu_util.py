"""Shared helpers of the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np
import torch

TORCH_DT = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64,
            "c128": torch.complex128}


def to_dev(sites, dtype: str, dev="cuda:0"):
    return [[torch.tensor(np.asarray(T), dtype=TORCH_DT[dtype], device=dev).contiguous() for T in row]
            for row in sites]


def tensor(a, dtype: str, dev="cuda:0"):
    return torch.tensor(np.asarray(a), dtype=TORCH_DT[dtype], device=dev).contiguous()


def sigma_errors(gpu_sig, records):
    """Normwise max |sigma_i - sigma_i^ref| / sigma_1^ref per step."""
    errs = []
    pos = 0
    for r in records:
        s = np.asarray(r["sigma"])
        g = gpu_sig[pos:pos + len(s)]
        pos += len(s)
        errs.append(np.max(np.abs(g - s)) / max(s[0], 1e-300))
    assert pos == len(gpu_sig)
    return np.array(errs)
