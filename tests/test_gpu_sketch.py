"""The GPU's sketch draw (Algorithm 4's first line) element by element
against the oracle's Philox4x64-10 stream (itself pinned against NumPy's
Philox bit generator), for both stream tags (0: the sketch Omega, 1: the
gauge vector), both distributions, real and complex, single and double
precision.

A single-precision sketch rounds each 53-bit uniform once to FP32 (the
oracle's draw_elements(..., single=True) does the same in exact integer
arithmetic and evaluates the rest in FP64).  Uniform variant (2u - 1):
bit-exact in both precisions.  Normals (Box-Muller, a = r cos t,
b = r sin t with r = sqrt(-2 log u0), t = 2 pi u1): the GPU uses its own
log / sincospi in the working precision, so each value is held to 4 units
in the last place of the pair's scale |a| + r (an absolute bound where cos t
or sin t crosses zero)."""
import numpy as np
import pytest
import torch

from oracle import philox
from paper_2006_15234_gb300 import libpeps

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64, "c128": torch.complex128}


def _oracle(N, ell, seed, inst, tag, cplx, kind, single):
    return philox.draw_elements(N * ell, seed, inst, tag, cplx, kind, single=single).reshape(ell, N)


def _scale(ref, cplx):
    """|a| + r per value, r the modulus of the Box-Muller pair."""
    if cplx:
        # a complex value is one pair (a + i b)/sqrt 2
        r = np.abs(ref) * np.sqrt(2.0)
        return np.abs(ref.real) * np.sqrt(2.0) + r, np.abs(ref.imag) * np.sqrt(2.0) + r
    flat = ref.reshape(-1)
    pad = np.concatenate([flat, np.zeros((-len(flat)) % 2)])
    pr = pad.reshape(-1, 2)
    r = np.repeat(np.hypot(pr[:, 0], pr[:, 1]), 2)[: len(flat)]
    return (np.abs(flat) + r).reshape(ref.shape), None


@pytest.mark.parametrize("dt", ["f32", "f64", "c64", "c128"])
@pytest.mark.parametrize("tag", [0, 1])
@pytest.mark.parametrize("kind", ["gauss", "uniform"])
def test_sketch_matches_oracle_stream(dt, tag, kind):
    N, ell, seed, inst = 1237, 19, 20200617, (1 << 32) | (3 << 16) | 5     # ragged: N*ell not a multiple of 4
    cplx = dt.startswith("c")
    kcode = libpeps.SKETCH_GAUSS if kind == "gauss" else libpeps.SKETCH_UNIFORM
    got = libpeps.debug_sketch(N, ell, seed, inst, DT[dt], tag, kcode).cpu().numpy()
    double = dt in ("f64", "c128")
    ref = _oracle(N, ell, seed, inst, tag, cplx, kind, not double)
    eps = np.finfo(np.float64 if double else np.float32).eps
    parts = [(got.real, ref.real), (got.imag, ref.imag)] if cplx else [(got, ref)]
    if kind == "uniform":
        for g, r in parts:
            # 2 u - 1 is exact in FP64 and rounded once to FP32 on both sides
            assert np.array_equal(g, r.astype(g.dtype))
        return
    sa, sb = _scale(ref, cplx)
    scales = [sa, sb] if cplx else [sa]
    for (g, r), sc in zip(parts, scales):
        if cplx:
            sc = sc / np.sqrt(2.0)
        err = np.abs(g.astype(np.float64) - r) / (eps * sc)
        assert err.max() <= 4.0, err.max()


def test_sketch_streams_differ_by_instance_and_tag():
    a = libpeps.debug_sketch(64, 4, 7, 1, torch.float64, 0).cpu().numpy()
    b = libpeps.debug_sketch(64, 4, 7, 2, torch.float64, 0).cpu().numpy()
    c = libpeps.debug_sketch(64, 4, 7, 1, torch.float64, 1).cpu().numpy()
    assert not np.allclose(a, b) and not np.allclose(a, c)
