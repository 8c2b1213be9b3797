"""Philox4x64-10 and the Gaussian sketch of Algorithm 4 (oracle side).

The generator follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4 x 64-bit counter,
a 2 x 64-bit key, ten rounds of two 64x64->128-bit multiplies with the
published multipliers, and a Weyl-sequence key schedule between rounds.

Sketch layout (the paper draws the start block Q of Algorithm 4 at random but
fixes neither generator nor layout; this is the library's reading):
  * block counter = (block, instance, tag, 0), key = (seed, 0);
  * element e of an N x l sketch is Omega[n, j] with e = j*N + n;
  * a block's four words x give uniforms u = ((x >> 11) + 0.5) * 2^-53;
  * Box-Muller on (u0,u1) and (u2,u3) gives normals n0..n3;
  * real sketch: element e is normal (e & 3) of block e >> 2;
  * complex sketch: element e is (n_{2c} + i n_{2c+1}) / sqrt(2) with
    c = e & 1 of block e >> 1;
  * the 'uniform' variant (the paper's [-1, 1] draw) uses 2u - 1 instead.
tag 0 draws sketches, tag 1 draws the gauge vector.
A single-precision sketch rounds each 53-bit uniform once to FP32 before it
is used (draw_elements(..., single=True)); the FP64 oracle itself draws with
the 53-bit uniforms.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
_MASK64 = (1 << 64) - 1

TAG_SKETCH = 0
TAG_GAUGE = 1


def philox4x64_scalar(counter, key):
    """One block, Python integers (reference for the vectorised version)."""
    c = [int(x) & _MASK64 for x in counter]
    k = [int(x) & _MASK64 for x in key]
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> 64, p0 & _MASK64
        hi1, lo1 = p1 >> 64, p1 & _MASK64
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        k = [(k[0] + W0) & _MASK64, (k[1] + W1) & _MASK64]
    return c


_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.uint64, b: np.ndarray):
    """Full 64x64 -> 128-bit product of a scalar and an array, as (hi, lo)."""
    a = np.uint64(a)
    a0, a1 = a & _M32, a >> _S32
    b0, b1 = b & _M32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _M32) + (p10 & _M32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64(c0: np.ndarray, c1, c2, c3, key0, key1):
    """Vectorised Philox4x64-10 over an array of first counter words."""
    with np.errstate(over="ignore"):
        c0 = np.asarray(c0, dtype=np.uint64)
        n = c0.shape
        c1 = np.full(n, np.uint64(c1 & _MASK64), dtype=np.uint64)
        c2 = np.full(n, np.uint64(c2 & _MASK64), dtype=np.uint64)
        c3 = np.full(n, np.uint64(c3 & _MASK64), dtype=np.uint64)
        k0, k1 = key0 & _MASK64, key1 & _MASK64
        for _ in range(10):
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                              hi0 ^ c3 ^ np.uint64(k1), lo0)
            k0 = (k0 + W0) & _MASK64
            k1 = (k1 + W1) & _MASK64
    return c0, c1, c2, c3


def _uniform(x: np.ndarray) -> np.ndarray:
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def _uniform_single(x: np.ndarray) -> np.ndarray:
    """The uniform ((x >> 11) + 1/2) 2^-53 = (2 (x >> 11) + 1) 2^-54 rounded
    once, to nearest with ties to even, to 24 significant bits (FP32), in
    integer arithmetic; returned as float64 values."""
    v = ((x >> np.uint64(11)) << np.uint64(1)) | np.uint64(1)         # odd, below 2^54
    out = np.empty(v.shape, dtype=np.float64)
    for i, vi in enumerate(v.tolist()):
        shift = max(vi.bit_length() - 24, 0)
        q = vi >> shift
        if shift:
            rem, half = vi & ((1 << shift) - 1), 1 << (shift - 1)
            if rem > half or (rem == half and q & 1):
                q += 1
        out[i] = float(q << shift) * 2.0 ** -54
    return out


def _normals(uniforms):
    u0, u1, u2, u3 = uniforms
    r0 = np.sqrt(-2.0 * np.log(u0))
    r1 = np.sqrt(-2.0 * np.log(u2))
    t0 = 2.0 * np.pi * u1
    t1 = 2.0 * np.pi * u3
    return r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)


def draw_elements(count: int, seed: int, instance: int, tag: int,
                  is_complex: bool, kind: str = "gauss", single: bool = False) -> np.ndarray:
    """Elements e = 0..count-1 of the (instance, tag) stream.

    single: round every uniform once to FP32 first (the draw of a
    single-precision sketch); the arithmetic after it stays in FP64."""
    per_block = 2 if is_complex else 4
    nblk = (count + per_block - 1) // per_block
    blocks = np.arange(nblk, dtype=np.uint64)
    words = philox4x64(blocks, instance, tag, 0, seed, 0)
    us = [_uniform_single(w) if single else _uniform(w) for w in words]
    if kind == "gauss":
        v = _normals(us)
    elif kind == "uniform":
        v = tuple(2.0 * u - 1.0 for u in us)
    else:
        raise ValueError(kind)
    if is_complex:
        s = 1.0 / np.sqrt(2.0) if kind == "gauss" else 1.0
        z0 = (v[0] + 1j * v[1]) * s
        z1 = (v[2] + 1j * v[3]) * s
        out = np.stack([z0, z1], axis=1).reshape(-1)
    else:
        out = np.stack(v, axis=1).reshape(-1)
    return out[:count]


def sketch(N: int, ell: int, seed: int, instance: int, is_complex: bool,
           kind: str = "gauss") -> np.ndarray:
    """Omega (N x ell) of Algorithm 4's first line, Omega[n, j] = element j*N+n."""
    flat = draw_elements(N * ell, seed, instance, TAG_SKETCH, is_complex, kind)
    return flat.reshape(ell, N).T.copy()


def gauge_vector(M: int, seed: int, instance: int, is_complex: bool) -> np.ndarray:
    """Fixed random vector g (length M) that pins singular-vector phases."""
    return draw_elements(M, seed, instance, TAG_GAUGE, is_complex, "gauss")


def instance_id(direction: int, row: int, col: int) -> int:
    """Stream id of one einsumsvd step of a boundary sweep."""
    return (direction << 32) | (row << 16) | col
