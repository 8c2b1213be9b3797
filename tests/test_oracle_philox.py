"""Pins of the oracle's Philox4x64-10 and sketch (Algorithm 4, first line).

The external pin is NumPy's own Philox bit generator, run as a library:
its first block for counter c is the block our definition computes at
counter c + 1 (NumPy increments before it generates).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _add256(ctr, inc):
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr)) + inc
    return tuple((v >> (64 * i)) & (2 ** 64 - 1) for i in range(4))


@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((0, 0, 0, 0), (5, 0)),
    ((123456789, 42, 1, 0), (20200616, 0)),
    ((2 ** 64 - 2, 2 ** 63, 7, 3), (2 ** 64 - 1, 99)),
])
def test_philox_matches_numpy_bitgenerator(ctr, key):
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(8)]
    c1 = _add256(ctr, 1)
    c2 = _add256(ctr, 2)
    assert raw[:4] == philox.philox4x64_scalar(c1, key)
    assert raw[4:] == philox.philox4x64_scalar(c2, key)


def test_vectorised_equals_scalar():
    blocks = np.array([0, 1, 2, 17, 2 ** 40 + 3, 2 ** 64 - 1], dtype=np.uint64)
    w = philox.philox4x64(blocks, 77, 1, 0, 12345, 0)
    for i, b in enumerate(blocks):
        ref = philox.philox4x64_scalar((int(b), 77, 1, 0), (12345, 0))
        assert [int(w[j][i]) for j in range(4)] == ref


def test_sketch_layout_and_prefix_property():
    # element e = j*N + n: widening the block only appends columns
    a = philox.sketch(37, 5, 9, 3, True)
    b = philox.sketch(37, 8, 9, 3, True)
    np.testing.assert_array_equal(a, b[:, :5])
    flat = philox.draw_elements(37 * 8, 9, 3, philox.TAG_SKETCH, True)
    np.testing.assert_array_equal(b[4, 6], flat[6 * 37 + 4])


def test_box_muller_by_hand():
    w = philox.philox4x64_scalar((0, 11, 0, 0), (3, 0))
    u = [((x >> 11) + 0.5) * 2.0 ** -53 for x in w]
    r0 = np.sqrt(-2 * np.log(u[0]))
    n0 = r0 * np.cos(2 * np.pi * u[1])
    n1 = r0 * np.sin(2 * np.pi * u[1])
    real = philox.draw_elements(4, 3, 11, 0, False)
    cplx = philox.draw_elements(2, 3, 11, 0, True)
    assert real[0] == pytest.approx(n0, rel=1e-15)
    assert real[1] == pytest.approx(n1, rel=1e-15)
    assert cplx[0] == pytest.approx((n0 + 1j * n1) / np.sqrt(2), rel=1e-15)


def test_gaussian_moments_and_ks():
    x = philox.draw_elements(200000, 1, 2, 0, False)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1) < 0.01
    assert stats.kstest(x, "norm").pvalue > 1e-3
    z = philox.draw_elements(100000, 1, 2, 0, True)
    assert abs(np.mean(np.abs(z) ** 2) - 1) < 0.01
    assert abs(np.mean(z * z)) < 0.01          # circular: E z^2 = 0


def test_uniform_variant_range():
    u = philox.draw_elements(50000, 4, 5, 0, False, "uniform")
    assert u.min() > -1 and u.max() < 1
    assert abs(u.mean()) < 0.01
    assert abs(u.var() - 1 / 3) < 0.01


def test_streams_are_distinct():
    a = philox.draw_elements(64, 1, 2, 0, True)
    b = philox.draw_elements(64, 1, 3, 0, True)
    c = philox.draw_elements(64, 1, 2, 1, True)
    assert not np.allclose(a, b) and not np.allclose(a, c)


def test_single_precision_uniform_is_one_correct_rounding():
    """Reading of the single-precision sketch: each 53-bit uniform
    ((x >> 11) + 1/2) 2^-53 is rounded once to FP32 (nearest, ties to even).
    Checked against exact rational arithmetic: the result is an FP32 value
    within half an FP32 unit of the exact uniform, ties going to the even
    significand (a tie needs 2 (x >> 11) + 1 = 2^24 + 1: x >> 11 = 2^23)."""
    from fractions import Fraction
    words = philox.philox4x64(np.arange(600, dtype=np.uint64), 5, 0, 0, 99, 0)
    xs = np.concatenate(list(words) + [np.array([0, 1 << 34, ((1 << 53) - 1) << 11, (1 << 52) << 11],
                                                dtype=np.uint64)])
    got = philox._uniform_single(xs)
    for x, g in zip(xs.tolist(), got.tolist()):
        assert float(np.float32(g)) == g
        exact = Fraction(2 * (x >> 11) + 1, 1 << 54)
        m, e = np.frexp(np.float32(g if g < 1.0 else 0.9999999))
        ulp = Fraction(2) ** (int(e) - 24)
        err = abs(Fraction(g) - exact)
        assert err <= ulp / 2
        if err == ulp / 2:
            assert (Fraction(g) / ulp).denominator == 1 and int(Fraction(g) / ulp) % 2 == 0
    assert philox._uniform_single(np.array([1 << 34], dtype=np.uint64))[0] == 2.0 ** -30


def test_single_draw_differs_from_double_by_the_uniform_rounding_only():
    """draw_elements(single=True) = the same Box-Muller / affine map applied to
    the FP32-rounded uniforms: uniform variant equals 2 u32 - 1 exactly."""
    a = philox.draw_elements(4000, 3, 7, 0, False, "uniform", single=True)
    words = philox.philox4x64(np.arange(1000, dtype=np.uint64), 7, 0, 0, 3, 0)
    u = np.stack([philox._uniform_single(w) for w in words], axis=1).reshape(-1)
    assert np.array_equal(a, 2.0 * u - 1.0)
    g64 = philox.draw_elements(4000, 3, 7, 0, False, "gauss")
    g32 = philox.draw_elements(4000, 3, 7, 0, False, "gauss", single=True)
    assert 0 < np.max(np.abs(g32 - g64)) < 1e-3
