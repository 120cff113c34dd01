"""CPU tests of the double-float arithmetic of the PAC_C128_DF kernels (no GPU).

A numpy model of the operations in csrc/df.cuh, step for step in FP32 (numpy
float32 arithmetic rounds every operation to nearest, like __fadd_rn /
__fmul_rn; a fused multiply-add is the FP64 value of a product of two floats,
which is exact, plus the addend, rounded once to FP32):

* a + b (two-sum of the high parts, low parts added, fast two-sum) is within
  2^-44 (|a| + |b|) of the exact sum, and a - a is 0;
* a * b (high product, its exact error, the two cross terms) is within
  2^-44 |a b| of the exact product;
* the split of an FP64 value into hi + lo (hi its significand truncated to 24
  bits, lo the rest rounded to 24 bits) is within 2^-48 of it, relative;
* a model radix-2 FFT in these operations matches numpy's FFT to 1e-13 on
  random data, where plain FP32 misses by 1e-7 — and a model with one term of
  the product dropped fails the same test (the bound has teeth).

Exact references are Python fractions.
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def fma32(a, b, c):
    """a * b + c rounded once to FP32 (the product of two floats is exact in FP64)"""
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def fast_two_sum(s, e):
    h = F32(s + e)
    return h, F32(e - F32(h - s))


def df_add(a, b):
    s = F32(a[0] + b[0])
    v = F32(s - a[0])
    e = F32(F32(a[0] - F32(s - v)) + F32(b[0] - v))
    e = F32(e + F32(a[1] + b[1]))
    return fast_two_sum(s, e)


def df_mul(a, b, drop_cross=False):
    p = F32(a[0] * b[0])
    e = fma32(a[0], b[0], -p)
    e = fma32(a[0], b[1], e)
    if not drop_cross:
        e = fma32(a[1], b[0], e)
    return p, e


def df_from_double(d):
    """hi: the significand truncated to 24 bits; lo: d - hi rounded to FP32"""
    if d == 0.0:
        return F32(0.0), F32(0.0)
    m, ex = np.frexp(d)                       # d = m 2^ex, 0.5 <= |m| < 1
    hi = np.ldexp(np.trunc(np.ldexp(m, 24)), ex - 24)
    return F32(hi), F32(d - hi)


def val(a):
    return Fraction(float(a[0])) + Fraction(float(a[1]))


def rand_df(rng, n, scale=1.0):
    return [df_from_double(float(rng.standard_normal() * scale)) for _ in range(n)]


def test_sum_is_within_the_bound_and_exact_cancellation():
    rng = np.random.default_rng(1)
    xs = rand_df(rng, 400, 1.0) + rand_df(rng, 100, 1e-5) + rand_df(rng, 100, 1e5)
    for i in range(0, len(xs) - 1):
        a, b = xs[i], xs[i + 1]
        got = val(df_add(a, b))
        exact = val(a) + val(b)
        assert abs(got - exact) <= Fraction(2) ** -44 * (abs(val(a)) + abs(val(b)))
        assert val(df_add(a, (-a[0], -a[1]))) == 0


def test_product_is_within_the_bound():
    rng = np.random.default_rng(2)
    xs = rand_df(rng, 300, 1.0) + rand_df(rng, 100, 1e-3)
    for i in range(0, len(xs) - 1):
        a, b = xs[i], xs[i + 1]
        got = val(df_mul(a, b))
        exact = val(a) * val(b)
        assert abs(got - exact) <= Fraction(2) ** -44 * abs(exact)


def test_split_of_a_double_keeps_48_bits():
    rng = np.random.default_rng(3)
    for d in list(rng.standard_normal(500) * 10.0 ** rng.integers(-20, 20, 500)) + [1.0, -2.5, 1e-30, 3e30]:
        hi, lo = df_from_double(float(d))
        assert abs(val((hi, lo)) - Fraction(float(d))) <= Fraction(2) ** -48 * abs(Fraction(float(d)))
        assert abs(float(hi)) <= abs(d)       # truncation toward zero: lo has the sign of d


def _neg(a):
    return (-a[0], -a[1])


def _model_fft(x, drop_cross=False):
    """radix-2 DIF FFT of a list of complex double-floats ((re_hi, re_lo), (im_hi, im_lo)),
    twiddles split from FP64, natural order out (bit reversal applied at the end)"""
    n = len(x)
    a = list(x)
    span = n
    while span > 1:
        h = span // 2
        for start in range(0, n, span):
            for j in range(h):
                w = np.exp(-2j * np.pi * j / span)
                wr, wi = df_from_double(w.real), df_from_double(w.imag)
                u, v = a[start + j], a[start + j + h]
                s = (df_add(u[0], v[0]), df_add(u[1], v[1]))
                d = (df_add(u[0], _neg(v[0])), df_add(u[1], _neg(v[1])))
                re = df_add(df_mul(d[0], wr, drop_cross), _neg(df_mul(d[1], wi, drop_cross)))
                im = df_add(df_mul(d[0], wi, drop_cross), df_mul(d[1], wr, drop_cross))
                a[start + j], a[start + j + h] = s, (re, im)
        span = h
    bits = n.bit_length() - 1
    out = [None] * n
    for k in range(n):
        out[int(format(k, f"0{bits}b")[::-1], 2)] = a[k]
    return np.array([float(val(z[0])) + 1j * float(val(z[1])) for z in out])


@pytest.mark.parametrize("n", [16, 64])
def test_model_fft_reaches_fp64_accuracy(n):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = [(df_from_double(c.real), df_from_double(c.imag)) for c in z]
    xz = np.array([float(val(c[0])) + 1j * float(val(c[1])) for c in x])
    want = np.fft.fft(xz)
    got = _model_fft(x)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-13, err
    # plain FP32 for scale: far above the bound
    f32 = np.fft.fft(xz.astype(np.complex64)).astype(np.complex128)
    assert np.linalg.norm(f32 - want) / np.linalg.norm(want) > 1e-9
    # a plausible mistake (one cross term of the product dropped) fails the bound
    bad = _model_fft(x, drop_cross=True)
    assert np.linalg.norm(bad - want) / np.linalg.norm(want) > 1e-13
