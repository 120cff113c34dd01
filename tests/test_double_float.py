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

The header itself (csrc/df.cuh) is also built for the host (tests/c/df_host.cpp,
with host definitions of the device intrinsics it calls) and checked against the
model: the FP64 split and the widening back bit for bit (subnormal low parts
within their spacing), the sum bit for bit, the product within its bound.

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


# ---- the header itself (csrc/df.cuh), built for the host with host definitions of the intrinsics


def _df_host():
    import os
    import shutil
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cuda_inc = next((p for p in ("/usr/local/cuda/include",) if os.path.exists(os.path.join(p, "cuda_runtime.h"))), None)
    if not shutil.which("g++") or cuda_inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = os.path.join(tempfile.mkdtemp(), "df_host")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-I", cuda_inc, "-I",
                    os.path.join(root, "paper_2506_12718_gb300", "csrc"), os.path.join(root, "tests", "c", "df_host.cpp"),
                    "-o", exe], check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
        return [[float.fromhex(t) for t in ln.split()] for ln in out.strip().splitlines()]
    return run


def test_header_split_and_widen_match_the_model_bit_for_bit():
    """df_from_double is the model's split (hi truncated to 24 bits, lo the
    rest rounded) bit for bit, and df_to_double is hi + lo rounded once to
    FP64 (subnormal low parts included); the round trip keeps 48 bits down to
    about 2^-102; out-of-range inputs flush to zero or saturate to infinity,
    NaN stays NaN."""
    run = _df_host()
    rng = np.random.default_rng(7)
    ds = list(rng.standard_normal(2000) * 10.0 ** rng.integers(-35, 35, 2000)) + [1.0, -1.0, 0.5, 3.0, -7.25]
    res = run([f"widen {float(d).hex()}" for d in ds])
    for d, (hi, lo, back) in zip(ds, res):
        mhi, mlo = df_from_double(float(d))
        assert hi == float(mhi), d
        if abs(float(mlo)) >= 2.0 ** -126:
            assert lo == float(mlo), d
        else:  # a subnormal low part: rounded twice (to 24 bits, then to the subnormal grid)
            assert abs(lo - float(mlo)) <= 2.0 ** -149, d
        assert back == float(np.float64(hi) + np.float64(lo))
        # 48 bits down to about 2^-102, where lo becomes subnormal (then within its spacing, 2^-149)
        assert abs(Fraction(back) - Fraction(float(d))) <= max(Fraction(2) ** -47 * abs(Fraction(float(d))),
                                                                Fraction(2) ** -149)
    special = run([f"split {v.hex()}" for v in (0.0, -0.0, 1e-40, -1e-45, 1e39, -1e300, float("inf"))] + ["split nan"])
    assert special[0] == [0.0, 0.0] and math_copysign(special[1][0]) < 0
    assert special[2] == [0.0, 0.0] and special[3][0] == 0.0
    assert special[4][0] == float("inf") and special[5][0] == -float("inf") and special[6][0] == float("inf")
    assert np.isnan(special[7][0])


def math_copysign(x):
    import math
    return math.copysign(1.0, x)


def test_header_sum_and_product_meet_the_bounds():
    """operator+ is the model's sum bit for bit (no fused operation in it);
    operator* is within 2^-44 of the exact product; both on operands of many
    magnitudes, cancellation included."""
    run = _df_host()
    rng = np.random.default_rng(8)
    xs = rand_df(rng, 300, 1.0) + rand_df(rng, 100, 1e-6) + rand_df(rng, 100, 1e6)
    pairs = [(xs[i], xs[i + 1]) for i in range(len(xs) - 1)] + [(xs[0], (-xs[0][0], -xs[0][1]))]
    fmt = lambda a, b: f"{float(a[0]).hex()} {float(a[1]).hex()} {float(b[0]).hex()} {float(b[1]).hex()}"
    sums = run([f"add {fmt(a, b)}" for a, b in pairs])
    prods = run([f"mul {fmt(a, b)}" for a, b in pairs])
    for (a, b), s, p in zip(pairs, sums, prods):
        ms = df_add(a, b)
        assert (s[0], s[1]) == (float(ms[0]), float(ms[1]))
        exact = val(a) * val(b)
        assert abs(Fraction(p[0]) + Fraction(p[1]) - exact) <= Fraction(2) ** -44 * abs(exact)
    assert sums[-1] == [0.0, 0.0]
