"""CPU tests of the twiddle tables (no GPU): every root a plan uploads and
every constant of the in-register DFT kernels is exp(-2 pi i e / L) computed
in FP64 and rounded once to the plan's precision.

* Against the exact value (mpmath, 60 digits): an FP32 entry is within half
  an FP32 ulp of it, plus the few FP64 ulps of the FP64 value it was rounded
  from; an FP64 entry is within the error its evaluation allows: the reduced
  angle a (at most an eighth turn) carries three FP64 roundings (2 pi, the
  product, the division), i.e. |da| <= 3 u a with u = 2^-53, which moves
  cos and sin by at most 3 u a, plus one ulp of the C library's cos / sin.
* Rounded once: the FP32 table of a problem equals its FP64 table rounded to
  FP32 entry by entry (no second computation in FP32).
* roots.h is exactly what gen_roots.py writes.
"""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import paper_2506_12718_gb300 as pac

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 60

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_12718_gb300", "csrc")
U64 = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_12718_gb300 import _build
    _build.build()


def exact_root(e, L):
    """exp(-2 pi i e / L) to 60 digits, as (re, im) mpf."""
    a = 2 * mpmath.pi * mpmath.mpf(int(e) % int(L)) / int(L)
    return mpmath.cos(a), -mpmath.sin(a)


def reduced_angle(e, L):
    """The angle the generator evaluates after the exact integer reduction (|a| <= pi/4)."""
    e %= L
    if 2 * e > L:
        e = L - e
    if 8 * e <= L:
        return 2 * math.pi * e / L
    if 8 * e <= 3 * L:
        return 2 * math.pi * (L - 4 * e) / (4 * L)
    return 2 * math.pi * (L - 2 * e) / (2 * L)


def check_entries(vals, exps, L, dtype):
    vals = np.asarray(vals)
    worst = 0.0
    for v, e in zip(vals, exps):
        re_x, im_x = exact_root(e, L)
        a = reduced_angle(int(e), int(L))
        for got, want in ((float(v.real), re_x), (float(v.imag), im_x)):
            err = abs(mpmath.mpf(got) - want) - mpmath.mpf(10) ** -50  # the reference's own rounding
            if dtype == "c64":
                bound = 0.5 * np.spacing(np.float32(abs(float(want)))) + 4 * U64
            else:
                bound = 3 * U64 * abs(a) + float(np.spacing(abs(float(want))))
            assert err <= bound, (e, L, got, float(want), float(err), bound)
            worst = max(worst, float(err) / bound)
    return worst


PROBLEMS = [((3125, 3125), 5), ((2187, 2187), 3), ((128, 128, 128), 4), ((128, 128, 128), 8),
            ((1 << 20,), 2), ((1 << 24, 2), 2), ((1000, 1000), 0), ((6000, 6000), 0), ((120, 120, 120), 0),
            ((3 ** 12,), 3), ((5 ** 8,), 5)]


def tables(dims, radix, dtype):
    groups = pac.pac_plan_groups(dims, radix, dtype)
    for g in range(len(groups)):
        for which in (0, 1, 2):
            vals, L, T = pac.pac_plan_twiddles(dims, radix, dtype, g, which)
            if which == 0:
                exps = np.arange(len(vals))
            elif which == 1:
                exps = np.arange(len(vals))
            else:
                exps = np.arange(len(vals)) * T
            yield g, which, vals, exps, L, T


@pytest.mark.parametrize("dims,radix", PROBLEMS)
def test_plan_twiddles_are_fp64_roots_rounded_once(dims, radix):
    rng = np.random.default_rng(sum(dims) + radix)
    seen = {}
    for dtype, name in ((pac.C128, "c128"), (pac.C64, "c64")):
        groups = pac.pac_plan_groups(dims, radix, dtype)
        for g, which, vals, exps, L, T in tables(dims, radix, dtype):
            assert vals.dtype == (np.complex128 if name == "c128" else np.complex64)
            if which == 0:
                assert L == groups[g][1] and len(vals) == L
            if len(vals) == 0:
                continue
            # against the exact roots: every entry of short tables, 256 seeded entries of long ones
            idx = np.arange(len(vals)) if len(vals) <= 256 else rng.choice(len(vals), 256, replace=False)
            check_entries(vals[idx], exps[idx], L, name)
            key = (which, L, T)
            if name == "c128":
                seen[key] = vals
            elif key in seen:
                # rounded once: the FP32 table is the FP64 table of the same roots rounded entry by entry
                assert np.array_equal(vals, seen[key].astype(np.complex64))
    assert seen


def test_plan_twiddles_external_tables_cover_every_exponent():
    # the two-level split e = hi T + lo reaches every exponent below L exactly once
    for dims, radix in [((1 << 20,), 2), ((6000, 6000), 0), ((3 ** 12,), 3)]:
        for g, which, vals, exps, L, T in tables(dims, radix, pac.C128):
            if which == 2 and len(vals):
                nlo = len(pac.pac_plan_twiddles(dims, radix, pac.C128, g, 1)[0])
                assert nlo == T and len(vals) == -(-L // T)
                assert (len(vals) - 1) * T + (T - 1) >= L - 1


def test_plan_twiddles_rejects_bad_arguments():
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_twiddles((128,), 2, pac.C64, 5, 0)
    assert ei.value.status == pac.Status.ERR_ARG
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_twiddles((128,), 2, pac.C64, 0, 3)
    assert ei.value.status == pac.Status.ERR_ARG
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_twiddles((100,), 2, pac.C64, 0, 0)
    assert ei.value.status == pac.Status.ERR_SIZE


def parse_roots_h(text):
    offs = {int(r): int(o) for r, o in re.findall(r"#define PAC_ROOT_OFF_(\d+) (\d+)", text)}
    body64 = text.split("c_roots64[PAC_ROOT_COUNT] = {")[1].split("};")[0]
    body32 = text.split("c_roots32[PAC_ROOT_COUNT] = {")[1].split("};")[0]
    pairs64 = re.findall(r"\{(\S+), (\S+)\}", body64)
    pairs32 = re.findall(r"\{(\S+)f, (\S+)f\}", body32)
    r64 = np.array([complex(float.fromhex(a), float.fromhex(b)) for a, b in pairs64])
    r32 = np.array([complex(float.fromhex(a), float.fromhex(b)) for a, b in pairs32])
    return offs, r64, r32


def test_roots_header_is_what_the_generator_writes():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_roots.py")], capture_output=True, text=True,
                         check=True).stdout
    with open(os.path.join(CSRC, "roots.h")) as f:
        assert f.read() == out


def test_roots_header_constants_are_fp64_roots_rounded_once():
    with open(os.path.join(CSRC, "roots.h")) as f:
        offs, r64, r32 = parse_roots_h(f.read())
    assert len(r64) == len(r32) and len(r64) > 0
    radices = sorted(offs)
    for i, R in enumerate(radices):
        end = offs[radices[i + 1]] if i + 1 < len(radices) else len(r64)
        assert end - offs[R] == R
        exps = np.arange(R)
        check_entries(r64[offs[R]:end], exps, R, "c128")
        check_entries(r32[offs[R]:end], exps, R, "c64")
        # the FP32 constants are the FP64 constants rounded once
        assert np.array_equal(r32[offs[R]:end].astype(np.complex64), r64[offs[R]:end].astype(np.complex64))
        assert np.array_equal(r32[offs[R]:end], r64[offs[R]:end].astype(np.complex64).astype(np.complex128))
