"""CPU tests of the twiddle tables (no GPU): every root a plan uploads is
exp(-2 pi i e / L) computed in FP64 and rounded once to the plan's precision.

* Against the exact value (mpmath, 60 digits): an FP32 entry is within half
  an FP32 ulp of it, plus the few FP64 ulps of the FP64 value it was rounded
  from; an FP64 entry is within the error its evaluation allows: the reduced
  angle a (at most an eighth turn) carries three FP64 roundings (2 pi, the
  product, the division), i.e. |da| <= 3 u a with u = 2^-53, which moves
  cos and sin by at most 3 u a, plus one ulp of the C library's cos / sin.
* Rounded once: the FP32 table of a problem equals its FP64 table rounded to
  FP32 entry by entry (no second computation in FP32).
* The in-register DFT constants (roots.h: the factored twiddles' tau and the
  stage-2 butterfly constants with the twiddles' real factors folded in)
  are the exact values rounded once to FP64 (within half an FP64 ulp of the
  60-digit value), the FP32 tables are the FP64 tables rounded once, and a
  numpy model of the kernels' in-register DFT built from those constants
  is the DFT; roots.h is exactly what gen_roots.py writes.
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
    """offsets and FP64 / FP32 arrays of the generated header"""
    def arr(name):
        body = text.split(name)[1].split("= {")[1].split("};")[0]
        return np.array([float.fromhex(x.strip().rstrip("f")) for x in body.split(",") if x.strip()])
    toff = {int(r): int(o) for r, o in re.findall(r"#define PAC_TAU_OFF_(\d+) (\d+)", text)}
    boff = {int(r): int(o) for r, o in re.findall(r"#define PAC_BFLY_OFF_(\d+) (\d+)", text)}
    return (toff, arr("c_tau64[PAC_TAU_COUNT]"), arr("c_tau32[PAC_TAU_COUNT]"),
            boff, arr("c_bfly64[PAC_BFLY_COUNT]"), arr("c_bfly32[PAC_BFLY_COUNT]"))


def parse_roots32(text):
    """offsets and values of the plain FP32 root table (power-of-two splits)"""
    roff = {int(r): int(o) for r, o in re.findall(r"#define PAC_ROOT32_OFF_(\d+) (\d+)", text)}
    body = text.split("c_roots32[PAC_ROOT32_COUNT] = {")[1].split("};")[0]
    pairs = re.findall(r"\{(\S+)f, (\S+)f\}", body)
    return roff, np.array([complex(float.fromhex(a), float.fromhex(b)) for a, b in pairs])


def test_fp32_root_table_is_the_roots_rounded_once():
    with open(os.path.join(CSRC, "roots.h")) as f:
        roff, r32 = parse_roots32(f.read())
    assert sorted(roff) == [8, 16, 32] and len(r32) == 8 + 16 + 32
    for R, off in roff.items():
        for e in range(R):
            c, im = exact_root(e, R)
            for got, want in ((r32[off + e].real, c), (r32[off + e].imag, im)):
                # the exact value rounded to FP64, then once to FP32
                assert got == float(np.float32(float(want))), (R, e, got, float(want))


def header():
    with open(os.path.join(CSRC, "roots.h")) as f:
        return parse_roots_h(f.read())


def test_roots_header_is_what_the_generator_writes():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_roots.py")], capture_output=True, text=True,
                         check=True).stdout
    with open(os.path.join(CSRC, "roots.h")) as f:
        assert f.read() == out


# ---- the factored twiddles and stage-2 butterfly constants, against mpmath


def stage2_radix(R):
    return 4 if R % 4 == 0 and R > 4 else (2 if R % 2 == 0 else (3 if R % 3 == 0 else 5))


def exact_factored(e, R, inv):
    """(sigma, tau) of w = w_R^e (conjugate when inv) as mpf: w = sigma (1 + i tau) when |cos| >= |sin|,
    else sigma (tau + i); quarter turns give tau = 0."""
    c, im = exact_root(e, R)
    if inv:
        im = -im
    e %= R
    if (4 * e) % R == 0:
        return ((mpmath.nint(c), mpmath.mpf(0)) if (2 * e) % R == 0 else (mpmath.nint(im), mpmath.mpf(0)))
    if form_c(e, R):  # |cos| >= |sin|, decided in integers (ties at the eighth turns go to the cosine form)
        assert abs(c) >= abs(im) - mpmath.mpf(10) ** -50
        return c, im / c
    assert abs(im) > abs(c)
    return im, c / im


def exact_bfly(B, sig, inv):
    """The constants a stage-2 DFT_B with input scales sig reads, in the kernels' order, as mpf."""
    if B == 2:
        return [sig[1]]
    if B == 4:
        return [sig[2], sig[3] / sig[1], sig[1]]
    c1, im1 = exact_root(1, B)          # w_B = c1 + i im1 (forward)
    if B == 3:
        sb = -im1 if inv else im1
        return [sig[2] / sig[1], sig[1], c1 * sig[1], sb * sig[1]]
    c2, im2 = exact_root(2, 5)
    s1 = im1 if inv else -im1           # forward: +sin(2 pi / 5)
    s2 = im2 if inv else -im2
    g1, g2 = s1 * sig[1], s2 * sig[1]
    return [sig[4] / sig[1], sig[3] / sig[2], sig[1], sig[2], c1 * sig[1], c2 * sig[2], c2 * sig[1], c1 * sig[2],
            s2 * sig[2] / g1, g1, s1 * sig[2] / g2, g2]


def bfly_layout(R):
    """(B, A) of the entries at PAC_BFLY_OFF_R: fwd then inv, A stage-1 frequencies each"""
    B = R if R in (3, 5) else stage2_radix(R)
    return B, R // B


NC = {2: 1, 3: 4, 4: 3, 5: 12}


def within_half_ulp(got64, want):
    """FP64 entry = the exact value rounded once (0.5 ulp, plus the reference's 1e-50)"""
    err = abs(mpmath.mpf(float(got64)) - want)
    return err <= 0.5 * float(np.spacing(abs(float(want)))) + mpmath.mpf(10) ** -50


def test_tau_table_is_exact_and_rounded_once():
    toff, t64, t32, _, _, _ = header()
    assert len(t64) == len(t32) and sorted(toff) == [3, 5, 8, 9, 16, 25, 27, 32]
    for R, off in toff.items():
        for e in range(R):
            _, tau = exact_factored(e, R, False)
            assert within_half_ulp(t64[off + e], tau), (R, e, t64[off + e], float(tau))
            assert abs(t64[off + e]) <= 1.0
            # the conjugate root has -tau: one table serves both directions
            assert exact_factored(e, R, True)[1] == -tau
    assert np.array_equal(t32, t64.astype(np.float32).astype(np.float64))


def test_bfly_table_is_exact_and_rounded_once():
    _, _, _, boff, b64, b32 = header()
    n = 0
    for R, off in boff.items():
        B, A = bfly_layout(R)
        for d, inv in enumerate((False, True)):
            for k1 in range(A):
                sig = [exact_factored(b * k1, R, inv)[0] for b in range(B)]
                want = exact_bfly(B, sig, inv)
                base = off + (d * A + k1) * NC[B]
                for i, w in enumerate(want):
                    assert within_half_ulp(b64[base + i], w), (R, inv, k1, i, b64[base + i], float(w))
                n += len(want)
    assert n == len(b64)
    assert np.array_equal(b32, b64.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("dims,radix", [((3125,), 5), ((2187, 9), 3), ((4096, 64), 4), ((1 << 16,), 2)])
def test_double_float_plan_twiddles_are_the_fp64_tables_split_once(dims, radix):
    """The twiddle tables a double-float plan uploads: every FP64 entry of the
    FP64 plan's table (same group, same root) as hi = the FP64 value rounded
    to FP32 and lo = the remainder rounded to FP32, so hi + lo is within
    2^-48 of it (relative to the root's modulus 1) and the pair is exact
    where the FP64 value has at most 24 significant bits."""
    groups = pac.pac_plan_groups(dims, radix, pac.C128_DF, None)
    seen = 0
    for g in range(len(groups)):
        for which in (0, 1, 2):
            pairs, L, T = pac.pac_plan_twiddles(dims, radix, pac.C128_DF, g, which)
            if len(pairs) == 0:
                continue
            # the FP64 table of the same group (the double-float schedule's group at the same index)
            ref, L64, T64 = pac.pac_plan_twiddles(dims, radix, pac.C128, g, which)
            assert (L, T) == (L64, T64) and len(ref) == len(pairs)
            for part, want in ((pairs[:, 0:2], ref.real), (pairs[:, 2:4], ref.imag)):
                hi, lo = part[:, 0].astype(np.float64), part[:, 1].astype(np.float64)
                assert np.array_equal(part[:, 0], want.astype(np.float32))
                assert np.array_equal(part[:, 1], (want - hi).astype(np.float32))
                assert np.max(np.abs(hi + lo - want)) <= 2.0 ** -48
            seen += 1
    assert seen >= 1


# ---- the double-float constant tables (c_taudf, c_bflydf): {hi, lo} FP32 pairs of the same values


def parse_df_pairs(text, name):
    body = text.split(name)[1].split("= {")[1].split("};")[0]
    pairs = re.findall(r"\{(\S+)f, (\S+)f\}", body)
    return [(float.fromhex(a), float.fromhex(b)) for a, b in pairs]


def test_double_float_tables_are_the_exact_values_split_once():
    """hi is the exact value rounded to FP32 (within half an FP32 ulp) and
    hi + lo is within 2^-48 of it relative (lo = the remainder rounded to
    FP32); the two tables have one pair per FP64 entry."""
    with open(os.path.join(CSRC, "roots.h")) as f:
        text = f.read()
    toff, t64, _, boff, b64, _ = parse_roots_h(text)
    tdf = parse_df_pairs(text, "c_taudf[PAC_TAU_COUNT]")
    bdf = parse_df_pairs(text, "c_bflydf[PAC_BFLY_COUNT]")
    assert len(tdf) == len(t64) and len(bdf) == len(b64)
    exact = [None] * len(t64)
    for R, off in toff.items():
        for e in range(R):
            exact[off + e] = exact_factored(e, R, False)[1]
    for R, off in boff.items():
        B, A = bfly_layout(R)
        for d, inv in enumerate((False, True)):
            for k1 in range(A):
                sig = [exact_factored(b * k1, R, inv)[0] for b in range(B)]
                for i, w in enumerate(exact_bfly(B, sig, inv)):
                    hi, lo = bdf[off + (d * A + k1) * NC[B] + i]
                    assert abs(mpmath.mpf(hi) - w) <= 0.5 * float(np.spacing(np.float32(abs(float(w))))) + 1e-50
                    assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - w) <= 2.0 ** -48 * abs(w) + 1e-50, (R, inv, k1, i)
    for (hi, lo), w in zip(tdf, exact):
        assert abs(mpmath.mpf(hi) - w) <= 0.5 * float(np.spacing(np.float32(abs(float(w))))) + 1e-50
        assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - w) <= 2.0 ** -48 * abs(w) + 1e-50
        assert np.float32(hi) == hi and np.float32(lo) == lo


# ---- a numpy model of the kernels' in-register DFT (fft_device.cuh: dft, dft_sc, tw_factored,
# and the plain-twiddle split of complex FP32 powers of two)


def form_c(e, R):
    f = (8 * e) % (4 * R)
    return f <= R or f >= 3 * R


def model_dft(v, R, inv, tabs, dt, roots32=None):
    """The kernels' in-register DFT_R of the vector v, step for step, with the table constants
    (complex FP32 powers of two 8, 16, 32: DFT_4 over stride R/4, plain twiddles from roots32)"""
    toff, t, boff, b = tabs
    if roots32 is not None and R in (8, 16, 32):
        roff, r32 = roots32
        A, B = 4, R // 4
        w = np.empty(R, dtype=v.dtype)
        for bb in range(B):
            z = model_dft(v[bb::B][:A], A, inv, tabs, dt, roots32)
            for k1 in range(A):
                e = (bb * k1) % R
                tw = r32[roff[R] + e]
                w[bb + B * k1] = z[k1] * (np.conj(tw) if inv else tw)
        out = np.empty(R, dtype=v.dtype)
        for k1 in range(A):
            y = model_dft(w[B * k1:B * k1 + B], B, inv, tabs, dt, roots32)
            for k2 in range(B):
                out[k1 + A * k2] = y[k2]
        return out
    if R == 1:
        return v.copy()
    if R == 2:
        return np.array([v[0] + v[1], v[0] - v[1]])
    if R == 4:
        s0, d0, s1, d1 = v[0] + v[2], v[0] - v[2], v[1] + v[3], v[1] - v[3]
        r1 = 1j * d1 if inv else -1j * d1
        return np.array([s0 + s1, d0 + r1, s0 - s1, d0 - r1])
    if R in (3, 5):
        return model_dft_sc(v, R, inv, b, boff[R] + (NC[R] if inv else 0), dt)
    B = stage2_radix(R)
    A = R // B
    w = np.empty(R, dtype=v.dtype)
    for bb in range(B):
        z = model_dft(v[bb::B][:A], A, inv, tabs, dt, roots32)
        for k1 in range(A):
            e = (bb * k1) % R
            if (4 * e) % R == 0:
                u = z[k1] if (2 * e) % R == 0 else 1j * z[k1]
            else:
                tau = dt(-t[toff[R] + e] if inv else t[toff[R] + e])
                u = z[k1] * (1 + 1j * tau) if form_c(e, R) else z[k1] * (tau + 1j)
            w[bb + B * k1] = u
    out = np.empty(R, dtype=v.dtype)
    for k1 in range(A):
        y = model_dft_sc(w[B * k1:B * k1 + B], B, inv, b, boff[R] + ((A if inv else 0) + k1) * NC[B], dt)
        for k2 in range(B):
            out[k1 + A * k2] = y[k2]
    return out


def model_dft_sc(u, B, inv, b, off, dt):
    c = [dt(x) for x in b[off:off + NC[B]]]
    if B == 2:
        return np.array([u[0] + c[0] * u[1], u[0] - c[0] * u[1]])
    if B == 3:
        rho, s1, cs, g = c
        t, d = u[1] + rho * u[2], u[1] - rho * u[2]
        m = u[0] + cs * t
        return np.array([u[0] + s1 * t, m + 1j * g * d, m - 1j * g * d])
    if B == 4:
        s2, rho, s1 = c
        s0, d0 = u[0] + s2 * u[2], u[0] - s2 * u[2]
        t1, d1 = u[1] + rho * u[3], u[1] - rho * u[3]
        f = -s1 if inv else s1
        return np.array([s0 + s1 * t1, d0 - 1j * f * d1, s0 - s1 * t1, d0 + 1j * f * d1])
    r14, r23, s1, s2, c11, c22, c21, c12, ra, g1, rb, g2 = c
    t1, d1 = u[1] + r14 * u[4], u[1] - r14 * u[4]
    t2, d2 = u[2] + r23 * u[3], u[2] - r23 * u[3]
    m1 = u[0] + c11 * t1 + c22 * t2
    m2 = u[0] + c21 * t1 + c12 * t2
    e1, e2 = d1 + ra * d2, d1 - rb * d2
    return np.array([u[0] + s1 * t1 + s2 * t2, m1 - 1j * g1 * e1, m2 - 1j * g2 * e2, m2 + 1j * g2 * e2,
                     m1 + 1j * g1 * e1])


@pytest.mark.parametrize("R", [3, 4, 5, 8, 9, 16, 25, 27, 32])
@pytest.mark.parametrize("inv", [False, True])
def test_in_register_dft_model_is_the_dft(R, inv):
    toff, t64, t32, boff, b64, b32 = header()
    with open(os.path.join(CSRC, "roots.h")) as f:
        roots32 = parse_roots32(f.read())
    rng = np.random.default_rng(R + 100 * inv)
    j = np.arange(R)
    F = np.exp((2j if inv else -2j) * np.pi * np.outer(j, j) / R)  # the DFT matrix (conjugate when inv)
    for tabs, dt, cdt, tol, r32 in (((toff, t64, boff, b64), np.float64, np.complex128, 4e-15, None),
                                    ((toff, t32, boff, b32), np.float32, np.complex64, 2.5e-6, roots32),
                                    ((toff, t32, boff, b32), np.float32, np.complex64, 2.5e-6, None)):
        for _ in range(4):
            x = (rng.standard_normal(R) + 1j * rng.standard_normal(R)).astype(cdt)
            got = model_dft(x, R, inv, tabs, dt, r32)
            want = F @ x.astype(np.complex128)
            assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want) * np.log2(R), (R, inv, dt)
        # every basis vector: a wrong constant anywhere shows
        for k in range(R):
            x = np.zeros(R, dtype=cdt)
            x[k] = 1
            got = model_dft(x, R, inv, tabs, dt, r32)
            assert np.allclose(got, F[:, k], atol=tol * 8 * R), (R, inv, k)
