"""Writes roots.h: the constants of the in-register DFT_R kernels.

* c_tau: the twiddles w_R^e = exp(-2 pi i e / R) between the two stages of
  an in-register Cooley-Tukey split R = A x B are applied in factored form,
  w = sigma (1 + i tau) when |cos| >= |sin| and w = sigma (tau + i)
  otherwise (|tau| <= 1 either way, the tangent or cotangent of the angle);
  the input is multiplied by the complex factor (two fused multiply-adds)
  and the real factor sigma is folded into the constants of the stage-2
  DFT_B that consumes it.  c_tau
  holds tau of the forward root (the conjugate root has -tau), for every
  e < R of each split size R.
* c_roots32: w_R^e itself for the complex FP32 power-of-two sizes R = 8, 16,
  32, whose splits apply plain complex twiddles (the factored form's constant
  operands cost those register-bound kernels more than the two saved
  instructions).
* c_bfly: the constants of each stage-2 DFT_B (B = 2, 3, 4, 5) with its
  inputs' sigma folded in (products and ratios of sigma with cos and sin of
  2 pi / B), per split R, stage-1 frequency k1 and direction; k1 = 0 (all
  sigma = 1) is the plain DFT_B, and R = 3, 5 hold only that entry.
  These are computed in 60-digit decimal arithmetic from the exact rational
  angle (pi by Machin's formula, sin and cos by their Taylor series after an
  exact reduction to at most an eighth turn), rounded once to FP64, and the
  FP32 table is the FP64 table rounded once.
* c_taudf, c_bflydf: the same constants as double-float pairs {hi, lo} for
  the double-float kernels: hi the decimal value rounded to FP32, lo the
  remainder rounded to FP32 (about 48 significant bits in all).

Literals are written as C hex floats, so the tables hold exactly these
values.  Run: python gen_roots.py > roots.h
"""
import decimal
import struct

RADICES = [3, 5, 8, 9, 16, 25, 27, 32]
# FP32 sizes with plain complex twiddles between the stages of their split
PLAIN32_RADICES = [8, 16, 32]
# in-register sizes with a stage-1 / stage-2 split, and the plain prime kernels
BFLY_RADICES = [3, 5, 8, 9, 16, 25, 27, 32]
# FP32 sizes with plain complex twiddles between the stages of their split
PLAIN32_RADICES = [8, 16, 32]

D = decimal.Decimal
CTX = decimal.Context(prec=60)


def f32(v):
    return struct.unpack("f", struct.pack("f", v))[0]


# ------------------------------------------------- 60-digit trigonometry


def _atan_inv(n):
    """atan(1/n) by its Taylor series."""
    x = CTX.divide(D(1), D(n))
    x2 = CTX.multiply(x, x)
    term, total, k = x, x, 1
    while True:
        term = CTX.multiply(term, x2)
        nxt = CTX.divide(term, D(2 * k + 1))
        if nxt == 0 or abs(nxt) < D(10) ** -70:
            break
        total = CTX.subtract(total, nxt) if k % 2 else CTX.add(total, nxt)
        k += 1
    return total


PI = CTX.subtract(CTX.multiply(D(16), _atan_inv(5)), CTX.multiply(D(4), _atan_inv(239)))


def _sin_cos_small(a):
    """sin and cos of |a| <= pi/4 by their Taylor series."""
    a2 = CTX.multiply(a, a)
    s, c = a, D(1)
    ts, tc = a, D(1)
    for k in range(1, 60):
        ts = CTX.divide(CTX.multiply(-ts, a2), D((2 * k) * (2 * k + 1)))
        tc = CTX.divide(CTX.multiply(-tc, a2), D((2 * k - 1) * (2 * k)))
        s, c = CTX.add(s, ts), CTX.add(c, tc)
    return s, c


def cos_sin(e, r):
    """cos and sin of 2 pi e / r (decimal), the angle reduced exactly to at most an eighth turn."""
    e %= r
    neg_s = False
    if 2 * e > r:
        e, neg_s = r - e, True
    if 8 * e <= r:
        s, c = _sin_cos_small(CTX.divide(CTX.multiply(2 * PI, D(e)), D(r)))
    elif 8 * e <= 3 * r:
        c, s = _sin_cos_small(CTX.divide(CTX.multiply(2 * PI, D(r - 4 * e)), D(4 * r)))
    else:
        s, c = _sin_cos_small(CTX.divide(CTX.multiply(2 * PI, D(r - 2 * e)), D(2 * r)))
        c = -c
    return c, (-s if neg_s else s)


def form_c(e, r):
    """True when |cos| >= |sin| for the angle 2 pi e / r (integer test)."""
    f = (8 * e) % (4 * r)
    return f <= r or f >= 3 * r


def factored(e, r, inv):
    """(sigma, tau) of w = w_r^e (conjugated when inv): w = sigma (1 + i tau) or sigma (tau + i)."""
    c, s = cos_sin(e, r)
    im = s if inv else -s  # w = c + i im
    if (4 * e) % r == 0:  # quarter turns: w = sigma or sigma i, tau = 0
        return (c, D(0)) if (2 * e) % r == 0 else (im, D(0))
    if form_c(e, r):
        return c, CTX.divide(im, c)
    return im, CTX.divide(c, im)


def small_factor(r):
    """Stage-2 radix of an in-register split (the same rule as the kernels)."""
    return 4 if r % 4 == 0 and r > 4 else (2 if r % 2 == 0 else (3 if r % 3 == 0 else 5))


BFLY_NC = {2: 1, 3: 4, 4: 3, 5: 12}


def bfly_consts(B, sig, inv):
    """Constants of a stage-2 DFT_B whose input b is sigma_b u_b (sig[0] = 1); the order the kernels read."""
    mul, div = CTX.multiply, CTX.divide
    if B == 2:
        return [sig[1]]
    if B == 4:
        return [sig[2], div(sig[3], sig[1]), sig[1]]
    c, s = cos_sin(1, B)  # w_B = c - i s forward
    if B == 3:
        sb = s if inv else -s  # Im of the B-point root used by the direction
        return [div(sig[2], sig[1]), sig[1], mul(c, sig[1]), mul(sb, sig[1])]
    c2, s2 = cos_sin(2, 5)
    s1 = -s if inv else s
    s2 = -s2 if inv else s2
    g1, g2 = mul(s1, sig[1]), mul(s2, sig[1])
    return [div(sig[4], sig[1]), div(sig[3], sig[2]), sig[1], sig[2],
            mul(c, sig[1]), mul(c2, sig[2]), mul(c2, sig[1]), mul(c, sig[2]),
            div(mul(s2, sig[2]), g1), g1, div(mul(s1, sig[2]), g2), g2]


def bfly_table():
    offs, vals = {}, []
    for r in BFLY_RADICES:
        B = small_factor(r) if r not in (3, 5) else r
        A = r // B
        offs[r] = len(vals)
        for inv in (False, True):
            for k1 in range(A):
                sig = [factored(b * k1, r, inv)[0] for b in range(B)]
                vals += bfly_consts(B, sig, inv)
    return offs, vals


def hexd(v):
    return float(v).hex()


def df_pair(v):
    """{hi, lo} float literals: v (decimal) rounded to FP32, then the remainder rounded to FP32"""
    hi = f32(float(v))
    lo = f32(float(CTX.subtract(v, D(hi))))
    return f"{{{hi.hex()}f, {lo.hex()}f}}"


def main():
    offs, taus = {}, []
    for r in RADICES:
        offs[r] = len(taus)
        taus += [factored(e, r, False)[1] for e in range(r)]
    boffs, bvals = bfly_table()
    print("// Generated by gen_roots.py -- do not edit.")
    print("// Factored twiddles (tau), stage-2 butterfly constants and FP32 roots of the in-register DFT splits,")
    print("// computed in 60-digit decimal arithmetic, rounded once to FP64 and FP64 rounded once to FP32;")
    print("// double-float pairs {hi, lo} of the same decimal values.")
    print("#pragma once")
    for r in RADICES:
        print(f"#define PAC_TAU_OFF_{r} {offs[r]}")
    print(f"#define PAC_TAU_COUNT {len(taus)}")
    for r in BFLY_RADICES:
        print(f"#define PAC_BFLY_OFF_{r} {boffs[r]}")
    print(f"#define PAC_BFLY_COUNT {len(bvals)}")
    roffs, roots = {}, []
    for r in PLAIN32_RADICES:
        roffs[r] = len(roots)
        roots += [cos_sin(e, r) for e in range(r)]
    for r in PLAIN32_RADICES:
        print(f"#define PAC_ROOT32_OFF_{r} {roffs[r]}")
    print(f"#define PAC_ROOT32_COUNT {len(roots)}")
    print("static __constant__ double c_tau64[PAC_TAU_COUNT] = {")
    print(",\n".join(f"    {hexd(t)}" for t in taus))
    print("};")
    print("static __constant__ float c_tau32[PAC_TAU_COUNT] = {")
    print(",\n".join(f"    {f32(float(t)).hex()}f" for t in taus))
    print("};")
    # w = cos - i sin, FP64 rounded once to FP32
    print("static __constant__ float2 c_roots32[PAC_ROOT32_COUNT] = {")
    print(",\n".join(f"    {{{f32(float(c)).hex()}f, {f32(-float(sn)).hex()}f}}" for c, sn in roots))
    print("};")
    print("static __constant__ double c_bfly64[PAC_BFLY_COUNT] = {")
    print(",\n".join(f"    {hexd(v)}" for v in bvals))
    print("};")
    print("static __constant__ float c_bfly32[PAC_BFLY_COUNT] = {")
    print(",\n".join(f"    {f32(float(v)).hex()}f" for v in bvals))
    print("};")
    print("static __constant__ float2 c_taudf[PAC_TAU_COUNT] = {")
    print(",\n".join(f"    {df_pair(t)}" for t in taus))
    print("};")
    print("static __constant__ float2 c_bflydf[PAC_BFLY_COUNT] = {")
    print(",\n".join(f"    {df_pair(v)}" for v in bvals))
    print("};")


if __name__ == "__main__":
    main()
