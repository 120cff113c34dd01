"""Writes roots.h: the constants of the in-register DFT_R kernels.

w_R^e = exp(-2 pi i e / R) for the composite in-register sizes R (the
constant twiddles between the sub-DFTs of an in-register Cooley-Tukey split)
and for the prime kernels R = 3, 5.  Computed in FP64 with the angle index
reduced exactly to the first half turn, then rounded once to FP32 for the
single-precision table.  Literals are written as C hex floats, so the tables
hold exactly these values.  Run: python gen_roots.py > roots.h
"""
import math
import struct

RADICES = [3, 5, 9, 16, 25, 27, 32]


def root(e, r):
    """exp(-2 pi i e / r) with the angle reduced to at most an eighth turn in exact integers."""
    e %= r
    conj = False
    if 2 * e > r:  # w^e = conj(w^(r-e))
        e, conj = r - e, True
    # now e/r in [0, 1/2]; evaluate cos(2 pi e/r), sin(2 pi e/r) from a small angle
    if 8 * e <= r:  # [0, 1/8]
        a = 2.0 * math.pi * e / r
        c, s = math.cos(a), math.sin(a)
    elif 8 * e <= 3 * r:  # (1/8, 3/8]: cos = sin(2 pi (1/4 - f)), sin = cos(...)
        a = 2.0 * math.pi * (r - 4 * e) / (4 * r)
        c, s = math.sin(a), math.cos(a)
    else:  # (3/8, 1/2]: cos = -cos(2 pi (1/2 - f)), sin = sin(...)
        a = 2.0 * math.pi * (r - 2 * e) / (2 * r)
        c, s = -math.cos(a), math.sin(a)
    re, im = c, -s
    return (re, -im) if conj else (re, im)


def f32(v):
    return struct.unpack("f", struct.pack("f", v))[0]


def main():
    offs, rows = {}, []
    for r in RADICES:
        offs[r] = len(rows)
        rows += [root(e, r) for e in range(r)]
    print("// Generated by gen_roots.py -- do not edit.")
    print("// w_R^e = exp(-2 pi i e / R), FP64 and FP64 rounded once to FP32.")
    print("#pragma once")
    for r in RADICES:
        print(f"#define PAC_ROOT_OFF_{r} {offs[r]}")
    print(f"#define PAC_ROOT_COUNT {len(rows)}")
    print("static __constant__ double2 c_roots64[PAC_ROOT_COUNT] = {")
    print(",\n".join(f"    {{{re.hex()}, {im.hex()}}}" for re, im in rows))
    print("};")
    print("static __constant__ float2 c_roots32[PAC_ROOT_COUNT] = {")
    print(",\n".join(f"    {{{f32(re).hex()}f, {f32(im).hex()}f}}" for re, im in rows))
    print("};")


if __name__ == "__main__":
    main()
