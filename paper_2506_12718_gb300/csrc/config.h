// Shared tiling rules of the pass kernels.  The host plan builder and the
// device kernels both include this file, so the in-CTA round split (which
// decides where each frequency sits in shared memory) is the same on both
// sides.
#pragma once

namespace pac {

constexpr int kTileBytes = 32 * 1024;  // target data bytes of one tile

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
constexpr int base_of(int m) { return m % 2 == 0 ? 2 : (m % 3 == 0 ? 3 : (m % 5 == 0 ? 5 : 1)); }
constexpr int ilog(int m, int b) { return m <= 1 ? 0 : 1 + ilog(m / b, b); }

// The tiling rules below take a key `esize`: the bytes of a complex element
// (8: complex FP32, 16: complex FP64), or kEsDf for the double-float kernels
// (16-byte elements, computed on the FP32 pipes: their own round and register
// rules).  ebytes(esize) is the element size in bytes.
constexpr int kEsDf = 17;
constexpr int ebytes(int esize) { return esize & ~1; }

// Largest in-register DFT size of one round.  The double-float kernels take
// rounds of 4, 3 and 5 points: a 25-point round held 100 FP32 values a
// thread, so only 3 warps per scheduler hid the double-float operations'
// chains of dependent instructions (issue active 31 %); small rounds at 64
// registers give several times the warps.  Measured (complex FP64 arrays,
// median of 20, L2 flushed): 3125^2 2.06 -> 1.05 ms (rounds of 25 -> 5),
// 2187^2 672 -> 535 us (9 -> 3), 128^3 267 -> 169 us, 4096^2 1591 -> 1383 us,
// 2^20 189 -> 116 us (16 -> 4; rounds of 8 at 96 registers: 220, 1588, 160).
constexpr int round_rmax(int base, int esize) {
    return esize == kEsDf ? (base == 2 ? 4 : base) : (base == 2 ? 16 : base == 3 ? (esize == 8 ? 27 : 9) : 25);
}

// Largest group (column length M) one CTA transforms in shared memory.
constexpr int group_mmax(int base, int esize) {
    return base == 2 ? (esize == 8 ? 4096 : 2048) : base == 3 ? 2187 : 3125;
}

// ------------------------------------------------------------ mixed groups
// A group whose stages have more than one prime base (mixed radix, Section
// 7.1): its rounds are the prime-power parts of M, each split like a one-base
// group into the fewest rounds of at most mix_rmax (16 for base 2, 9 for base
// 3, 25 for base 5) with the exponent spread evenly, all sorted larger first
// (1000 = 25 x 8 x 5, 120 = 8 x 5 x 3, 48 = 16 x 3).  A few sizes have
// compiled pass kernels (mixed_compiled); the others run in the runtime-radix
// kernel (mix.cuh).
constexpr int mix_rmax(int base) { return base == 2 ? 16 : base == 3 ? 9 : 25; }
constexpr int exponent_of(int m, int p) {
    int e = 0;
    while (m > 1 && m % p == 0) {
        m /= p;
        ++e;
    }
    return e;
}
constexpr bool is_mixed(int m) { return m > 1 && (m % 2 == 0) + (m % 3 == 0) + (m % 5 == 0) > 1; }
constexpr int mixed_round_count(int m) {
    const int ps[3] = {2, 3, 5};
    int n = 0;
    for (int k = 0; k < 3; ++k) {
        const int e = exponent_of(m, ps[k]), er = ilog(mix_rmax(ps[k]), ps[k]);
        n += (e + er - 1) / er;
    }
    return n;
}
constexpr int mixed_round_radix(int m, int i) {
    const int ps[3] = {2, 3, 5};
    int r[16] = {};
    int n = 0;
    for (int k = 0; k < 3; ++k) {
        const int p = ps[k], e = exponent_of(m, p), er = ilog(mix_rmax(p), p);
        const int nr = (e + er - 1) / er;
        for (int j = 0; j < nr && n < 16; ++j) r[n++] = ipow(p, e / nr + (j < e % nr ? 1 : 0));
    }
    for (int a = 1; a < n; ++a)  // larger first
        for (int b = a; b > 0 && r[b - 1] < r[b]; --b) {
            const int t = r[b];
            r[b] = r[b - 1];
            r[b - 1] = t;
        }
    return i < n ? r[i] : 1;
}
// mixed group sizes with compiled pass kernels: whole axes of 1000, 120 and
// 6000 points (a 6000-point tile of 4 FP32 or 2 FP64 columns is 192 KB of
// shared memory, one CTA per SM), and 48 (6000 = 48 x 125 when the runtime
// form's 2048-point limit applies)
constexpr bool mixed_compiled(int m) { return m == 48 || m == 120 || m == 1000 || m == 6000; }

// Number of rounds for a column of length m: ceil(log_base m / log_base rmax)
// for one base, the mixed list otherwise.
constexpr int round_count(int m, int esize) {
    return m <= 1 ? 0
           : is_mixed(m)
               ? mixed_round_count(m)
               : (ilog(m, base_of(m)) + ilog(round_rmax(base_of(m), esize), base_of(m)) - 1) /
                     ilog(round_rmax(base_of(m), esize), base_of(m));
}

// Radix of round i: the exponent of m is spread evenly, larger rounds first.
constexpr int round_radix(int m, int esize, int i) {
    return is_mixed(m) ? mixed_round_radix(m, i)
                       : ipow(base_of(m), ilog(m, base_of(m)) / round_count(m, esize) +
                                              (i < ilog(m, base_of(m)) % round_count(m, esize) ? 1 : 0));
}

constexpr int floor_pow2(int v) { return v >= 2 ? 2 * floor_pow2(v / 2) : 1; }
constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Columns per tile: about kTileBytes of data, at least one 32-byte sector and
// at most 256 bytes per row segment (so a warp's 32 threads cover whole rows).
// A group of one round (m <= the round size: no shared-memory exchange) takes
// up to 1 KB per row segment, so that its CTAs get enough tasks: with 256
// bytes a 3-point group would run 32 tasks in a 64-thread CTA (measured on
// mixed-radix 6000^2: 3.2 -> 1.7 ms; 120^3: 260 -> 130 us).
// The large complex FP64 groups (2187 and 3125 points) are bound by the FP64
// pipe, not by HBM: one column per tile (a 16-byte row segment) halves the
// CTA so that two CTAs share an SM and one computes while the other waits on
// its loads.
constexpr int tile_wmin(int m, int esize) { return ebytes(esize) == 16 && m >= 2187 ? 1 : 32 / ebytes(esize); }
constexpr int tile_w0(int m, int esize) {
    return clampi(floor_pow2(kTileBytes / (m * ebytes(esize))), tile_wmin(m, esize),
                  (round_count(m, esize) == 1 ? 1024 : 256) / ebytes(esize));
}
// The narrow tile variant (nv = 1), one of the autotuner's candidates: half
// the columns, for one-base groups whose half-width rows still span at least
// 128 bytes (one 32-byte sector per 8-byte lane of a quarter warp, and the
// bank model finds every round of these shapes conflict-free with the pads
// below).
constexpr bool has_narrow(int m, int esize) { return !is_mixed(m) && (tile_w0(m, esize) / 2) * ebytes(esize) >= 128; }
constexpr int tile_w(int m, int esize, int nv = 0) {
    return nv && has_narrow(m, esize) ? tile_w0(m, esize) / 2 : tile_w0(m, esize);
}

// Row padding of the shared-memory exchange buffer, in elements.  Chosen per
// group size and layout by counting the bank wavefronts of every round's
// access pattern (8-byte accesses served per half-warp, 16-byte per quarter
// warp) over pads 0..32 and taking the smallest pad with the fewest.  Rows
// case (column-fastest tasks): no padding.  Lines case: the tasks that touch
// global memory run in-line-fastest order when the tile is at least 8 lines
// wide, which wants the padding below; narrower tiles keep column-fastest
// order and no padding.
constexpr int tile_pad(int m, int esize, bool lines, int nv = 0) {
    if (!lines || tile_w(m, esize, nv) < 8) return 0;
    if (esize == 8) {
        switch (m) {
            case 32: return 4;
            case 64: case 128: return 2;
            case 81: case 243: return 9;
            case 125: return 13;
            case 256: case 512: return 1;
            default: return 0;
        }
    }
    switch (m) {
        case 32: return 2;
        case 27: case 243: return 3;
        case 125: return 5;
        case 64: case 128: case 256: case 81: return 1;
        default: return 0;
    }
}
// Row swizzle of the exchange buffer of base-2 groups with tiles of 32 bytes a
// row (4 FP32 or 2 FP64 columns, M >= 1024 points).  In their last
// round (block length R, one task per R consecutive rows) a half-warp spans
// four tasks whose rows lie 32 bytes x R apart, all on the same banks, and no
// pitch separates them (a bank model of every round: 1.75x the wavefronts for
// 1024-4096 points); storing row r at r ^ ((r >> log2 R) & 3) puts them on four
// bank groups and keeps every other round's accesses within aligned groups of
// four rows.  Returns log2 R, or 0 for no swizzle.
constexpr int tile_row_swizzle(int m, int esize) {
    return (!is_mixed(m) && base_of(m) == 2 && round_count(m, esize) >= 2 && tile_w(m, esize) * ebytes(esize) <= 32 &&
            round_radix(m, esize, round_count(m, esize) - 1) >= 4)
               ? ilog(round_radix(m, esize, round_count(m, esize) - 1), 2)
               : 0;
}

// Row pitch of the exchange buffer in elements.
constexpr int tile_pitch(int m, int esize, bool lines, int nv = 0) {
    return tile_w(m, esize, nv) + tile_pad(m, esize, lines, nv);
}
constexpr int tile_elems(int m, int esize, bool lines, int nv = 0) { return m * tile_pitch(m, esize, lines, nv); }

// Threads per CTA: one per task of the first (largest) round, rounded up to
// whole warps, within [64, 512].  A multiple of 32, hence of the tile width,
// so in the rows case every task of a thread has the same column.
// Large base-3 FP32 groups (27-point rounds) run 256 threads at 128
// registers so that two CTAs share an SM (measured 2187^2: 121 -> 108 us);
// for base 2 and 5 the 512-thread form measured faster.
constexpr bool two_ctas_per_sm(int m, int esize) { return esize == 8 && base_of(m) == 3 && m >= 729; }
constexpr int pass_threads(int m, int esize, int nv = 0) {
    return clampi(((tile_w(m, esize, nv) * (m / round_radix(m, esize, 0)) + 31) / 32) * 32, 64,
                  two_ctas_per_sm(m, esize) ? 256 : 512);
}

// Register budget per thread the kernel is compiled for: enough for the
// largest in-register round without spilling, small enough to keep several
// CTAs resident.  Complex FP64 3125-point groups fit 168 registers (three
// 128-thread CTAs per SM; measured 3.38 -> 3.36 ms on 3125^2, a shorter last
// wave of the 3125 one-column tiles); smaller FP64 groups with 25-point
// rounds spill at 168.
constexpr int max_round_radix(int m, int esize) { return round_radix(m, esize, 0); }  // rounds are sorted, largest first
constexpr int reg_target(int m, int esize) {
    return esize == 8
               ? (max_round_radix(m, esize) >= 25 ? (two_ctas_per_sm(m, esize) ? 128 : 168)
                  : (round_count(m, esize) >= 2 && round_radix(m, esize, 1) >= 16 ? 96 : 64))
               : (max_round_radix(m, esize) >= 25 ? (m >= 3125 ? 168 : 255)
                  : (round_count(m, esize) >= 2 && round_radix(m, esize, 1) >= 16 ? 168 : 128));
}
constexpr int min_blocks(int m, int esize, int nv = 0) {
    return clampi(65536 / (pass_threads(m, esize, nv) * reg_target(m, esize)), 1, 8);
}
// The double-float kernels: rounds of at most 5 points (round_rmax) keep
// about 20 FP32 values a thread live, which fits 64 registers without
// spills.
constexpr int reg_target_df(int) { return 64; }
constexpr int min_blocks_df(int m) { return clampi(65536 / (pass_threads(m, kEsDf) * reg_target_df(m)), 1, 8); }

// ------------------------------------------------- the runtime-radix kernel
// Mixed groups without a compiled kernel run in the runtime-radix kernel
// (mix.cuh): the tile is copied into shared memory, transformed by the mixed
// group's rounds (radices given at launch), and copied out.
constexpr int kMixThreads = 256;
constexpr int kMixMaxRounds = 8;
constexpr int kMixMmax = 2048;  // largest mixed group
constexpr int mix_w(int m, int esize) { return clampi(floor_pow2(kTileBytes / (m * esize)), 32 / esize, 256 / esize); }
constexpr int mix_pitch(int m, int esize) { return mix_w(m, esize) + 1; }
constexpr int mix_smem_bytes(int m, int esize) { return m * mix_pitch(m, esize) * esize; }
// the largest tile: about kTileBytes of data plus one pitch column of padding
constexpr int kMixSmemMax = 2 * kTileBytes + kMixMmax * 16;

// ------------------------------------------------------------------ planes
// A plane pass holds whole n1 x n2 planes (the last two axes) in one CTA's
// shared memory, element (i1, i2) at i1 * plane_pitch + i2.  Padding chosen
// like tile_pad, over both axes' round patterns.
constexpr int plane_pad(int m1, int m2, int esize) {
    return esize == 8 ? (base_of(m2) == 2 ? (m2 >= 32 ? 3 : 1) : (m2 == 81 || m2 == 125 ? 8 : 0))
                      : (base_of(m2) == 2 ? 1 : 0);
}
constexpr int plane_pitch(int m1, int m2, int esize) { return m2 + plane_pad(m1, m2, esize); }
constexpr int plane_smem_bytes(int m1, int m2, int esize) { return m1 * plane_pitch(m1, m2, esize) * esize; }
// threads of a plane CTA (K CTAs per plane): the larger first-round task count
constexpr int plane_threads(int m1, int m2, int esize, int k) {
    return clampi((((m1 / k * (m2 / round_radix(m2, esize, 0)) > m2 / k * (m1 / round_radix(m1, esize, 0))
                         ? m1 / k * (m2 / round_radix(m2, esize, 0))
                         : m2 / k * (m1 / round_radix(m1, esize, 0))) + 31) / 32) * 32,
                  64, k > 1 ? 256 : 512);
}
// resident CTAs per SM a plane kernel is compiled for: split planes (K > 1)
// keep two per SM so that one cluster's barriers overlap another's work
constexpr int plane_min_blocks(int k) { return k > 1 ? 2 : 1; }
// largest plane the plane pass takes (bytes of shared memory)
constexpr int kPlaneSmemMax = 200 * 1024;

}  // namespace pac

namespace pac {
static_assert(mixed_round_count(1000) == 3 && mixed_round_radix(1000, 0) == 25 && mixed_round_radix(1000, 1) == 8 &&
                  mixed_round_radix(1000, 2) == 5,
              "1000 = 25 x 8 x 5");
static_assert(mixed_round_count(120) == 3 && mixed_round_radix(120, 0) == 8 && mixed_round_radix(120, 2) == 3,
              "120 = 8 x 5 x 3");
static_assert(mixed_round_count(48) == 2 && mixed_round_radix(48, 0) == 16, "48 = 16 x 3");
}  // namespace pac
