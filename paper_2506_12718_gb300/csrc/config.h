// Shared tiling rules of the pass kernels.  The host plan builder and the
// device kernels both include this file, so the in-CTA round split (which
// decides where each frequency sits in shared memory) is the same on both
// sides.
#pragma once

namespace pac {

constexpr int kMaxRounds = 6;
constexpr int kTileBudget = 8 * 1024;  // target shared-memory bytes of one tile

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
constexpr int base_of(int m) { return m % 2 == 0 ? 2 : (m % 3 == 0 ? 3 : (m % 5 == 0 ? 5 : 1)); }
constexpr int ilog(int m, int b) { return m <= 1 ? 0 : 1 + ilog(m / b, b); }

// Largest in-register DFT size of one round.  esize = bytes per complex element.
constexpr int round_rmax(int base, int esize) {
    return base == 2 ? 16 : base == 3 ? (esize == 8 ? 27 : 9) : 25;
}

// Largest group (column length M) one CTA transforms in shared memory.
constexpr int group_mmax(int base, int esize) {
    return base == 2 ? (esize == 8 ? 4096 : 2048) : base == 3 ? 2187 : 3125;
}

// Number of rounds for a column of length m: ceil(log_base m / log_base rmax).
constexpr int round_count(int m, int esize) {
    return m <= 1 ? 0
                  : (ilog(m, base_of(m)) + ilog(round_rmax(base_of(m), esize), base_of(m)) - 1) /
                        ilog(round_rmax(base_of(m), esize), base_of(m));
}

// Radix of round i: the exponent of m is spread evenly, larger rounds first.
constexpr int round_radix(int m, int esize, int i) {
    return ipow(base_of(m), ilog(m, base_of(m)) / round_count(m, esize) +
                                (i < ilog(m, base_of(m)) % round_count(m, esize) ? 1 : 0));
}

constexpr int floor_pow2(int v) { return v >= 2 ? 2 * floor_pow2(v / 2) : 1; }
constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Columns per tile: about kTileBudget bytes, at least one 32-byte sector per row.
constexpr int tile_w(int m, int esize) {
    return clampi(floor_pow2(kTileBudget / (m * esize)), 32 / esize, 256);
}
// Row pitch of the tile in elements (odd: conflict-free column walks).
constexpr int tile_pitch(int m, int esize) { return tile_w(m, esize) + 1; }
constexpr int tile_elems(int m, int esize) { return m * tile_pitch(m, esize); }
// Tile buffers per CTA: two (the copy of the next tile overlaps the current
// one) when they fit in a quarter of the shared memory, else one.
constexpr int tile_stages(int m, int esize) { return 2 * tile_elems(m, esize) * esize <= 56 * 1024 ? 2 : 1; }

// Threads per CTA: one per task of the first round (a multiple of the warp
// size and of the tile width), within [64, 256].
constexpr int pass_threads(int m, int esize) {
    return clampi(((tile_w(m, esize) * (m / round_radix(m, esize, 0)) + 31) / 32) * 32, 64, 256);
}

// Register budget per thread the kernel is compiled for: enough for the
// largest in-register round without spilling, small enough to keep several
// CTAs resident.  FP64 rounds of 16+ complex values keep the full file.
constexpr int reg_target(int m, int esize) {
    return esize == 8 ? (round_radix(m, esize, 0) >= 25 ? 255 : (m >= 2048 ? 104 : 80))
                      : (round_radix(m, esize, 0) <= 9 ? 128 : 255);
}
constexpr int min_blocks(int m, int esize) {
    return clampi(65536 / (pass_threads(m, esize) * reg_target(m, esize)), 1, 8);
}

}  // namespace pac
