// Device building blocks of the permutation-avoiding convolution: complex
// arithmetic, in-register DFTs and the generic column-pass kernel.
//
// A "pass" applies one group of consecutive decimation-in-frequency stages of
// one axis (a product of the butterfly matrices B^T_{r,k} of Eq. 25, in the
// order of Algorithm 13) to the whole array, or the adjoint group (conjugate
// butterflies, Algorithm 12 order) for the inverse.  Algebraically a group of
// stages with product M, acting on blocks of length L = M * L', is: for each
// column j in [0, L') of a block, an M-point DFT over the elements j + L' m,
// then the factor w_L^{j k'} on output frequency k', written to block
// position p(k') * L' + j, where p is the digit-reversed position of k' for
// the group's stage list (Sections 2.1 and 7.1).  The kernel computes exactly
// that map; inside the CTA it evaluates the M-point DFT in "rounds" of
// in-register DFTs through shared memory.  Only the placement p matters for
// the result, and it comes from the plan's tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "config.h"
#include "df.cuh"
#include "pass_args.h"
#include "roots.h"

namespace pac {

// ------------------------------------------------------------------ complex

// key of the tiling rules of element type V (config.h)
template <typename V> constexpr int cfg_es() { return std::is_same<V, dfloat2>::value ? kEsDf : (int)sizeof(V); }

template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };
template <> struct Real<dfloat2> { using T = dfloat; };  // double-float (df.cuh)

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// a * (-i) and a * (+i)
template <typename V> __device__ __forceinline__ V mul_mi(V a) { return V{a.y, -a.x}; }
template <typename V> __device__ __forceinline__ V mul_pi(V a) { return V{-a.y, a.x}; }
template <typename V> __device__ __forceinline__ V cscale(V a, typename Real<V>::T s) { return V{a.x * s, a.y * s}; }

// Constants of the in-register DFTs (roots.h, generated): tau of the factored
// twiddles and the stage-2 butterfly constants, FP64 or FP64 rounded once.
template <typename V> __device__ __forceinline__ typename Real<V>::T tau_const(int off);
template <> __device__ __forceinline__ float tau_const<float2>(int off) { return c_tau32[off]; }
template <> __device__ __forceinline__ double tau_const<double2>(int off) { return c_tau64[off]; }
template <> __device__ __forceinline__ dfloat tau_const<dfloat2>(int off) {
    const float2 f = c_taudf[off];
    return dfloat(f.x, f.y);
}
template <typename V> __device__ __forceinline__ typename Real<V>::T bfly_const(int off);
template <> __device__ __forceinline__ float bfly_const<float2>(int off) { return c_bfly32[off]; }
template <> __device__ __forceinline__ double bfly_const<double2>(int off) { return c_bfly64[off]; }
template <> __device__ __forceinline__ dfloat bfly_const<dfloat2>(int off) {
    const float2 f = c_bflydf[off];
    return dfloat(f.x, f.y);
}

__host__ __device__ constexpr int tau_off(int r) {
    return r == 3 ? PAC_TAU_OFF_3
         : r == 5 ? PAC_TAU_OFF_5
         : r == 8 ? PAC_TAU_OFF_8
         : r == 9 ? PAC_TAU_OFF_9
         : r == 16 ? PAC_TAU_OFF_16
         : r == 25 ? PAC_TAU_OFF_25
         : r == 27 ? PAC_TAU_OFF_27
         : r == 32 ? PAC_TAU_OFF_32
                   : -1;
}
__host__ __device__ constexpr int bfly_off(int r) {
    return r == 3 ? PAC_BFLY_OFF_3
         : r == 5 ? PAC_BFLY_OFF_5
         : r == 8 ? PAC_BFLY_OFF_8
         : r == 9 ? PAC_BFLY_OFF_9
         : r == 16 ? PAC_BFLY_OFF_16
         : r == 25 ? PAC_BFLY_OFF_25
         : r == 27 ? PAC_BFLY_OFF_27
         : r == 32 ? PAC_BFLY_OFF_32
                   : -1;
}
// constants per stage-2 butterfly of radix B
__host__ __device__ constexpr int bfly_nc(int b) { return b == 2 ? 1 : b == 3 ? 4 : b == 4 ? 3 : 12; }

// Stage-2 radix of an in-register split R = A x B (B in 2, 3, 4, 5; A may be composite).
constexpr int small_factor(int r) { return r % 4 == 0 && r > 4 ? 4 : (r % 2 == 0 ? 2 : (r % 3 == 0 ? 3 : 5)); }

// |cos| >= |sin| for the angle 2 pi e / r (exact integer test)
__host__ __device__ constexpr bool form_c(int e, int r) {
    return (8 * e) % (4 * r) <= r || (8 * e) % (4 * r) >= 3 * r;
}

// Factored twiddle.  w = w_R^e (its conjugate when INV) is sigma (1 + i tau)
// when |cos| >= |sin| and sigma (tau + i) otherwise, |tau| <= 1; this returns
// u = w z / sigma (two fused multiply-adds, none for quarter turns), and the
// real sigma is folded into the constants of the stage-2 butterfly that
// consumes u.  e and R are compile-time constants after unrolling.
template <int R, bool INV, typename V> __device__ __forceinline__ V tw_factored(V z, int e) {
    using T = typename Real<V>::T;
    e %= R;
    if ((4 * e) % R == 0) return (2 * e) % R == 0 ? z : mul_pi(z);  // w = sigma or sigma i
    const T t0 = tau_const<V>(tau_off(R) + e);
    const T t = INV ? -t0 : t0;
    if (form_c(e, R)) return V{z.x - t * z.y, z.y + t * z.x};
    return V{t * z.x - z.y, t * z.y + z.x};
}

// DFT_B (B = 2, 3, 4, 5) of inputs sigma_b u_b, sigma_0 = 1, in place on
// u[0..B): the sigma_b are folded into the constants at bfly_const(off ...),
// so the butterfly costs what the plain one does.  Forward w = exp(-2 pi i / B),
// conjugate when INV; natural order in and out, no scaling.
template <int B, bool INV, typename V> __device__ __forceinline__ void dft_sc(V* v, int off) {
    using T = typename Real<V>::T;
    if constexpr (B == 2) {
        const T s1 = bfly_const<V>(off);
        const V a = v[0], b = v[1];
        v[0] = V{a.x + s1 * b.x, a.y + s1 * b.y};
        v[1] = V{a.x - s1 * b.x, a.y - s1 * b.y};
    } else if constexpr (B == 3) {
        const T rho = bfly_const<V>(off), s1 = bfly_const<V>(off + 1);
        const T cs = bfly_const<V>(off + 2), g = bfly_const<V>(off + 3);
        const V a = v[0];
        const V t = V{v[1].x + rho * v[2].x, v[1].y + rho * v[2].y};
        const V d = V{v[1].x - rho * v[2].x, v[1].y - rho * v[2].y};
        const V m = V{a.x + cs * t.x, a.y + cs * t.y};
        v[0] = V{a.x + s1 * t.x, a.y + s1 * t.y};
        v[1] = V{m.x - g * d.y, m.y + g * d.x};  // m + i g d
        v[2] = V{m.x + g * d.y, m.y - g * d.x};  // m - i g d
    } else if constexpr (B == 4) {
        const T s2 = bfly_const<V>(off), rho = bfly_const<V>(off + 1), s1 = bfly_const<V>(off + 2);
        const V a = v[0];
        const V s0 = V{a.x + s2 * v[2].x, a.y + s2 * v[2].y};
        const V d0 = V{a.x - s2 * v[2].x, a.y - s2 * v[2].y};
        const V t1 = V{v[1].x + rho * v[3].x, v[1].y + rho * v[3].y};
        const V d1 = V{v[1].x - rho * v[3].x, v[1].y - rho * v[3].y};
        v[0] = V{s0.x + s1 * t1.x, s0.y + s1 * t1.y};
        v[2] = V{s0.x - s1 * t1.x, s0.y - s1 * t1.y};
        // forward: v1 = d0 - i s1 d1, v3 = d0 + i s1 d1 (signs swapped when INV)
        const T f = INV ? -s1 : s1;
        v[1] = V{d0.x + f * d1.y, d0.y - f * d1.x};
        v[3] = V{d0.x - f * d1.y, d0.y + f * d1.x};
    } else {
        static_assert(B == 5, "stage-2 radices are 2, 3, 4, 5");
        const T r14 = bfly_const<V>(off), r23 = bfly_const<V>(off + 1);
        const T s1 = bfly_const<V>(off + 2), s2 = bfly_const<V>(off + 3);
        const T c11 = bfly_const<V>(off + 4), c22 = bfly_const<V>(off + 5);
        const T c21 = bfly_const<V>(off + 6), c12 = bfly_const<V>(off + 7);
        const T ra = bfly_const<V>(off + 8), g1 = bfly_const<V>(off + 9);
        const T rb = bfly_const<V>(off + 10), g2 = bfly_const<V>(off + 11);
        const V a = v[0];
        const V t1 = V{v[1].x + r14 * v[4].x, v[1].y + r14 * v[4].y};
        const V d1 = V{v[1].x - r14 * v[4].x, v[1].y - r14 * v[4].y};
        const V t2 = V{v[2].x + r23 * v[3].x, v[2].y + r23 * v[3].y};
        const V d2 = V{v[2].x - r23 * v[3].x, v[2].y - r23 * v[3].y};
        const V m1 = V{a.x + c11 * t1.x + c22 * t2.x, a.y + c11 * t1.y + c22 * t2.y};
        const V m2 = V{a.x + c21 * t1.x + c12 * t2.x, a.y + c21 * t1.y + c12 * t2.y};
        const V e1 = V{d1.x + ra * d2.x, d1.y + ra * d2.y};
        const V e2 = V{d1.x - rb * d2.x, d1.y - rb * d2.y};
        v[0] = V{a.x + s1 * t1.x + s2 * t2.x, a.y + s1 * t1.y + s2 * t2.y};
        v[1] = V{m1.x + g1 * e1.y, m1.y - g1 * e1.x};  // m1 - i g1 e1
        v[4] = V{m1.x - g1 * e1.y, m1.y + g1 * e1.x};  // m1 + i g1 e1
        v[2] = V{m2.x + g2 * e2.y, m2.y - g2 * e2.x};  // m2 - i g2 e2
        v[3] = V{m2.x - g2 * e2.y, m2.y + g2 * e2.x};  // m2 + i g2 e2
    }
}

// Complex FP32 power-of-two sizes keep plain twiddles: their pass kernels run
// at 64 registers a thread, and the factored form's stage-2 constants (kept
// in registers across a tile's tasks) cost them spills that outweigh the two
// instructions a twiddle saves (measured on 128^3 FP32: 38 -> 41 us).
template <typename V, int R> constexpr bool plain_twiddles() {
    return sizeof(V) == 8 && (R == 8 || R == 16 || R == 32);
}
__host__ __device__ constexpr int root32_off(int r) {
    return r == 8 ? PAC_ROOT32_OFF_8 : r == 16 ? PAC_ROOT32_OFF_16 : r == 32 ? PAC_ROOT32_OFF_32 : -1;
}

// z * w_R^e (forward) or z * conj(w_R^e) (inverse), complex FP32; e and R are
// compile-time constants after unrolling, so the special cases fold away.
template <int R, bool INV> __device__ __forceinline__ float2 twiddle_root32(float2 z, int e) {
    e %= R;
    if (e == 0) return z;
    if ((8 * e) % R == 0) {
        const float h = 0.70710678118654752440f;
        switch (INV ? (8 - (8 * e) / R) : (8 * e) / R) {  // multiply by exp(-2 pi i o / 8)
            case 1: return float2{(z.x + z.y) * h, (z.y - z.x) * h};
            case 2: return mul_mi(z);
            case 3: return float2{(z.y - z.x) * h, -(z.x + z.y) * h};
            case 4: return float2{-z.x, -z.y};
            case 5: return float2{-(z.x + z.y) * h, (z.x - z.y) * h};
            case 6: return mul_pi(z);
            default: return float2{(z.x - z.y) * h, (z.x + z.y) * h};
        }
    }
    const float2 w = c_roots32[root32_off(R) + e];
    return INV ? cmulc(z, w) : cmul(z, w);
}

// In-register DFT of size R, natural order in and out: v[k] = sum_j v[j] w^{jk}
// with w = exp(-2 pi i / R), or its conjugate (no scaling) when INV.
// Composite R = A x B (B = small_factor(R)), decimation in frequency: B DFT_A
// over stride B, the twiddles w_R^{b k1} in factored form, then A stage-2
// DFT_B with the twiddles' real factors in their constants.  Complex FP32
// powers of two: DFT_4 over stride R/4, plain twiddles, then DFT_{R/4}.
template <int R, bool INV, typename V> __device__ __forceinline__ void dft(V* v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const V a = v[0], b = v[1], c = v[2], d = v[3];
        const V s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
        const V r1 = INV ? mul_pi(d1) : mul_mi(d1);
        v[0] = cadd(s0, s1);
        v[2] = csub(s0, s1);
        v[1] = cadd(d0, r1);
        v[3] = csub(d0, r1);
    } else if constexpr (R == 3 || R == 5) {
        dft_sc<R, INV>(v, bfly_off(R) + (INV ? bfly_nc(R) : 0));
    } else if constexpr (plain_twiddles<V, R>()) {
        constexpr int A = 4;
        constexpr int B = R / A;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            V z[A];
#pragma unroll
            for (int a = 0; a < A; ++a) z[a] = v[b + B * a];
            dft<A, INV>(z);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[b + B * k1] = twiddle_root32<R, INV>(z[k1], b * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) dft<B, INV>(v + B * k1);
        V t[R];
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) t[k1 + A * k2] = v[B * k1 + k2];
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = t[e];
    } else {
        constexpr int B = small_factor(R);
        constexpr int A = R / B;
        static_assert(bfly_off(R) >= 0 && tau_off(R) >= 0, "in-register size without constants");
#pragma unroll
        for (int b = 0; b < B; ++b) {
            V z[A];
#pragma unroll
            for (int a = 0; a < A; ++a) z[a] = v[b + B * a];
            dft<A, INV>(z);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[b + B * k1] = tw_factored<R, INV>(z[k1], b * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) dft_sc<B, INV>(v + B * k1, bfly_off(R) + ((INV ? A : 0) + k1) * bfly_nc(B));
        V t[R];
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) t[k1 + A * k2] = v[B * k1 + k2];
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = t[e];
    }
}

// ------------------------------------------------------------------ passes
//
// One tile = W columns of the pass (columns q0 .. q0+W-1) x all M rows of the
// group.  The first round of a tile reads its R values straight from global
// memory into registers (coalesced along the tile's columns, or along a line
// in the lines case), every later round exchanges through a shared-memory
// buffer of M rows x P (pitch) elements, and the last round writes registers
// straight to global memory.  So a pass costs one global read and one global
// write per element, plus one shared-memory write and read per round
// boundary; there is no separate copy-in or copy-out of the tile.

// read-only loads of a complex element (double-float: one 16-byte load)
template <typename V> __device__ __forceinline__ V ldg_v(const V* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfloat2 ldg_v<dfloat2>(const dfloat2* p) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    return dfloat2{dfloat(f.x, f.y), dfloat(f.z, f.w)};
}

// Loads and stores of the arrays a pass reads and writes.  The double-float
// passes keep their intermediate arrays as double-float pairs (16 bytes an
// element, like complex FP64) and read the caller's input / write the
// caller's output as complex FP64 (PassArgs::df bits kDfSrc64 / kDfDst64).
template <typename V> __device__ __forceinline__ V gload(const PassArgs&, const V* p, uint32_t i) { return p[i]; }
template <> __device__ __forceinline__ dfloat2 gload<dfloat2>(const PassArgs& a, const dfloat2* p, uint32_t i) {
    if (a.df & kDfSrc64) return df2_from_double2(reinterpret_cast<const double2*>(p)[i]);
    const float4 f = reinterpret_cast<const float4*>(p)[i];
    return dfloat2{dfloat(f.x, f.y), dfloat(f.z, f.w)};
}
template <typename V> __device__ __forceinline__ void gstore(const PassArgs&, V* p, uint32_t i, V v) { p[i] = v; }
template <> __device__ __forceinline__ void gstore<dfloat2>(const PassArgs& a, dfloat2* p, uint32_t i, dfloat2 v) {
    if (a.df & kDfDst64)
        reinterpret_cast<double2*>(p)[i] = df2_to_double2(v);
    else
        reinterpret_cast<float4*>(p)[i] = float4{v.x.hi, v.x.lo, v.y.hi, v.y.lo};
}

template <typename V> __device__ __forceinline__ V ld_tw(const void* p, int64_t i) {
    return ldg_v(reinterpret_cast<const V*>(p) + i);
}

// external factor w_L^e, e < L, from the two-level table
template <typename V> __device__ __forceinline__ V ext_twiddle(const PassArgs& a, int64_t e) {
    int64_t hi, lo;
    if (a.tw_shift >= 0) {
        hi = e >> a.tw_shift;
        lo = e & ((int64_t(1) << a.tw_shift) - 1);
    } else {
        hi = e / a.tw_T;
        lo = e - hi * a.tw_T;
    }
    return cmul(ld_tw<V>(a.tw_lo, lo), ld_tw<V>(a.tw_hi, hi));
}

template <int M, int ES, int RI> struct RoundGeom {
    static constexpr int R = round_radix(M, ES, RI);
    // block length before this round: M / (R_0 ... R_{RI-1})
    static constexpr int S = RI == 0 ? M : RoundGeom<M, ES, RI - 1>::S / RoundGeom<M, ES, RI - 1>::R;
    static constexpr int SP = S / R;
};
template <int M, int ES> struct RoundGeom<M, ES, -1> {
    static constexpr int R = 1, S = M * 1, SP = M;
};

// NV = 1: the narrow tile variant (has_narrow in config.h)
template <typename V, int M, bool LINES = false, int NV = 0> struct Shape {
    static constexpr int ES = cfg_es<V>();
    static constexpr int W = tile_w(M, ES, NV);
    static constexpr int P = tile_pitch(M, ES, LINES, NV);
    static constexpr int NR = round_count(M, ES);
    static constexpr int NT = pass_threads(M, ES, NV);
    static constexpr int TILE = M * P;
    static_assert(NT % W == 0, "a thread's tasks must share one column in the rows case");
};

// Geometry of one group's rounds inside a CTA: M rows (the transformed
// axis), W independent columns, NT threads, element (row, w) of the exchange
// buffer at row * RS + w * WS.
// PF: a thread with several tasks in a round that reads global memory
// issues all their loads first (needs registers for all of them).
// KS > 1: the M rows are split over the KS CTAs of a thread-block cluster
// (rows [k M/KS, (k+1) M/KS) in CTA k's buffer, reached through distributed
// shared memory), and rounds synchronise the whole cluster.
// SPLIT: the CTA is several independent units of NT threads (the persistent
// batched kernel), each running its own tile: task numbering uses the
// thread's index within its unit, and rounds synchronise the unit with a
// named barrier instead of the whole CTA.
// RSW > 0: rows of the exchange buffer are stored swizzled, row r at
// r ^ ((r >> RSW) & 3) (tile_row_swizzle in config.h).
template <typename V_, int M_, int W_, int NT_, int RS_, int WS_, bool PF_, int KS_ = 1, bool SPLIT_ = false,
          int RSW_ = 0>
struct Geo {
    using V = V_;
    static constexpr int M = M_, W = W_, NT = NT_, RS = RS_, WS = WS_, ES = cfg_es<V_>(), KS = KS_;
    static constexpr int NR = round_count(M_, ES);
    static constexpr bool PF = PF_;
    static constexpr bool SPLIT = SPLIT_;
    static constexpr int RSW = RSW_;
    static_assert(RSW_ == 0 || KS_ == 1, "row swizzle in single-CTA tiles only");
    __device__ __forceinline__ static int tid() { return SPLIT_ ? (int)(threadIdx.x % NT_) : (int)threadIdx.x; }
};
// the pass kernels' geometry: a tile of W columns, buffer [row][w] of pitch
// P; several CTAs per SM hide latency, so registers are not spent on prefetch
template <typename V, int M, bool LINES, int NV = 0>
using PassGeo = Geo<V, M, Shape<V, M, LINES, NV>::W, Shape<V, M, LINES, NV>::NT, Shape<V, M, LINES, NV>::P, 1, false,
                    1, false, tile_row_swizzle(M, cfg_es<V>())>;

// Task tau of round RI: column w of the tile, offset jp inside its block of
// S rows, first row row0 = block * S + jp; the task transforms rows
// row0 + SP * u, u < R.  Column-fastest order (a warp covers consecutive
// columns of the same row: coalesced in the rows case, conflict-free in shared
// memory) or, for JFAST, offset-fastest order (a warp covers consecutive rows
// of one line: coalesced in the lines case).
template <int M, int ES, int W, int RI, bool JFAST> struct Task {
    using G = RoundGeom<M, ES, RI>;
    static constexpr int TASKS = W * (M / G::R);
    int w, jp, row0;
    __device__ __forceinline__ explicit Task(int tau) {
        if constexpr (JFAST) {
            jp = tau % G::SP;
            const int t2 = tau / G::SP;
            w = t2 % W;
            row0 = (t2 / W) * G::S + jp;
        } else {
            w = tau % W;
            const int t2 = tau / W;
            jp = t2 % G::SP;
            row0 = (t2 / G::SP) * G::S + jp;
        }
    }
};

// Storage order of the filter spectrum.  The spectrum is produced once and
// read only by the last forward round of the fused pass, so it is stored in
// the order that round reads it: element (tile t, register u, task tau) at
// t * W * M + u * TASKS + tau, TASKS = W * M / R for the round's radix R
// (column-fastest tasks, SP = 1: task tau = w + W * b handles rows b R + u).
// spec_slot maps an element's position in the plain index-reversed (DIF)
// order of the array to its slot.  For a plane pass the product is taken in
// the last forward round of axis d-2 over columns w = the in-CTA row of axis
// d-1; with a plane split over a K-CTA cluster, CTA k owns columns
// [k n2/K, (k+1) n2/K), so (plane, k, u, task) with task = w - k n2/K + (n2/K) b.

__device__ __forceinline__ uint32_t spec_slot(const SpecOrder& o, uint32_t e) {
    if (o.M2) {  // plane pass: (plane, axis d-2 position g1, axis d-1 position g2)
        const uint32_t ps = o.M * o.M2, wk = o.M2 / o.K;
        const uint32_t pl = e / ps, rem = e - pl * ps;
        const uint32_t g1 = rem / o.M2, g2 = rem - g1 * o.M2;
        const uint32_t r1 = (uint32_t)__ldg(o.rowmap + g1), r2 = (uint32_t)__ldg(o.rowmap2 + g2);
        const uint32_t b = r1 / o.R, u = r1 - b * o.R;
        const uint32_t rank = r2 / wk, wl = r2 - rank * wk;  // the cluster CTA that owns column r2
        return pl * ps + rank * (ps / o.K) + u * o.tasks + wl + wk * b;
    }
    uint32_t q, g;
    if (o.C == 1) {
        q = e / o.M;
        g = e - q * o.M;
    } else {
        const uint32_t blk = o.M * o.C;
        const uint32_t beta = e / blk, rem = e - beta * blk;
        g = rem / o.C;
        q = beta * o.C + (rem - g * o.C);
    }
    const uint32_t t = q / o.W, w = q - t * o.W;
    const uint32_t r = (uint32_t)__ldg(o.rowmap + g);
    const uint32_t b = r / o.R, u = r - b * o.R;
    return t * o.W * o.M + u * o.tasks + w + o.W * b;
}

// CTAs of a thread-block cluster a split plane may use (the portable maximum).
constexpr int kMaxClusterCtas = 8;

// Per-tile facts.  Rows case (C > 1): a thread's column w = tid mod W is
// fixed, so its global offset and external-twiddle column are computed once
// per tile.  Offsets are 32-bit element offsets (plans keep N < 2^31).
template <typename V> struct TileCtx {
    const PassArgs* a;
    V* s;              // exchange buffer, [row][w], pitch P
    const V* twi;      // w_M^u
    uint32_t t;        // tile index within the pass
    uint32_t q0;       // first column of the tile
    uint32_t Q;        // columns of the pass
    uint32_t C;        // row stride
    uint32_t base;     // rows case: global offset of row 0 of this thread's column
    uint32_t j;        // rows case: external twiddle column j = (q mod C) / I
    bool valid;        // rows case: this thread's column exists (q < Q)
    int wofs;          // column offset of this CTA's columns in the buffer (split rows)
    uint32_t sk[kMaxClusterCtas];  // split planes: the buffer of each CTA of the cluster (shared::cluster addresses)
};

// Loads and stores of distributed shared memory (a CTA of the cluster,
// 32-bit shared::cluster address).
__device__ __forceinline__ float2 ld_dsmem(uint32_t a, float2*) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_dsmem(uint32_t a, double2*) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];\n" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_dsmem(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_dsmem(uint32_t a, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

// shared::cluster address of element (row, w) of a split buffer: rows of CTA
// `part` at sk[part] (selected without run-time array indexing, which would
// put the array in local memory)
template <typename GEO>
__device__ __forceinline__ uint32_t dsmem_addr(const TileCtx<typename GEO::V>& c, int row, int w) {
    constexpr int H = GEO::M / GEO::KS;
    const int part = row / H;
    static_assert(GEO::KS <= kMaxClusterCtas, "cluster larger than the address table");
    uint32_t b = c.sk[0];
#pragma unroll
    for (int k = 1; k < GEO::KS; ++k) b = part == k ? c.sk[k] : b;
    return b + (uint32_t)(((row - part * H) * GEO::RS + (w + c.wofs) * GEO::WS) * (int)sizeof(typename GEO::V));
}

// buffer row of tile row `row` (the row swizzle of tile_row_swizzle)
template <typename GEO> __device__ __forceinline__ int srow(int row) {
    if constexpr (GEO::RSW > 0)
        return row ^ ((row >> GEO::RSW) & 3);
    else
        return row;
}

// Element (row, w) of a round's exchange buffer.
template <typename GEO>
__device__ __forceinline__ typename GEO::V sld(const TileCtx<typename GEO::V>& c, int row, int w) {
    if constexpr (GEO::KS == 1)
        return c.s[srow<GEO>(row) * GEO::RS + w * GEO::WS];
    else
        return ld_dsmem(dsmem_addr<GEO>(c, row, w), static_cast<typename GEO::V*>(nullptr));
}
template <typename GEO>
__device__ __forceinline__ void sst(const TileCtx<typename GEO::V>& c, int row, int w, typename GEO::V v) {
    if constexpr (GEO::KS == 1)
        c.s[srow<GEO>(row) * GEO::RS + w * GEO::WS] = v;
    else
        st_dsmem(dsmem_addr<GEO>(c, row, w), v);
}

// barrier of every thread of a cluster, with release/acquire ordering of
// shared-memory accesses (distributed shared memory included)
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// barrier of the NT-thread unit this thread belongs to (units of 256 threads
// use named barriers 1-2, units of 128 threads 3-6; 0 is the CTA's)
template <int NT> __device__ __forceinline__ void unit_sync() {
    static_assert(NT == 128 || NT == 256, "units of 128 or 256 threads");
    const unsigned id = (NT == 256 ? 1u : 3u) + threadIdx.x / NT;
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(NT) : "memory");
}

// synchronisation between two rounds of a geometry
template <typename GEO> __device__ __forceinline__ void round_sync() {
    if constexpr (GEO::KS > 1)
        cluster_sync_all();
    else if constexpr (GEO::SPLIT)
        unit_sync<GEO::NT>();
    else
        __syncthreads();
}

enum : int { kFromSmem = 0, kFromNatural = 1, kFromPlaced = 2 };
enum : int { kToSmem = 0, kToNatural = 1, kToPlaced = 2 };

// Global position of a task's column: offset of its row 0, external-twiddle
// column, and whether the column exists.
struct TaskCol {
    uint32_t base, j;
    bool valid;
};

template <bool LINES, int M, typename V>
__device__ __forceinline__ TaskCol task_col(const TileCtx<V>& c, int w) {
    if constexpr (LINES) {
        const uint32_t q = c.q0 + (uint32_t)w;
        return TaskCol{q * (uint32_t)M, 0u, q < c.Q};
    } else {
        return TaskCol{c.base, c.j, c.valid};
    }
}

// Everything of a task after its R values are in registers: twiddles and
// DFTs, the product with the spectrum values hs (MUL), and the store.
template <typename GEO, bool LINES, int RI, bool INV, int SRC, int DST, bool MUL, typename TT>
__device__ __forceinline__ void task_body(const TileCtx<typename GEO::V>& c, const TT& t, const TaskCol& col,
                                          typename GEO::V* v, const typename GEO::V* hs) {
    using V = typename GEO::V;
    constexpr int M = GEO::M;
    using G = RoundGeom<M, GEO::ES, RI>;
    constexpr int R = G::R, SP = G::SP, STEP = M / G::S;
    const PassArgs& a = *c.a;
    V* dst = reinterpret_cast<V*>(a.dst);
    const uint32_t stride = LINES ? 1u : c.C;
    if constexpr (INV) {
        if constexpr (SRC == kFromPlaced && !LINES) {
            if (a.has_ext && col.j != 0) {
#pragma unroll
                for (int u = 0; u < R; ++u)
                    v[u] = cmulc(v[u], ext_twiddle<V>(a, (int64_t)col.j * __ldg(a.r2f + t.row0 + SP * u)));
            }
        }
        if constexpr (SP > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], c.twi[STEP * t.jp * k]);
        }
        dft<R, true>(v);
    } else {
        dft<R, false>(v);
        if constexpr (MUL) {
            if (col.valid) {
#pragma unroll
                for (int u = 0; u < R; ++u) v[u] = cmul(v[u], hs[u]);
            }
            dft<R, true>(v);
        } else if constexpr (SP > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = cmul(v[k], c.twi[STEP * t.jp * k]);
        }
    }
    if constexpr (DST == kToSmem) {
#pragma unroll
        for (int u = 0; u < R; ++u) sst<GEO>(c, t.row0 + SP * u, t.w, v[u]);
    } else if constexpr (DST == kToNatural) {
        if (col.valid) {
#pragma unroll
            for (int u = 0; u < R; ++u) gstore(a, dst, col.base + (uint32_t)(t.row0 + SP * u) * stride, v[u]);
        }
    } else {
        if (col.valid) {
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int row = t.row0 + SP * u;
                V o = v[u];
                if constexpr (!LINES) {
                    if (a.has_ext && col.j != 0) o = cmul(o, ext_twiddle<V>(a, (int64_t)col.j * __ldg(a.r2f + row)));
                }
                gstore(a, dst, col.base + (uint32_t)__ldg(a.r2g + row) * stride, o);
            }
        }
    }
}

// a task's R input values from global memory (natural or placed rows)
template <typename GEO, bool LINES, int RI, int SRC, typename TT>
__device__ __forceinline__ void load_src(const TileCtx<typename GEO::V>& c, const TT& t, const TaskCol& col,
                                         typename GEO::V* v) {
    using V = typename GEO::V;
    using G = RoundGeom<GEO::M, GEO::ES, RI>;
    const PassArgs& a = *c.a;
    const V* src = reinterpret_cast<const V*>(a.src);
    const uint32_t stride = LINES ? 1u : c.C;
#pragma unroll
    for (int u = 0; u < G::R; ++u) {
        const int row = t.row0 + G::SP * u;
        const uint32_t g = SRC == kFromNatural ? (uint32_t)row : (uint32_t)__ldg(a.r2g + row);
        v[u] = col.valid ? gload(a, src, col.base + g * stride) : V{0, 0};
    }
}

// the spectrum values of task tau's R outputs: the spectrum is stored in the
// order this round consumes it, slot (tile, u, task), so a warp reads 32
// consecutive elements
template <typename GEO, int RI, typename TT>
__device__ __forceinline__ void load_spec(const TileCtx<typename GEO::V>& c, int tau, const TaskCol& col,
                                          typename GEO::V* hs) {
    using V = typename GEO::V;
    using G = RoundGeom<GEO::M, GEO::ES, RI>;
    constexpr int TASKS = TT::TASKS;
    const V* spec = reinterpret_cast<const V*>(c.a->spec) + (size_t)c.t * (GEO::W * GEO::M) + tau;
#pragma unroll
    for (int u = 0; u < G::R; ++u) hs[u] = col.valid ? ldg_v(spec + u * TASKS) : V{0, 0};
}

// One round of a tile.  SRC: shared memory, natural global rows, or global
// rows in the pass' output placement (row r of the tile's rounds holds the
// data of global row r2g[r]).  Forward: DFT_R, then w_S^{jp k} (SP > 1).
// Inverse (adjoint): conj twiddles, then the conjugate DFT.  MUL (the last
// forward round of a fused pass): DFT, product with the filter spectrum at
// the same global position, conjugate DFT.  DST as SRC; a placed store also
// applies w_L^{j k'}, a placed load (first inverse round) the
// conjugate w_L^{j k'}.  When a thread has a few tasks in the round and the
// round reads global memory, every global load of all its tasks is issued
// before the first task is computed, so their latencies overlap.
template <typename GEO, bool LINES, int RI, bool INV, int SRC, int DST, bool MUL>
__device__ __forceinline__ void round_exec(const TileCtx<typename GEO::V>& c) {
    using V = typename GEO::V;
    constexpr int M = GEO::M;
    using G = RoundGeom<M, GEO::ES, RI>;
    constexpr int R = G::R, SP = G::SP;
    constexpr bool JFAST = LINES && !MUL && (SRC == kFromNatural || DST == kToNatural) && GEO::W >= 8;
    using T = Task<M, GEO::ES, GEO::W, RI, JFAST>;
    static_assert(!MUL || SP == 1, "the product is taken after the last forward round");
    constexpr bool GSRC = SRC != kFromSmem;
    constexpr int ITER = (T::TASKS + GEO::NT - 1) / GEO::NT;
    constexpr bool PREFETCH = GEO::PF && ITER > 1 && ITER * R * ebytes(GEO::ES) <= 256 && (GSRC || MUL);
    if constexpr (PREFETCH) {
        V pre[ITER][R];
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int tau = GEO::tid() + it * GEO::NT;
            if (tau < T::TASKS) {
                const T t(tau);
                const TaskCol col = task_col<LINES, M>(c, t.w);
                if constexpr (GSRC)
                    load_src<GEO, LINES, RI, SRC>(c, t, col, pre[it]);
                else
                    load_spec<GEO, RI, T>(c, tau, col, pre[it]);
            }
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int tau = GEO::tid() + it * GEO::NT;
            if (tau < T::TASKS) {
                const T t(tau);
                const TaskCol col = task_col<LINES, M>(c, t.w);
                V v[R];
                V hs[MUL ? R : 1];
                if constexpr (GSRC) {
#pragma unroll
                    for (int u = 0; u < R; ++u) v[u] = pre[it][u];
                    if constexpr (MUL) load_spec<GEO, RI, T>(c, tau, col, hs);
                } else {
#pragma unroll
                    for (int u = 0; u < R; ++u) v[u] = sld<GEO>(c, t.row0 + SP * u, t.w);
                    if constexpr (MUL) {
#pragma unroll
                        for (int u = 0; u < R; ++u) hs[u] = pre[it][u];
                    }
                }
                task_body<GEO, LINES, RI, INV, SRC, DST, MUL>(c, t, col, v, hs);
            }
        }
    } else {
#pragma unroll 1
        for (int tau = GEO::tid(); tau < T::TASKS; tau += GEO::NT) {
            const T t(tau);
            const TaskCol col = task_col<LINES, M>(c, t.w);
            V v[R];
            V hs[MUL ? R : 1];
            if constexpr (GSRC) {
                load_src<GEO, LINES, RI, SRC>(c, t, col, v);
            } else {
#pragma unroll
                for (int u = 0; u < R; ++u) v[u] = sld<GEO>(c, t.row0 + SP * u, t.w);
            }
            if constexpr (MUL) load_spec<GEO, RI, T>(c, tau, col, hs);
            task_body<GEO, LINES, RI, INV, SRC, DST, MUL>(c, t, col, v, hs);
        }
    }
}

// forward rounds RI .. NR-2, shared memory in and out
template <typename GEO, bool LINES, int RI>
__device__ __forceinline__ void fwd_middle(const TileCtx<typename GEO::V>& c) {
    if constexpr (RI < GEO::NR - 1) {
        round_exec<GEO, LINES, RI, false, kFromSmem, kToSmem, false>(c);
        round_sync<GEO>();
        fwd_middle<GEO, LINES, RI + 1>(c);
    }
}

// inverse rounds RI, RI-1, ..., 1, shared memory in and out
template <typename GEO, bool LINES, int RI>
__device__ __forceinline__ void inv_middle(const TileCtx<typename GEO::V>& c) {
    if constexpr (RI >= 1) {
        round_exec<GEO, LINES, RI, true, kFromSmem, kToSmem, false>(c);
        round_sync<GEO>();
        inv_middle<GEO, LINES, RI - 1>(c);
    }
}

// kFwd: natural rows in, placed rows out (with w_L^{j k'}).
template <typename GEO, bool LINES>
__device__ __forceinline__ void tile_forward(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    if constexpr (NR == 1) {
        round_exec<GEO, LINES, 0, false, kFromNatural, kToPlaced, false>(c);
    } else {
        round_exec<GEO, LINES, 0, false, kFromNatural, kToSmem, false>(c);
        round_sync<GEO>();
        fwd_middle<GEO, LINES, 1>(c);
        round_exec<GEO, LINES, NR - 1, false, kFromSmem, kToPlaced, false>(c);
    }
}

// kInv: placed rows in (with conj w_L^{j k'}), natural rows out.
template <typename GEO, bool LINES>
__device__ __forceinline__ void tile_inverse(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    if constexpr (NR == 1) {
        round_exec<GEO, LINES, 0, true, kFromPlaced, kToNatural, false>(c);
    } else {
        round_exec<GEO, LINES, NR - 1, true, kFromPlaced, kToSmem, false>(c);
        round_sync<GEO>();
        inv_middle<GEO, LINES, NR - 2>(c);
        round_exec<GEO, LINES, 0, true, kFromSmem, kToNatural, false>(c);
    }
}

// kFused: natural rows in, forward rounds, product, inverse rounds, natural rows out.
template <typename GEO, bool LINES>
__device__ __forceinline__ void tile_fused(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    if constexpr (NR == 1) {
        round_exec<GEO, LINES, 0, false, kFromNatural, kToNatural, true>(c);
    } else {
        round_exec<GEO, LINES, 0, false, kFromNatural, kToSmem, false>(c);
        round_sync<GEO>();
        fwd_middle<GEO, LINES, 1>(c);
        round_exec<GEO, LINES, NR - 1, false, kFromSmem, kToSmem, true>(c);
        round_sync<GEO>();
        inv_middle<GEO, LINES, NR - 2>(c);
        round_exec<GEO, LINES, 0, true, kFromSmem, kToNatural, false>(c);
    }
}

// Programmatic dependent launch: let the next pass in the stream be scheduled
// now; wait here until the previous pass' writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Set up the per-tile facts of tile t.
template <typename V, int M, bool LINES, int NV = 0>
__device__ __forceinline__ void tile_setup(TileCtx<V>& c, const PassArgs& a, uint32_t t) {
    using SH = Shape<V, M, false, NV>;
    c.t = t;
    c.q0 = t * SH::W;
    c.valid = false;
    c.base = 0;
    c.j = 0;
    if constexpr (!LINES) {
        const uint32_t q = c.q0 + threadIdx.x % SH::W;
        if (q < c.Q) {
            const uint32_t cq = q % c.C;
            c.valid = true;
            c.base = (q - cq) * (uint32_t)M + cq;
            c.j = a.has_ext ? cq / (uint32_t)a.I : 0;
        }
    }
}

template <typename V, int M, bool LINES, int NV = 0>
__device__ __forceinline__ void tile_run(const TileCtx<V>& c, int mode) {
    using GEO = PassGeo<V, M, LINES, NV>;
    if (mode == kFwd)
        tile_forward<GEO, LINES>(c);
    else if (mode == kFused)
        tile_fused<GEO, LINES>(c);
    else
        tile_inverse<GEO, LINES>(c);
}

template <typename V> __device__ __forceinline__ void ctx_init(TileCtx<V>& c, const PassArgs& a, V* s) {
    c.a = &a;
    c.s = s;
    c.twi = reinterpret_cast<const V*>(a.tw_int);
    c.Q = (uint32_t)a.Q;
    c.C = (uint32_t)a.C;
    c.wofs = 0;
    for (int k = 0; k < kMaxClusterCtas; ++k) c.sk[k] = 0;
}

// One pass over all tiles, CTAs walking tiles blockIdx.x, +gridDim.x, ...
template <typename V, int M, bool LINES, int NV = 0>
__device__ __forceinline__ void run_phase(const PassArgs& a, V* s) {
    TileCtx<V> c;
    ctx_init(c, a, s);
    const uint32_t tiles = (uint32_t)a.tiles;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        tile_setup<V, M, LINES, NV>(c, a, (uint32_t)a.tile0 + t);
        tile_run<V, M, LINES, NV>(c, a.mode);
        __syncthreads();  // the next tile reuses the exchange buffer
    }
}

template <typename V, int M, int NV = 0> constexpr int pass_smem_bytes(bool lines) {
    return (lines ? Shape<V, M, true, NV>::TILE : Shape<V, M, false, NV>::TILE) * (int)sizeof(V);
}

// CTAs per SM the pass kernels are compiled for (the register budget)
template <typename V, int M, int NV> constexpr int pass_min_blocks() {
    return std::is_same<V, dfloat2>::value ? min_blocks_df(M) : min_blocks(M, sizeof(V), NV);
}

// Generic pass kernel: one pass of a convolution (see run_phase).
template <typename V, int M, bool LINES, int NV = 0>
__global__ void __launch_bounds__(pass_threads(M, cfg_es<V>(), NV), (pass_min_blocks<V, M, NV>()))
    pass_kernel(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    pdl_wait();
    run_phase<V, M, LINES, NV>(a, reinterpret_cast<V*>(smem_raw));
}

// Many passes of one kernel shape in one launch (batched convolutions): the
// tiles of passes list[0..n) are numbered consecutively, pass i owning global
// tiles [tile_start[i], tile_start[i+1]); CTAs walk the global tiles.
template <typename V, int M, bool LINES, int NV = 0>
__global__ void __launch_bounds__(pass_threads(M, cfg_es<V>(), NV), (pass_min_blocks<V, M, NV>()))
    pass_multi_kernel(const PassArgs* __restrict__ list, const uint32_t* __restrict__ tile_start, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const uint32_t total = __ldg(tile_start + n);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = n - 1;  // the last pass whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tile_start + mid) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const PassArgs& a = list[lo];
        TileCtx<V> c;
        ctx_init(c, a, s);
        tile_setup<V, M, LINES, NV>(c, a, t - __ldg(tile_start + lo));
        tile_run<V, M, LINES, NV>(c, a.mode);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ planes
//
// Plane pass: the last group of axis d-2 (n1 = its size M1; it never carries
// an external twiddle) and the single group of axis d-1 (M2) for whole
// M1 x M2 planes in one CTA's shared memory.  Axis d-1 forward (first round
// from global, lines coalesced), axis d-2 forward with the product in its
// last round, axis d-2 inverse, axis d-1 inverse (last round to global): the
// convolution of the two innermost axes in one pass, so a 3-D convolution
// takes 3 passes and a 2-D one a single launch.

// K = 1: one CTA per plane.  K > 1: a cluster of K CTAs per plane, CTA k
// holding plane rows [k n1/K, (k+1) n1/K) (its own lines of axis d-1) and,
// for axis d-2, transforming columns [k n2/K, (k+1) n2/K) over all rows.
template <typename V, int M1, int M2, int K> struct PlaneShape {
    static constexpr int ES = sizeof(V);
    static constexpr int P2 = plane_pitch(M1, M2, ES);
    static constexpr int NT = plane_threads(M1, M2, ES, K);
    static constexpr int SMEM = plane_smem_bytes(M1 / K, M2, ES);
    using G2 = Geo<V, M2, M1 / K, NT, 1, P2, true, 1>;  // axis d-1: rows i2, columns = local lines
    using G1 = Geo<V, M1, M2 / K, NT, P2, 1, true, K>;  // axis d-2: rows i1 (split), columns i2
    static_assert(SMEM <= kPlaneSmemMax, "plane too large for one CTA");
    static_assert(M1 % K == 0 && M2 % K == 0, "the plane must split evenly");
    static_assert(K >= 1 && K <= kMaxClusterCtas, "CTAs per plane beyond the cluster address table");
};

// A plane geometry of NT threads (the persistent batched kernel: its
// whole-CTA items, or with SPLIT its units of NT threads).
template <typename V, int M1, int M2, int NT_, bool SPLIT = false> struct PlaneShapeNT {
    static constexpr int ES = sizeof(V);
    static constexpr int P2 = plane_pitch(M1, M2, ES);
    static constexpr int NT = NT_;
    static constexpr int SMEM = plane_smem_bytes(M1, M2, ES);
    using G2 = Geo<V, M2, M1, NT, 1, P2, true, 1, SPLIT>;
    using G1 = Geo<V, M1, M2, NT, P2, 1, true, 1, SPLIT>;
};

// forward rounds 0..NR-1, the first from global (natural rows), all results in shared memory
template <typename GEO, bool LINES>
__device__ __forceinline__ void fwd_all_to_smem(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    round_exec<GEO, LINES, 0, false, kFromNatural, kToSmem, false>(c);
    if constexpr (NR > 1) {
        round_sync<GEO>();
        fwd_middle<GEO, LINES, 1>(c);
        round_exec<GEO, LINES, NR - 1, false, kFromSmem, kToSmem, false>(c);
    }
}

// forward rounds, product, inverse rounds, all in shared memory
template <typename GEO>
__device__ __forceinline__ void fused_in_smem(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    if constexpr (NR == 1) {
        round_exec<GEO, false, 0, false, kFromSmem, kToSmem, true>(c);
    } else {
        round_exec<GEO, false, 0, false, kFromSmem, kToSmem, false>(c);
        round_sync<GEO>();
        fwd_middle<GEO, false, 1>(c);
        round_exec<GEO, false, NR - 1, false, kFromSmem, kToSmem, true>(c);
        round_sync<GEO>();
        inv_middle<GEO, false, NR - 2>(c);
        round_exec<GEO, false, 0, true, kFromSmem, kToSmem, false>(c);
    }
}

// inverse rounds NR-1..0 from shared memory, the last to global (natural rows)
template <typename GEO, bool LINES>
__device__ __forceinline__ void inv_all_from_smem(const TileCtx<typename GEO::V>& c) {
    constexpr int NR = GEO::NR;
    if constexpr (NR == 1) {
        round_exec<GEO, LINES, 0, true, kFromSmem, kToNatural, false>(c);
    } else {
        round_exec<GEO, LINES, NR - 1, true, kFromSmem, kToSmem, false>(c);
        round_sync<GEO>();
        inv_middle<GEO, LINES, NR - 2>(c);
        round_exec<GEO, LINES, 0, true, kFromSmem, kToNatural, false>(c);
    }
}

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared-memory location in CTA `rank` of the cluster
template <typename V> __device__ __forceinline__ uint32_t map_cluster(V* p, unsigned rank) {
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(out) : "r"(local), "r"(rank));
    return out;
}

// PS: the plane geometry (PlaneShape, or a whole-CTA geometry of another
// thread count for the persistent batched kernel)
template <typename V, int M1, int M2, int K, typename PS = PlaneShape<V, M1, M2, K>>
__device__ __forceinline__ void plane_run(const PlaneArgs& pa, uint32_t plane, unsigned rank, V* s) {
    TileCtx<V> c2, c1;
    ctx_init(c2, pa.a2, s);
    c2.t = plane;
    c2.q0 = plane * (uint32_t)M1 + rank * (uint32_t)(M1 / K);  // this CTA's lines
    c2.valid = true;
    c2.base = 0;
    c2.j = 0;
    ctx_init(c1, pa.a1, s);
    c1.t = plane * K + rank;  // spectrum slots of this CTA's columns
    c1.q0 = 0;
    c1.valid = true;
    c1.base = 0;
    c1.j = 0;
    c1.wofs = (int)rank * (M2 / K);
    if constexpr (K > 1) {
        for (int k = 0; k < K; ++k) c1.sk[k] = map_cluster(s, (unsigned)k);
    }
    fwd_all_to_smem<typename PS::G2, true>(c2);
    round_sync<typename PS::G1>();
    fused_in_smem<typename PS::G1>(c1);
    round_sync<typename PS::G1>();
    inv_all_from_smem<typename PS::G2, true>(c2);
}

template <typename V, int M1, int M2, int K>
__global__ void __launch_bounds__(PlaneShape<V, M1, M2, K>::NT, plane_min_blocks(K))
    plane_kernel(const __grid_constant__ PlaneArgs pa) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    pdl_wait();
    V* s = reinterpret_cast<V*>(smem_raw);
    const unsigned rank = K > 1 ? cluster_ctarank() : 0u;
    if constexpr (K > 1) cluster_sync_all();  // every CTA of the cluster is running
    for (uint32_t p = blockIdx.x / K; p < (uint32_t)pa.planes; p += gridDim.x / K) {
        plane_run<V, M1, M2, K>(pa, p, rank, s);
        __syncthreads();
    }
}

// batched form: planes of list[0..n) numbered consecutively (tile_start as in pass_multi_kernel)
template <typename V, int M1, int M2, int K>
__global__ void __launch_bounds__(PlaneShape<V, M1, M2, K>::NT, plane_min_blocks(K))
    plane_multi_kernel(const PlaneArgs* __restrict__ list, const uint32_t* __restrict__ start, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const unsigned rank = K > 1 ? cluster_ctarank() : 0u;
    if constexpr (K > 1) cluster_sync_all();
    const uint32_t total = __ldg(start + n);
    for (uint32_t t = blockIdx.x / K; t < total; t += gridDim.x / K) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(start + mid) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        plane_run<V, M1, M2, K>(list[lo], t - __ldg(start + lo), rank, s);
        __syncthreads();
    }
}

// Grid-wide barrier for the cooperative convolution kernel (all CTAs are
// co-resident).  The arrival counter only grows; barrier k of a launch waits
// for base + (k+1) * gridDim.x arrivals (plus target_bias, which only the
// timeout test hook sets, to a target no launch reaches).  The wait is
// bounded: after spin_limit polls (default kBarrierSpinLimit) the CTA
// records the failure in *error and goes on (no hang).
constexpr unsigned kBarrierSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void grid_barrier(const ConvArgs& args, unsigned k) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = args.base + (k + 1) * gridDim.x + args.target_bias;
        const unsigned limit = args.spin_limit ? args.spin_limit : kBarrierSpinLimit;
        __threadfence();
        atomicAdd(args.barrier, 1u);
        unsigned spins = 0;
        while ((int)(ld_acquire_gpu(args.barrier) - target) < 0) {
            if (++spins > limit) {
                atomicExch(args.error, 1u);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

// A whole convolution in one launch: the passes of the plan (forward groups,
// the fused one, inverse groups), all with the same group size M, as phases.
template <typename V, int M>
__global__ void __launch_bounds__(pass_threads(M, sizeof(V)), min_blocks(M, sizeof(V)))
    conv_kernel(const __grid_constant__ ConvArgs args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sbase = reinterpret_cast<V*>(smem_raw);
    for (int p = 0; p < args.npasses; ++p) {
        if (p > 0) grid_barrier(args, (unsigned)(p - 1));
        const PassArgs& a = args.pass[p];
        if (a.C == 1)
            run_phase<V, M, true>(a, sbase);
        else
            run_phase<V, M, false>(a, sbase);
    }
}

}  // namespace pac
