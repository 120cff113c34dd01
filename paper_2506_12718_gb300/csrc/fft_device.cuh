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
// the group's stage list (Sections 2.1 and 6.1).  The kernel computes exactly
// that map; inside the CTA it evaluates the M-point DFT in "rounds" of
// in-register DFTs through shared memory.  Only the placement p matters for
// the result, and it comes from the plan's tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "config.h"
#include "pass_args.h"
#include "roots.h"

namespace pac {

// ------------------------------------------------------------------ complex

template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

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

// the root w_R^e = exp(-2 pi i e / R) (conjugated when INV) from the constant tables
template <typename V> __device__ __forceinline__ V root_const(int off);
template <> __device__ __forceinline__ float2 root_const<float2>(int off) { return c_roots32[off]; }
template <> __device__ __forceinline__ double2 root_const<double2>(int off) { return c_roots64[off]; }

__host__ __device__ constexpr int root_off(int r) {
    return r == 3 ? PAC_ROOT_OFF_3
         : r == 5 ? PAC_ROOT_OFF_5
         : r == 9 ? PAC_ROOT_OFF_9
         : r == 16 ? PAC_ROOT_OFF_16
         : r == 25 ? PAC_ROOT_OFF_25
         : r == 27 ? PAC_ROOT_OFF_27
         : r == 32 ? PAC_ROOT_OFF_32
                   : -1;
}

// z * w_R^e (forward) or z * conj(w_R^e) (inverse).  e and R are compile-time
// constants after unrolling, so the special cases fold away.
template <int R, bool INV, typename V> __device__ __forceinline__ V twiddle_const(V z, int e) {
    using T = typename Real<V>::T;
    e %= R;
    if (e == 0) return z;
    if ((8 * e) % R == 0) {
        const int o = (8 * e) / R;  // eighth turns
        const T h = T(0.70710678118654752440);
        V r;
        switch (INV ? (8 - o) : o) {  // multiply by exp(-2 pi i o / 8)
            case 1: r = V{(z.x + z.y) * h, (z.y - z.x) * h}; break;
            case 2: r = mul_mi(z); break;
            case 3: r = V{(z.y - z.x) * h, -(z.x + z.y) * h}; break;
            case 4: r = V{-z.x, -z.y}; break;
            case 5: r = V{-(z.x + z.y) * h, (z.x - z.y) * h}; break;
            case 6: r = mul_pi(z); break;
            default: r = V{(z.x - z.y) * h, (z.x + z.y) * h}; break;
        }
        return r;
    }
    const V w = root_const<V>(root_off(R) + e);
    return INV ? cmulc(z, w) : cmul(z, w);
}

constexpr int small_factor(int r) { return r % 4 == 0 && r > 4 ? 4 : (r % 2 == 0 ? 2 : (r % 3 == 0 ? 3 : 5)); }

// In-register DFT of size R, natural order in and out: v[k] = sum_j v[j] w^{jk}
// with w = exp(-2 pi i / R), or its conjugate (no scaling) when INV.
template <int R, bool INV, typename V> __device__ __forceinline__ void dft(V* v) {
    using T = typename Real<V>::T;
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const V w1 = root_const<V>(PAC_ROOT_OFF_3 + 1);  // (-1/2, -sqrt(3)/2)
        const V t = cadd(v[1], v[2]);
        const V d = csub(v[1], v[2]);
        const V m = V{v[0].x + w1.x * t.x, v[0].y + w1.x * t.y};
        // u = i * Im(w1) * d : forward Im(w1) = -sqrt(3)/2
        const T s = INV ? -w1.y : w1.y;
        const V u = V{-s * d.y, s * d.x};
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    } else if constexpr (R == 4) {
        const V a = v[0], b = v[1], c = v[2], d = v[3];
        const V s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
        const V r1 = INV ? mul_pi(d1) : mul_mi(d1);
        v[0] = cadd(s0, s1);
        v[2] = csub(s0, s1);
        v[1] = cadd(d0, r1);
        v[3] = csub(d0, r1);
    } else if constexpr (R == 5) {
        const V w1 = root_const<V>(PAC_ROOT_OFF_5 + 1);  // (cos 2pi/5, -sin 2pi/5)
        const V w2 = root_const<V>(PAC_ROOT_OFF_5 + 2);  // (cos 4pi/5, -sin 4pi/5)
        const T c1 = w1.x, c2 = w2.x;
        const T s1 = INV ? w1.y : -w1.y, s2 = INV ? w2.y : -w2.y;  // forward: +sin
        const V a = v[0];
        const V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        const V d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        const V m1 = V{a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
        const V m2 = V{a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
        // e1 = s1 d1 + s2 d2, e2 = s2 d1 - s1 d2; outputs m -/+ i e
        const V e1 = V{s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y};
        const V e2 = V{s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y};
        v[0] = cadd(a, cadd(t1, t2));
        v[1] = cadd(m1, mul_mi(e1));
        v[4] = cadd(m1, mul_pi(e1));
        v[2] = cadd(m2, mul_mi(e2));
        v[3] = cadd(m2, mul_pi(e2));
    } else {
        // Cooley-Tukey in registers: R = A * B, decimation in frequency.
        constexpr int A = small_factor(R);
        constexpr int B = R / A;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            V z[A];
#pragma unroll
            for (int a = 0; a < A; ++a) z[a] = v[b + B * a];
            dft<A, INV>(z);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[b + B * k1] = twiddle_const<R, INV>(z[k1], b * k1);
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
    }
}

// ------------------------------------------------------------------ passes

template <typename V> __device__ __forceinline__ V ld_tw(const void* p, int64_t i) {
    return __ldg(reinterpret_cast<const V*>(p) + i);
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

// asynchronous global -> shared copies (one element per instruction)
template <int BYTES> __device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

// Per-tile facts shared by the rounds of one tile.  Rows case (C > 1): a
// thread's column w = tid mod W is fixed within a tile.  Offsets are 32-bit
// element offsets (plans keep N < 2^31).
template <typename V> struct TileCtx {
    const PassArgs* a;
    V* s;              // tile in shared memory, [m][w], pitch P
    const V* hs;       // kFused, lines case: the spectrum tile in shared memory (or null)
    const V* twi;      // w_M^u
    uint32_t q0;       // first column of the tile
    uint32_t base;     // rows case: global offset of row 0 of this thread's column
    uint32_t C;        // row stride
    uint32_t j;        // rows case: external twiddle column j = (q mod C) / I
    bool valid;        // rows case: this thread's column exists (q < Q)
    bool do_scale;     // kFwd: multiply by `scale` on store (decided once, not per element)
    typename Real<V>::T scale;
};

// Task decomposition of round RI: task tau -> column w (fastest, so a warp
// reads consecutive shared-memory words), in-block offset jp, block bp.
template <int M, int W, int ES, int RI> struct Task {
    using G = RoundGeom<M, ES, RI>;
    static constexpr int TASKS = W * (M / G::R);
    int w, jp, row0;
    __device__ __forceinline__ explicit Task(int tau) {
        w = tau % W;
        const int t2 = tau / W;
        jp = t2 % G::SP;
        row0 = (t2 / G::SP) * G::S + jp;
    }
};

template <typename V, int M> struct Shape {
    static constexpr int ES = sizeof(V);
    static constexpr int W = tile_w(M, ES);
    static constexpr int P = tile_pitch(M, ES);
    static constexpr int NR = round_count(M, ES);
    static constexpr int NT = pass_threads(M, ES);
    static constexpr int TILE = M * P;
    // the fused lines pass stages the spectrum tile in shared memory when it fits
    static constexpr bool SPEC_SMEM = 2 * TILE * ES <= 200 * 1024;
};

// In-place forward round (rounds 0 .. NR-2): DFT_R then twiddles w_S^{jp k}.
template <typename V, int M, int RI>
__device__ __forceinline__ void fwd_round(const TileCtx<V>& c) {
    using SH = Shape<V, M>;
    using G = RoundGeom<M, SH::ES, RI>;
    using T = Task<M, SH::W, SH::ES, RI>;
    constexpr int R = G::R, SP = G::SP, STEP = M / G::S, P = SH::P;
    for (int tau = threadIdx.x; tau < T::TASKS; tau += SH::NT) {
        const T t(tau);
        V v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = c.s[(t.row0 + SP * u) * P + t.w];
        dft<R, false>(v);
        if constexpr (SP > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = cmul(v[k], c.twi[STEP * t.jp * k]);
        }
#pragma unroll
        for (int u = 0; u < R; ++u) c.s[(t.row0 + SP * u) * P + t.w] = v[u];
    }
}

// In-place inverse round RI (adjoint of forward round RI): conj twiddles,
// then the conjugate DFT.  FIRST_EXT: the pass' first inverse round in kInv,
// which also applies conj(w_L^{j k'}) to the rows loaded from the previous
// pass.  LAST_GLOBAL: round 0 of the rows case, stored straight to global.
template <typename V, int M, int RI, bool FIRST_EXT, bool LAST_GLOBAL>
__device__ __forceinline__ void inv_round(const TileCtx<V>& c) {
    using SH = Shape<V, M>;
    using G = RoundGeom<M, SH::ES, RI>;
    using T = Task<M, SH::W, SH::ES, RI>;
    constexpr int R = G::R, SP = G::SP, STEP = M / G::S, P = SH::P;
    const PassArgs& a = *c.a;
    V* dst = reinterpret_cast<V*>(a.dst);
    for (int tau = threadIdx.x; tau < T::TASKS; tau += SH::NT) {
        const T t(tau);
        V v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = c.s[(t.row0 + SP * u) * P + t.w];
        if constexpr (FIRST_EXT) {
            if (a.has_ext && c.j != 0) {
#pragma unroll
                for (int u = 0; u < R; ++u)
                    v[u] = cmulc(v[u], ext_twiddle<V>(a, (int64_t)c.j * __ldg(a.r2f + t.row0 + SP * u)));
            }
        }
        if constexpr (SP > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], c.twi[STEP * t.jp * k]);
        }
        dft<R, true>(v);
        if constexpr (LAST_GLOBAL) {
            if (c.valid) {
#pragma unroll
                for (int u = 0; u < R; ++u) dst[c.base + (uint32_t)(t.row0 + SP * u) * c.C] = v[u];
            }
        } else {
#pragma unroll
            for (int u = 0; u < R; ++u) c.s[(t.row0 + SP * u) * P + t.w] = v[u];
        }
    }
}

template <typename V, int M, int RI, bool LINES>
__device__ __forceinline__ void inv_rounds_from(const TileCtx<V>& c) {
    // rounds RI, RI-1, ..., 0; round RI is not the pass' first (no external factor)
    if constexpr (RI >= 0) {
        inv_round<V, M, RI, false, (!LINES && RI == 0)>(c);
        if constexpr (RI > 0 || LINES) __syncthreads();
        inv_rounds_from<V, M, RI - 1, LINES>(c);
    }
}

template <typename V, int M, int RI>
__device__ __forceinline__ void fwd_rounds_upto(const TileCtx<V>& c) {
    // rounds RI .. NR-2 in place
    if constexpr (RI < Shape<V, M>::NR - 1) {
        fwd_round<V, M, RI>(c);
        __syncthreads();
        fwd_rounds_upto<V, M, RI + 1>(c);
    }
}

// Last forward round (SP = 1: no internal twiddle).  kFwd, rows case: store
// to global row r2g[r] with w_L^{j k'} and the scale.  kFwd, lines case:
// in place (the store loop places rows).  kFused: product with the filter
// spectrum at the same global position, then the adjoint of this round.
template <typename V, int M, bool LINES, bool FUSED>
__device__ __forceinline__ void last_fwd_round(const TileCtx<V>& c) {
    using SH = Shape<V, M>;
    constexpr int RI = SH::NR - 1, P = SH::P;
    using G = RoundGeom<M, SH::ES, RI>;
    using T = Task<M, SH::W, SH::ES, RI>;
    constexpr int R = G::R;
    static_assert(G::SP == 1, "the last round acts on whole sub-blocks");
    const PassArgs& a = *c.a;
    V* dst = reinterpret_cast<V*>(a.dst);
    const V* spec = reinterpret_cast<const V*>(a.spec);
    for (int tau = threadIdx.x; tau < T::TASKS; tau += SH::NT) {
        const T t(tau);
        V v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = c.s[(t.row0 + u) * P + t.w];
        dft<R, false>(v);
        if constexpr (FUSED) {
            if constexpr (LINES && SH::SPEC_SMEM) {
#pragma unroll
                for (int u = 0; u < R; ++u) v[u] = cmul(v[u], c.hs[__ldg(a.r2g + t.row0 + u) * P + t.w]);
            } else {
                bool ok;
                uint32_t base;
                if constexpr (LINES) {
                    const uint32_t q = c.q0 + t.w;
                    ok = q < (uint32_t)a.Q;
                    base = q * M;
                } else {
                    ok = c.valid;
                    base = c.base;
                }
                if (ok) {
#pragma unroll
                    for (int u = 0; u < R; ++u) {
                        const uint32_t g = __ldg(a.r2g + t.row0 + u);
                        v[u] = cmul(v[u], __ldg(spec + base + g * c.C));
                    }
                }
            }
            dft<R, true>(v);
            if constexpr (!LINES && SH::NR == 1) {  // the only round: natural rows straight to global
                if (c.valid) {
#pragma unroll
                    for (int u = 0; u < R; ++u) dst[c.base + (uint32_t)(t.row0 + u) * c.C] = v[u];
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < R; ++u) c.s[(t.row0 + u) * P + t.w] = v[u];
        } else if constexpr (LINES) {
#pragma unroll
            for (int u = 0; u < R; ++u) c.s[(t.row0 + u) * P + t.w] = v[u];
        } else {
            if (c.valid) {
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int r = t.row0 + u;
                    V o = v[u];
                    if (a.has_ext && c.j != 0) o = cmul(o, ext_twiddle<V>(a, (int64_t)c.j * __ldg(a.r2f + r)));
                    if (c.do_scale) o = cscale(o, c.scale);
                    dst[c.base + (uint32_t)__ldg(a.r2g + r) * c.C] = o;
                }
            }
        }
    }
}

// Issue the asynchronous copy of one tile of `src` (natural rows; with
// `perm`, rows placed at rowmap[g], the in-CTA position of their frequency).
// Global order is walked contiguously: along rows of W columns (rows case)
// or along lines (C = 1).
template <typename V, int M, bool LINES>
__device__ __forceinline__ void load_tile(const PassArgs& a, const V* src, V* s, uint32_t q0, bool perm) {
    using SH = Shape<V, M>;
    constexpr int W = SH::W, P = SH::P, NT = SH::NT;
    const uint32_t Q = (uint32_t)a.Q;
    if constexpr (LINES) {
        const V* tile = src + q0 * M;
#pragma unroll 4
        for (int idx = threadIdx.x; idx < W * M; idx += NT) {
            const int w = idx / M, g = idx - (idx / M) * M;
            if (q0 + w >= Q) break;
            const int r = perm ? __ldg(a.rowmap + g) : g;
            cp_async<sizeof(V)>(s + r * P + w, tile + idx);
        }
    } else {
        const int w = threadIdx.x % W;
        const uint32_t q = q0 + w;
        if (q < Q) {
            const uint32_t C = (uint32_t)a.C;
            const uint32_t cq = q % C;
            const V* col = src + ((q - cq) * M + cq);
#pragma unroll 4
            for (int g = threadIdx.x / W; g < M; g += NT / W) {
                const int r = perm ? __ldg(a.rowmap + g) : g;
                cp_async<sizeof(V)>(s + r * P + w, col + (uint32_t)g * C);
            }
        }
    }
}

// Lines case: coalesced store of the tile; kFwd reads the row that holds
// global row g (rowmap) and scales, otherwise natural rows.
template <typename V, int M>
__device__ __forceinline__ void store_lines(const TileCtx<V>& c, bool placed) {
    using SH = Shape<V, M>;
    constexpr int W = SH::W, P = SH::P, NT = SH::NT;
    const PassArgs& a = *c.a;
    const V* s = c.s;
    const uint32_t q0 = c.q0;
    V* tile = reinterpret_cast<V*>(a.dst) + q0 * M;
    const uint32_t Q = (uint32_t)a.Q;
    for (int idx = threadIdx.x; idx < W * M; idx += NT) {
        const int w = idx / M, g = idx - (idx / M) * M;
        if (q0 + w >= Q) break;
        V v;
        if (placed) {
            v = s[__ldg(a.rowmap + g) * P + w];
            if (c.do_scale) v = cscale(v, c.scale);
        } else {
            v = s[g * P + w];
        }
        tile[idx] = v;
    }
}

// Programmatic dependent launch: let the next pass in the stream be scheduled
// now; wait here until the previous pass' writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Transform one tile that is resident in shared memory (all modes).
template <typename V, int M, bool LINES>
__device__ __forceinline__ void process_tile(TileCtx<V>& c) {
    using SH = Shape<V, M>;
    constexpr int NR = SH::NR;
    const PassArgs& a = *c.a;
    if (a.mode == kFwd) {
        fwd_rounds_upto<V, M, 0>(c);
        last_fwd_round<V, M, LINES, false>(c);
        if constexpr (LINES) {
            __syncthreads();
            store_lines<V, M>(c, true);
        }
    } else if (a.mode == kFused) {
        fwd_rounds_upto<V, M, 0>(c);
        last_fwd_round<V, M, LINES, true>(c);
        if constexpr (NR > 1 || LINES) __syncthreads();
        inv_rounds_from<V, M, NR - 2, LINES>(c);
        if constexpr (LINES) store_lines<V, M>(c, false);
    } else {
        // first inverse round: adjoint of the last forward round, with conj(w_L^{j k'})
        inv_round<V, M, NR - 1, true, (!LINES && NR == 1)>(c);
        if constexpr (NR > 1 || LINES) __syncthreads();
        inv_rounds_from<V, M, NR - 2, LINES>(c);
        if constexpr (LINES) store_lines<V, M>(c, false);
    }
}

// One pass over all tiles, CTAs walking tiles blockIdx.x, +gridDim.x, ...;
// with two buffers the asynchronous copy of the next tile (and, in the fused
// lines pass, of its spectrum tile) is in flight while the current tile is
// transformed.
template <typename V, int M, bool LINES>
__device__ __forceinline__ void run_phase(const PassArgs& a, V* sbase) {
    using SH = Shape<V, M>;
    constexpr int W = SH::W, STAGES = tile_stages(M, sizeof(V));
    constexpr bool HSMEM = LINES && SH::SPEC_SMEM;
    // buffer b: data at sbase + b * STRIDE, spectrum (HSMEM) right after it
    constexpr int STRIDE = (HSMEM ? 2 : 1) * SH::TILE;

    TileCtx<V> c;
    c.a = &a;
    c.twi = reinterpret_cast<const V*>(a.tw_int);
    c.C = (uint32_t)a.C;
    c.do_scale = a.mode == kFwd && a.scale != 1.0;
    c.scale = (typename Real<V>::T)a.scale;
    const uint32_t Q = (uint32_t)a.Q;
    const uint32_t tiles = (uint32_t)a.tiles;
    const V* src = reinterpret_cast<const V*>(a.src);
    const V* spec = reinterpret_cast<const V*>(a.spec);
    const bool perm = a.mode == kInv;
    const bool with_spec = HSMEM && a.mode == kFused;

    uint32_t t = blockIdx.x;
    if (STAGES == 2 && t < tiles) {
        load_tile<V, M, LINES>(a, src, sbase, t * W, perm);
        if (with_spec) load_tile<V, M, true>(a, spec, sbase + SH::TILE, t * W, false);
    }
    cp_async_commit();
    for (int it = 0; t < tiles; t += gridDim.x, ++it) {
        V* cur = sbase + (STAGES == 2 ? (it & 1) * STRIDE : 0);
        if constexpr (STAGES == 2) {
            const uint32_t tn = t + gridDim.x;
            if (tn < tiles) {
                V* nxt = sbase + ((it + 1) & 1) * STRIDE;
                load_tile<V, M, LINES>(a, src, nxt, tn * W, perm);
                if (with_spec) load_tile<V, M, true>(a, spec, nxt + SH::TILE, tn * W, false);
            }
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            load_tile<V, M, LINES>(a, src, cur, t * W, perm);
            if (with_spec) load_tile<V, M, true>(a, spec, cur + SH::TILE, t * W, false);
            cp_async_commit();
            cp_async_wait<0>();
        }
        __syncthreads();
        c.s = cur;
        c.hs = with_spec ? cur + SH::TILE : nullptr;
        c.q0 = t * W;
        c.valid = false;
        c.base = 0;
        c.j = 0;
        if constexpr (!LINES) {
            const uint32_t q = c.q0 + threadIdx.x % W;
            if (q < Q) {
                const uint32_t cq = q % c.C;
                c.valid = true;
                c.base = (q - cq) * M + cq;
                c.j = a.has_ext ? cq / (uint32_t)a.I : 0;
            }
        }
        process_tile<V, M, LINES>(c);
        __syncthreads();
    }
    cp_async_wait<0>();
}

template <typename V, int M> constexpr int pass_smem_bytes(bool lines) {
    return tile_stages(M, sizeof(V)) * ((lines && Shape<V, M>::SPEC_SMEM) ? 2 : 1) * Shape<V, M>::TILE *
           (int)sizeof(V);
}

// Generic pass kernel: one pass of a convolution (see run_phase).
template <typename V, int M, bool LINES>
__global__ void __launch_bounds__(pass_threads(M, sizeof(V)), min_blocks(M, sizeof(V))) pass_kernel(const PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    pdl_wait();
    run_phase<V, M, LINES>(a, reinterpret_cast<V*>(smem_raw));
}

// Grid-wide barrier for the cooperative convolution kernel (all CTAs are
// co-resident).  The arrival counter only grows; barrier k of a launch waits
// for base + (k+1) * gridDim.x arrivals.  The wait is bounded: after the
// limit the CTA records the failure in *error and goes on (no hang).
constexpr unsigned kBarrierSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void grid_barrier(const ConvArgs& args, unsigned k) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = args.base + (k + 1) * gridDim.x;
        __threadfence();
        atomicAdd(args.barrier, 1u);
        unsigned spins = 0;
        while ((int)(ld_acquire_gpu(args.barrier) - target) < 0) {
            if (++spins > kBarrierSpinLimit) {
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
    conv_kernel(const ConvArgs args) {
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
