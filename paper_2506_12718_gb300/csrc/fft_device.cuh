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

template <int M, int ES, int RI> struct RoundGeom {
    static constexpr int R = round_radix(M, ES, RI);
    // block length before this round: M / (R_0 ... R_{RI-1})
    static constexpr int S = RI == 0 ? M : RoundGeom<M, ES, RI - 1>::S / RoundGeom<M, ES, RI - 1>::R;
    static constexpr int SP = S / R;
};
template <int M, int ES> struct RoundGeom<M, ES, -1> {
    static constexpr int R = 1, S = M * 1, SP = M;
};

// One in-place decimation-in-frequency round over every column of the tile
// (forward), or its adjoint (INV): pre-twiddle by conj, then conj DFT.
template <typename V, int M, int W, int P, int RI, bool INV>
__device__ __forceinline__ void tile_round(V* s, const V* __restrict__ twi) {
    constexpr int ES = sizeof(V);
    using G = RoundGeom<M, ES, RI>;
    constexpr int R = G::R, S = G::S, SP = G::SP;
    constexpr int TASKS = W * (M / R);
    constexpr int STEP = M / S;  // w_S^x = w_M^{STEP x}
    for (int tau = threadIdx.x; tau < TASKS; tau += kThreads) {
        const int w = tau % W;
        const int t2 = tau / W;
        const int jp = t2 % SP;
        const int bp = t2 / SP;
        const int row0 = bp * S + jp;
        V v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = s[(row0 + SP * u) * P + w];
        if constexpr (INV) {
            if constexpr (SP > 1) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], twi[STEP * jp * k]);
            }
            dft<R, true>(v);
        } else {
            dft<R, false>(v);
            if constexpr (SP > 1) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twi[STEP * jp * k]);
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) s[(row0 + SP * u) * P + w] = v[u];
    }
}

template <typename V, int M, int W, int P, int RI, int NR>
__device__ __forceinline__ void rounds_fwd(V* s, const V* twi) {
    if constexpr (RI < NR) {
        tile_round<V, M, W, P, RI, false>(s, twi);
        __syncthreads();
        rounds_fwd<V, M, W, P, RI + 1, NR>(s, twi);
    }
}
template <typename V, int M, int W, int P, int RI>
__device__ __forceinline__ void rounds_inv(V* s, const V* twi) {
    if constexpr (RI >= 0) {
        tile_round<V, M, W, P, RI, true>(s, twi);
        __syncthreads();
        rounds_inv<V, M, W, P, RI - 1>(s, twi);
    }
}

// Generic pass kernel: a tile is W consecutive columns x M rows, held in
// shared memory as [m][w] (pitch P).  Columns are independent M-point
// transforms.  Loads and stores walk global memory contiguously: along the
// rows (W columns side by side, C > 1) or along whole lines (C == 1).
template <typename V, int M>
__global__ void __launch_bounds__(kThreads) pass_kernel(const PassArgs a) {
    constexpr int ES = sizeof(V);
    constexpr int W = tile_w(M, ES);
    constexpr int P = tile_pitch(M, ES);
    constexpr int NR = round_count(M, ES);
    constexpr int GS = kThreads / W;  // rows a thread block covers per step (rows case)
    static_assert(W <= kThreads && kThreads % W == 0, "tile width");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const V* src = reinterpret_cast<const V*>(a.src);
    V* dst = reinterpret_cast<V*>(a.dst);
    const V* twi = reinterpret_cast<const V*>(a.tw_int);
    const V* spec = reinterpret_cast<const V*>(a.spec);
    const bool lines = (a.C == 1);
    const int wr = threadIdx.x % W;   // rows case: this thread's column
    const int g0 = threadIdx.x / W;   // rows case: first row

    for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
        const int64_t q0 = tile * W;
        // per-thread column facts for the rows case
        const int64_t qr = q0 + wr;
        const bool qr_ok = qr < a.Q;
        int64_t base_r = 0, j_r = 0;
        if (!lines && qr_ok) {
            const int64_t cq = qr % a.C;
            base_r = (qr - cq) * M + cq;
            if (a.has_ext) j_r = cq / a.I;
        }
        // ---------------------------------------------------------- load
        if (lines) {
            for (int idx = threadIdx.x; idx < W * M; idx += kThreads) {
                const int w = idx / M, g = idx - (idx / M) * M;
                const int64_t q = q0 + w;
                if (q >= a.Q) break;
                const int r = (a.mode == kInv) ? __ldg(a.rowmap + g) : g;  // L' = 1: no external factor
                s[r * P + w] = src[q * M + g];
            }
        } else if (qr_ok) {
            for (int g = g0; g < M; g += GS) {
                V v = src[base_r + g * a.C];
                int r = g;
                if (a.mode == kInv) {
                    r = __ldg(a.rowmap + g);
                    if (a.has_ext) v = cmulc(v, ext_twiddle<V>(a, j_r * __ldg(a.freq + g)));
                }
                s[r * P + wr] = v;
            }
        }
        __syncthreads();
        // ---------------------------------------------------------- compute
        if (a.mode != kInv) rounds_fwd<V, M, W, P, 0, NR>(s, twi);
        if (a.mode == kFused) {
            if (lines) {
                for (int idx = threadIdx.x; idx < W * M; idx += kThreads) {
                    const int w = idx / M, g = idx - (idx / M) * M;
                    const int64_t q = q0 + w;
                    if (q >= a.Q) break;
                    const int r = __ldg(a.rowmap + g);
                    s[r * P + w] = cmul(s[r * P + w], __ldg(spec + q * M + g));
                }
            } else if (qr_ok) {
                for (int g = g0; g < M; g += GS) {
                    const int r = __ldg(a.rowmap + g);
                    s[r * P + wr] = cmul(s[r * P + wr], __ldg(spec + base_r + g * a.C));
                }
            }
            __syncthreads();
        }
        if (a.mode != kFwd) rounds_inv<V, M, W, P, NR - 1>(s, twi);
        // ---------------------------------------------------------- store
        if (lines) {
            for (int idx = threadIdx.x; idx < W * M; idx += kThreads) {
                const int w = idx / M, g = idx - (idx / M) * M;
                const int64_t q = q0 + w;
                if (q >= a.Q) break;
                V v;
                if (a.mode == kFwd) {
                    v = s[__ldg(a.rowmap + g) * P + w];
                    if (a.scale != 1.0) v = cscale(v, (typename Real<V>::T)a.scale);
                } else {
                    v = s[g * P + w];
                }
                dst[q * M + g] = v;
            }
        } else if (qr_ok) {
            for (int g = g0; g < M; g += GS) {
                V v;
                if (a.mode == kFwd) {
                    v = s[__ldg(a.rowmap + g) * P + wr];
                    if (a.has_ext) v = cmul(v, ext_twiddle<V>(a, j_r * __ldg(a.freq + g)));
                    if (a.scale != 1.0) v = cscale(v, (typename Real<V>::T)a.scale);
                } else {
                    v = s[g * P + wr];
                }
                dst[base_r + g * a.C] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace pac
