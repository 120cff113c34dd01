// Runtime-radix pass kernel for mixed groups (mixed radix, Section 7.1).
//
// A mixed group is a run of DIF stages of several prime bases (e.g. 48 =
// 16 x 3 or 1000 = 8 x 125 of an axis 2^a 3^b 5^c).  One kernel serves every
// such group size: the tile (W columns x M rows) is copied into shared
// memory (element (row, w) at row * P + w), transformed by rounds whose
// radices come with the launch (a switch over the radices a round can have
// selects the in-register DFT), and copied out.  The copy-in and copy-out
// carry what the first and last rounds of the one-base kernels do in
// registers: the placement of frequencies (rowmap) and the external factor
// w_L^{j k'}.  Round i has block length S_i = M / (R_0 ... R_{i-1})
// and applies w_{S_i}^{jp k} after its forward DFT, as in round_exec.
#pragma once

#include "fft_device.cuh"

namespace pac {

template <typename V> struct MixCtx {
    const PassArgs* a;
    V* s;           // the tile, [row][w], pitch P
    int M, W, P;
    uint32_t t;     // tile index
    uint32_t q0;    // first column
};

// One round of radix R over the tile (block length S).  INV: conjugate
// twiddles, then the conjugate DFT.  MUL (the last forward round, S == R):
// DFT, product with the spectrum slots of this tile, conjugate DFT.
template <typename V, int R, bool INV, bool MUL>
__device__ __forceinline__ void mix_round(const MixCtx<V>& c, int S) {
    const int SP = S / R, STEP = c.M / S;
    const int tasks = c.W * (c.M / R);
    const V* twi = reinterpret_cast<const V*>(c.a->tw_int);
    const V* spec = nullptr;
    if constexpr (MUL) spec = reinterpret_cast<const V*>(c.a->spec) + (size_t)c.t * c.W * c.M;
#pragma unroll 1
    for (int tau = threadIdx.x; tau < tasks; tau += blockDim.x) {
        const int w = tau % c.W, t2 = tau / c.W;
        const int jp = t2 % SP, row0 = (t2 / SP) * S + jp;
        V v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = c.s[(row0 + SP * u) * c.P + w];
        if constexpr (INV) {
            if (SP > 1) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], __ldg(twi + STEP * jp * k));
            }
            dft<R, true>(v);
        } else {
            dft<R, false>(v);
            if constexpr (MUL) {
#pragma unroll
                for (int u = 0; u < R; ++u) v[u] = cmul(v[u], __ldg(spec + u * tasks + tau));
                dft<R, true>(v);
            } else {
                if (SP > 1) {
#pragma unroll
                    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], __ldg(twi + STEP * jp * k));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) c.s[(row0 + SP * u) * c.P + w] = v[u];
    }
}

// the round radices a mixed group can have (mix_rmax of each base and its divisors)
template <typename V, bool INV, bool MUL>
__device__ __forceinline__ void mix_round_rt(const MixCtx<V>& c, int R, int S) {
    switch (R) {
        case 2: mix_round<V, 2, INV, MUL>(c, S); break;
        case 3: mix_round<V, 3, INV, MUL>(c, S); break;
        case 4: mix_round<V, 4, INV, MUL>(c, S); break;
        case 5: mix_round<V, 5, INV, MUL>(c, S); break;
        case 8: mix_round<V, 8, INV, MUL>(c, S); break;
        case 9: mix_round<V, 9, INV, MUL>(c, S); break;
        case 16: mix_round<V, 16, INV, MUL>(c, S); break;
        case 25: mix_round<V, 25, INV, MUL>(c, S); break;
        default: break;  // the plan builder never forms other radices
    }
}

// Copies between the tile and global memory keep kMixBatch loads of each
// thread in flight.  Rows case: NT is a multiple of W, so a thread keeps one
// column w = tid mod W (its global offset and external-twiddle column j are
// computed once) and walks rows tid / W, + NT / W, ...; a warp reads row
// segments.  Lines case: the tile's lines are contiguous in global memory
// and the threads walk them in order.
constexpr int kMixBatch = 8;

struct MixCol {
    uint32_t base, j;
    bool valid;
};

template <typename V> __device__ __forceinline__ MixCol mix_col(const MixCtx<V>& c, int w) {
    const PassArgs& a = *c.a;
    const uint32_t q = c.q0 + (uint32_t)w, C = (uint32_t)a.C;
    MixCol k;
    k.valid = q < (uint32_t)a.Q;
    const uint32_t cq = k.valid ? q % C : 0u;
    k.base = k.valid ? (q - cq) * (uint32_t)c.M + cq : 0u;
    k.j = a.has_ext && k.valid ? cq / (uint32_t)a.I : 0u;
    return k;
}

// elements of the tile's lines that exist (lines case)
template <typename V> __device__ __forceinline__ uint32_t mix_line_elems(const MixCtx<V>& c) {
    const uint32_t Q = (uint32_t)c.a->Q;
    const uint32_t q1 = c.q0 + (uint32_t)c.W < Q ? c.q0 + (uint32_t)c.W : Q;
    return (q1 - c.q0) * (uint32_t)c.M;
}

// Copy-in.  Natural rows (forward input): in-tile row = global row.  Placed
// rows (inverse input): global row g holds frequency freq[g] at in-tile row
// rowmap[g]; the conjugate external factor is applied on the way in.
template <typename V, bool LINES>
__device__ __forceinline__ void mix_load(const MixCtx<V>& c, bool placed) {
    const PassArgs& a = *c.a;
    const V* src = reinterpret_cast<const V*>(a.src);
    const int NT = blockDim.x;
    if constexpr (LINES) {
        const uint32_t n = mix_line_elems(c), base = c.q0 * (uint32_t)c.M;
#pragma unroll 1
        for (uint32_t e0 = threadIdx.x; e0 < n; e0 += kMixBatch * NT) {
            V v[kMixBatch];
#pragma unroll
            for (int b = 0; b < kMixBatch; ++b) {
                const uint32_t e = e0 + (uint32_t)(b * NT);
                if (e < n) v[b] = src[base + e];
            }
#pragma unroll
            for (int b = 0; b < kMixBatch; ++b) {
                const uint32_t e = e0 + (uint32_t)(b * NT);
                if (e < n) {
                    const int w = (int)(e / (uint32_t)c.M), g = (int)e - w * c.M;
                    const int row = placed ? __ldg(a.rowmap + g) : g;
                    c.s[row * c.P + w] = v[b];
                }
            }
        }
    } else {
        const int w = threadIdx.x % c.W, step = NT / c.W;
        const MixCol k = mix_col(c, w);
        if (!k.valid) return;
        const uint32_t C = (uint32_t)a.C;
#pragma unroll 1
        for (int g0 = threadIdx.x / c.W; g0 < c.M; g0 += kMixBatch * step) {
            V v[kMixBatch];
#pragma unroll
            for (int b = 0; b < kMixBatch; ++b) {
                const int g = g0 + b * step;
                if (g < c.M) v[b] = src[k.base + (uint32_t)g * C];
            }
#pragma unroll
            for (int b = 0; b < kMixBatch; ++b) {
                const int g = g0 + b * step;
                if (g < c.M) {
                    V x = v[b];
                    int row = g;
                    if (placed) {
                        row = __ldg(a.rowmap + g);
                        if (k.j != 0) x = cmulc(x, ext_twiddle<V>(a, (int64_t)k.j * __ldg(a.freq + g)));
                    }
                    c.s[row * c.P + w] = x;
                }
            }
        }
    }
}

// Copy-out.  Placed rows (forward output): global row g takes in-tile row
// rowmap[g], times w_L^{j freq[g]}; natural rows otherwise.
template <typename V, bool LINES>
__device__ __forceinline__ void mix_store(const MixCtx<V>& c, bool placed) {
    const PassArgs& a = *c.a;
    V* dst = reinterpret_cast<V*>(a.dst);
    const int NT = blockDim.x;
    if constexpr (LINES) {
        const uint32_t n = mix_line_elems(c), base = c.q0 * (uint32_t)c.M;
#pragma unroll 4
        for (uint32_t e = threadIdx.x; e < n; e += NT) {
            const int w = (int)(e / (uint32_t)c.M), g = (int)e - w * c.M;
            const int row = placed ? __ldg(a.rowmap + g) : g;
            V v = c.s[row * c.P + w];
            dst[base + e] = v;
        }
    } else {
        const int w = threadIdx.x % c.W, step = NT / c.W;
        const MixCol k = mix_col(c, w);
        if (!k.valid) return;
        const uint32_t C = (uint32_t)a.C;
#pragma unroll 4
        for (int g = threadIdx.x / c.W; g < c.M; g += step) {
            const int row = placed ? __ldg(a.rowmap + g) : g;
            V v = c.s[row * c.P + w];
            if (placed) {
                if (k.j != 0) v = cmul(v, ext_twiddle<V>(a, (int64_t)k.j * __ldg(a.freq + g)));
                }
            dst[k.base + (uint32_t)g * C] = v;
        }
    }
}

// One tile of a mixed pass: kFwd (natural in, placed out), kInv (placed in,
// natural out) or kFused (natural in, forward rounds, product, inverse
// rounds, natural out).
template <typename V, bool LINES>
__device__ __forceinline__ void mix_tile(const PassArgs& a, V* s, uint32_t t) {
    MixCtx<V> c;
    c.a = &a;
    c.s = s;
    c.M = a.mix_m;
    c.W = a.mix_w;
    c.P = a.mix_w + 1;
    c.t = t;
    c.q0 = t * (uint32_t)a.mix_w;
    const int nr = a.mix_nr;
    int S[kMixMaxRounds];
    S[0] = c.M;
    for (int i = 1; i < nr; ++i) S[i] = S[i - 1] / a.mix_r[i - 1];
    if (a.mode == kInv) {
        mix_load<V, LINES>(c, true);
        for (int i = nr - 1; i >= 0; --i) {
            __syncthreads();
            mix_round_rt<V, true, false>(c, a.mix_r[i], S[i]);
        }
        __syncthreads();
        mix_store<V, LINES>(c, false);
    } else {
        mix_load<V, LINES>(c, false);
        const bool fused = a.mode == kFused;
        for (int i = 0; i < nr; ++i) {
            __syncthreads();
            if (fused && i == nr - 1)
                mix_round_rt<V, false, true>(c, a.mix_r[i], S[i]);
            else
                mix_round_rt<V, false, false>(c, a.mix_r[i], S[i]);
        }
        if (fused) {
            for (int i = nr - 2; i >= 0; --i) {
                __syncthreads();
                mix_round_rt<V, true, false>(c, a.mix_r[i], S[i]);
            }
        }
        __syncthreads();
        mix_store<V, LINES>(c, !fused);
    }
}

constexpr int mix_min_blocks(int esize) { return esize == 8 ? 2 : 1; }

// one CTA per tile
template <typename V, bool LINES>
__global__ void __launch_bounds__(kMixThreads, mix_min_blocks(sizeof(V))) mix_kernel(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    pdl_wait();
    mix_tile<V, LINES>(a, reinterpret_cast<V*>(smem_raw), blockIdx.x);
}

// batched form: the tiles of list[0..n) numbered consecutively (as pass_multi_kernel)
template <typename V, bool LINES>
__global__ void __launch_bounds__(kMixThreads, mix_min_blocks(sizeof(V)))
    mix_multi_kernel(const PassArgs* __restrict__ list, const uint32_t* __restrict__ tile_start, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const uint32_t total = __ldg(tile_start + n);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tile_start + mid) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        mix_tile<V, LINES>(list[lo], s, t - __ldg(tile_start + lo));
        __syncthreads();
    }
}

}  // namespace pac
