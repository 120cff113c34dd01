// TMA-fed lines pass: the pass of a contiguous-axis group of large size M
// (the axis whose lines are contiguous; for a convolution the fused pass:
// forward rounds, product with the filter spectrum, inverse rounds).
//
// A tile is W consecutive lines, i.e. one contiguous stretch of W * M
// elements, and the fused pass' spectrum tile is one contiguous stretch of
// W * M slots.  Each CTA is persistent: it walks tiles blockIdx.x,
// + gridDim.x, ... and, while it computes tile k in shared-memory buffer
// k mod 2, the bulk copy engine (cp.async.bulk, completing on an mbarrier)
// brings tile k + 1 into the other buffer.  The first round reads the staged
// lines in place (round_staged), the later rounds exchange through the same
// buffer, and the last round writes global memory from registers.  Tiles
// whose stretch is not 16-byte aligned or sized (a last partial tile of an
// odd-length FP32 line) are copied in by the CTA's threads instead.  A wait
// that does not complete within about a second records 1 in the library's
// device error word, waits (bounded) for the copies it issued and returns.
#pragma once
#include "fft_device.cuh"
#include "tma.cuh"

namespace pac {

template <typename V, int M> struct TmaShape {
    static constexpr int ES = sizeof(V);
    static constexpr int W = tma_w(M, ES);
    static constexpr int NT = tma_threads(M, ES);
    static constexpr int P = tma_pitch(M, ES);
    static constexpr int BUF = tma_buf(M, ES);
    using GEO = Geo<V, M, W, NT, P, 1, false>;
    static_assert(NT % W == 0, "whole tasks per thread");
};

// Arguments: one pass (n == 1, `one`) or n passes of this shape whose tiles
// are numbered consecutively (list and starts in device memory, as for
// pass_multi_kernel).
struct LinesTmaArgs {
    PassArgs one;
    const PassArgs* list;
    const uint32_t* starts;
    int n;
    uint32_t total;      // tiles over all passes
    int stage_spec;      // the launch has fused passes: stage their spectrum tiles too
    unsigned* error;     // device error word
};

constexpr long long kTmaWaitCycles = 2000000000LL;  // about a second at the GPU's clocks

template <typename V, int M> struct TmaTile {
    const PassArgs* a;
    uint32_t lt;      // tile within its pass
    uint32_t q0;      // first line
    uint32_t lines;   // lines in the tile
};

template <typename V, int M>
__device__ __forceinline__ TmaTile<V, M> tma_tile(const LinesTmaArgs& ta, uint32_t gt) {
    using TS = TmaShape<V, M>;
    TmaTile<V, M> r;
    if (ta.n == 1) {
        r.a = &ta.one;
        r.lt = gt;
    } else {
        int lo = 0, hi = ta.n - 1;  // the last pass whose first tile is <= gt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(ta.starts + mid) <= gt)
                lo = mid;
            else
                hi = mid - 1;
        }
        r.a = ta.list + lo;
        r.lt = gt - __ldg(ta.starts + lo);
    }
    r.q0 = r.lt * (uint32_t)TS::W;
    const uint32_t Q = (uint32_t)r.a->Q;
    r.lines = Q - r.q0 < (uint32_t)TS::W ? Q - r.q0 : (uint32_t)TS::W;
    return r;
}

// bytes of the tile's lines and of its spectrum slots (0: none), and whether
// both can be bulk-copied (16-byte aligned start and size)
template <typename V, int M>
__device__ __forceinline__ bool tma_ok(const TmaTile<V, M>& tl, bool spec, unsigned* xb, unsigned* sb) {
    using TS = TmaShape<V, M>;
    const uintptr_t xs = reinterpret_cast<uintptr_t>(tl.a->src) + (uintptr_t)tl.q0 * M * sizeof(V);
    *xb = tl.lines * (unsigned)M * (unsigned)sizeof(V);
    bool ok = (xs % 16) == 0 && (*xb % 16) == 0;
    *sb = 0;
    if (spec) {
        const uintptr_t ss = reinterpret_cast<uintptr_t>(tl.a->spec) + (uintptr_t)tl.lt * TS::W * M * sizeof(V);
        *sb = (unsigned)(TS::W * M * sizeof(V));
        ok = ok && (ss % 16) == 0 && (*sb % 16) == 0;
    }
    return ok;
}

template <typename V, int M>
__device__ __forceinline__ void tma_issue(const TmaTile<V, M>& tl, bool spec, unsigned xb, unsigned sb, V* xbuf,
                                          V* sbuf, uint64_t* bar) {
    using TS = TmaShape<V, M>;
    fence_proxy_async_smem();  // the buffer's earlier reads and writes by the CTA come first
    mbar_arrive_expect_tx(bar, xb + sb);
    bulk_copy_g2s(xbuf, reinterpret_cast<const V*>(tl.a->src) + (size_t)tl.q0 * M, xb, bar);
    if (spec) bulk_copy_g2s(sbuf, reinterpret_cast<const V*>(tl.a->spec) + (size_t)tl.lt * TS::W * M, sb, bar);
}

template <typename V, int M>
__global__ void __launch_bounds__(TmaShape<V, M>::NT, 1) lines_tma_kernel(const __grid_constant__ LinesTmaArgs ta) {
    using TS = TmaShape<V, M>;
    using GEO = typename TS::GEO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // two barriers, one per buffer
    V* const x0 = reinterpret_cast<V*>(smem_raw + 128);
    V* const x1 = x0 + TS::BUF;
    V* const s0 = x1 + TS::BUF;
    V* const s1 = s0 + TS::W * M;
    __shared__ int s_ok;
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(bar + 0, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();  // the previous pass' output is complete and visible
    // per buffer: the parity of its next phase, and (thread 0) whether a bulk copy into it is in flight;
    // kept as scalars selected by the buffer index (no local-memory arrays)
    unsigned par0 = 0u, par1 = 0u;
    bool pend0 = false, pend1 = false;
    const uint32_t G = gridDim.x;
    uint32_t gt = blockIdx.x;
    if (gt < ta.total && threadIdx.x == 0) {  // the first tile's copy
        const TmaTile<V, M> tl = tma_tile<V, M>(ta, gt);
        const bool spec = ta.stage_spec && tl.a->mode == kFused;
        unsigned xb, sb;
        if (tma_ok<V, M>(tl, spec, &xb, &sb)) {
            tma_issue<V, M>(tl, spec, xb, sb, x0, s0, bar + 0);
            pend0 = true;
        }
    }
    for (uint32_t k = 0; gt < ta.total; ++k, gt += G) {
        const bool odd = (k & 1u) != 0;
        V* const xcur = odd ? x1 : x0;
        V* const scur = odd ? s1 : s0;
        uint64_t* const bcur = bar + (odd ? 1 : 0);
        const TmaTile<V, M> tl = tma_tile<V, M>(ta, gt);
        const bool spec = ta.stage_spec && tl.a->mode == kFused;
        unsigned xb, sb;
        const bool bulk = tma_ok<V, M>(tl, spec, &xb, &sb);
        // the next tile's copy into the other buffer (free: the previous tile ended with a barrier)
        const uint32_t gn = gt + G;
        if (gn < ta.total && threadIdx.x == 0) {
            const TmaTile<V, M> tn = tma_tile<V, M>(ta, gn);
            const bool nspec = ta.stage_spec && tn.a->mode == kFused;
            unsigned nxb, nsb;
            if (tma_ok<V, M>(tn, nspec, &nxb, &nsb)) {
                tma_issue<V, M>(tn, nspec, nxb, nsb, odd ? x0 : x1, odd ? s0 : s1, bar + (odd ? 0 : 1));
                if (odd)
                    pend0 = true;
                else
                    pend1 = true;
            }
        }
        if (bulk) {
            const unsigned pc = odd ? par1 : par0;
            if (threadIdx.x == 0) s_ok = mbar_wait_bounded(bcur, pc, kTmaWaitCycles) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {  // the copy did not complete: report, wait (bounded) for the copies in flight, return
                if (threadIdx.x == 0) {
                    atomicExch(ta.error, 1u);
                    (void)mbar_wait_bounded(bcur, pc, kTmaWaitCycles);
                    if (odd ? pend0 : pend1) (void)mbar_wait_bounded(bar + (odd ? 0 : 1), odd ? par0 : par1,
                                                                     kTmaWaitCycles);
                }
                return;
            }
            (void)mbar_test_parity(bcur, pc);  // each thread observes the completed phase
            if (odd) {
                par1 ^= 1u;
                pend1 = false;
            } else {
                par0 ^= 1u;
                pend0 = false;
            }
        } else {  // a tile the bulk engine cannot take: the threads copy it
            const V* xs = reinterpret_cast<const V*>(tl.a->src) + (size_t)tl.q0 * M;
            for (uint32_t i = threadIdx.x; i < tl.lines * (uint32_t)M; i += TS::NT) xcur[i] = xs[i];
            if (spec) {
                const V* ss = reinterpret_cast<const V*>(tl.a->spec) + (size_t)tl.lt * TS::W * M;
                for (uint32_t i = threadIdx.x; i < (uint32_t)(TS::W * M); i += TS::NT) scur[i] = ss[i];
            }
            __syncthreads();
        }
        TileCtx<V> c;
        ctx_init(c, *tl.a, xcur);
        c.t = tl.lt;
        c.q0 = tl.q0;
        c.valid = true;
        c.base = 0;
        c.j = 0;
        c.stage = xcur;
        c.sstage = spec ? scur : nullptr;
        const int mode = tl.a->mode;
        if (mode == kFwd)
            tile_forward_staged<GEO>(c);
        else if (mode == kFused)
            tile_fused_staged<GEO>(c);
        else
            tile_inverse_staged<GEO>(c);
        __syncthreads();  // the buffer is free for the copy issued at the start of tile k + 2
    }
}

}  // namespace pac
