// Persistent batched kernel: every pass of every instance of a batch in one
// launch.
//
// A CTA of kPersistThreads threads stays resident (one per SM) and pulls
// tiles from two device work lists in turn.  First the whole-CTA list (tiles
// of large groups and planes), then the quarter list: the CTA splits into
// four independent units of kPersistUnit threads, each pulling its own tiles
// of small groups into its quarter of the shared memory and synchronising
// with its own named barrier.  Within each list the passes are in level
// order.  A tile of pass p may start only when every tile of the pass before
// it in the same instance is done: per-pass counters of finished tiles,
// incremented after a tile's stores (a release-ordered add) and read with
// acquire loads by the unit's first thread before it starts.  Because tiles
// are handed out in level order and a unit takes its tiles in the order it
// got them (it fetches the next index while it runs the current tile), a
// wait only ever depends on tiles handed out earlier to running units, so it
// ends; it is
// still bounded (wait_cycles), after which the unit records 1 in the
// library's device error word and goes on.  The last CTA to finish resets
// the counters, so the same launch can be replayed (a captured graph).
#include <atomic>

#include "fft_device.cuh"
#include "pac_internal.h"
#include "persist.h"

namespace pac {

namespace {

// completion of a tile: one release-ordered add (the unit's stores, ordered by
// the unit's barrier before it, are visible to whoever acquires the count)
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// wait (first thread of the unit) until pass p's dependency is complete
__device__ __forceinline__ void wait_dep(const PersistArgs& A, const PersistPass& pp) {
    if (pp.dep < 0) return;
    const unsigned* c = A.ctr + 3 + pp.dep;
    const unsigned target = pp.dep_tiles + A.bias;
    if (ld_acquire(c) >= target) return;
    const long long t0 = clock64();
    while (ld_acquire(c) < target) {
        if (clock64() - t0 > A.wait_cycles) {
            atomicExch(A.error, 1u);
            return;
        }
        __nanosleep(64);
    }
}

// copy a pass record to shared memory with n threads (i = this thread's index among them)
__device__ __forceinline__ void copy_pass(const PersistPass* src, PersistPass* dst, int i, int n) {
    static_assert(sizeof(PersistPass) % 16 == 0, "whole 16-byte words");
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(dst);
    for (int k = i; k < (int)(sizeof(PersistPass) / 16); k += n) d4[k] = __ldg(s4 + k);
}

// one tile of a group pass with geometry GEO (GEO::tid() is the thread's index in its unit)
template <typename GEO, bool LINES>
__device__ __forceinline__ void group_tile(const PassArgs& a, uint32_t t, float2* s) {
    constexpr int M = GEO::M;
    TileCtx<float2> c;
    ctx_init(c, a, s);
    c.t = t;
    c.q0 = t * (uint32_t)GEO::W;
    c.valid = false;
    c.base = 0;
    c.j = 0;
    if constexpr (!LINES) {
        const uint32_t q = c.q0 + (uint32_t)(GEO::tid() % GEO::W);
        if (q < c.Q) {
            const uint32_t cq = q % c.C;
            c.valid = true;
            c.base = (q - cq) * (uint32_t)M + cq;
            c.j = a.has_ext ? cq / (uint32_t)a.I : 0;
        }
    }
    if (a.mode == kFwd)
        tile_forward<GEO, LINES>(c);
    else if (a.mode == kFused)
        tile_fused<GEO, LINES>(c);
    else
        tile_inverse<GEO, LINES>(c);
}

template <int M, bool LINES, int NT, bool SPLIT>
using PGeo = Geo<float2, M, tile_w(M, 8), NT, tile_pitch(M, 8, LINES), 1, SPLIT && kPersistPrefetch, 1, SPLIT,
                 tile_row_swizzle(M, 8)>;

// one item of shape I
template <int I>
__device__ __forceinline__ void shape_body(const PersistPass& pp, uint32_t t, float2* s) {
    constexpr PersistShape S = kPersistShapes[I];
    if constexpr (S.m2 > 0 && persist_quarter(I)) {
        plane_run<float2, S.m, S.m2, 1, PlaneShapeNT<float2, S.m, S.m2, kPersistUnit, true>>(pp.pa, t, 0u, s);
    } else if constexpr (S.m2 > 0) {
        plane_run<float2, S.m, S.m2, 1, PlaneShapeNT<float2, S.m, S.m2, kPersistThreads>>(pp.pa, t, 0u, s);
    } else if constexpr (persist_quarter(I)) {
        group_tile<PGeo<S.m, S.lines != 0, kPersistUnit, true>, S.lines != 0>(pp.pa.a1, t, s);
    } else {
        group_tile<PGeo<S.m, S.lines != 0, kPersistThreads, false>, S.lines != 0>(pp.pa.a1, t, s);
    }
}

// Most shapes are compiled as functions of their own, which the kernel
// calls (one inlined body of every shape takes minutes to compile); the
// groups of 512 and 1024 points, the bulk of a batch of mixed sizes, are
// inlined into the kernel (no call: no registers saved across it).
constexpr bool persist_inlined(int i) {
    return kPersistShapes[i].m2 == 0 && (kPersistShapes[i].m == 512 || kPersistShapes[i].m == 1024);
}

template <int I>
__device__ __noinline__ void shape_item(const PersistPass& pp, uint32_t t, float2* s) {
    shape_body<I>(pp, t, s);
}

// the item of shape `shape` (whole CTA when !QUARTER, a quarter unit otherwise)
template <bool QUARTER, int I = 0>
__device__ __forceinline__ void run_shape(int shape, const PersistPass& pp, uint32_t t, float2* s) {
    if constexpr (I < kPersistShapeCount) {
        if constexpr (persist_quarter(I) == QUARTER) {
            if (shape == I) {
                if constexpr (persist_inlined(I))
                    shape_body<I>(pp, t, s);
                else
                    shape_item<I>(pp, t, s);
                return;
            }
        }
        run_shape<QUARTER, I + 1>(shape, pp, t, s);
    }
}

__global__ void __launch_bounds__(kPersistThreads, 1) persist_kernel(const __grid_constant__ PersistArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    __shared__ uint32_t s_item[kPersistUnits];
    __shared__ int s_last;
    // the current item's pass record, copied into shared memory by its unit (or the whole CTA), so
    // that the tile code's many reads of its arguments hit shared memory, not a cold cache line
    __shared__ __align__(16) PersistPass s_pp[kPersistUnits];
    // whole-CTA items; the next index is fetched while the current item runs
    // (items are still taken in order, so every wait is on an earlier item)
    const uint32_t nfull_tiles = __ldg(A.starts + A.nfull);
    uint32_t next = 0;
    if (threadIdx.x == 0) next = atomicAdd(A.ctr + 0, 1u);
    for (;;) {
        if (threadIdx.x == 0) s_item[0] = next;
        __syncthreads();
        const uint32_t g = s_item[0];
        if (g >= nfull_tiles) break;
        if (threadIdx.x == 0) next = atomicAdd(A.ctr + 0, 1u);
        const int p = (int)__ldg(A.pass_of + g);
        copy_pass(A.passes + p, s_pp + 0, (int)threadIdx.x, kPersistThreads);
        if (threadIdx.x == 0) wait_dep(A, A.passes[p]);
        __syncthreads();
        const PersistPass& pp = s_pp[0];
        run_shape<false>(pp.shape, pp, g - __ldg(A.starts + p), s);
        __syncthreads();  // the tile's stores, and every read of s_item before the next write
        if (threadIdx.x == 0) red_release_add(A.ctr + 3 + p, 1u);
    }
    __syncthreads();  // every thread has read the last whole-CTA index before the units reuse s_item
    // quarter units
    if (A.npass > A.nfull) {
        const int unit = (int)(threadIdx.x / kPersistUnit);
        const bool lead = threadIdx.x % kPersistUnit == 0;
        float2* su = s + (size_t)unit * (kPersistQuarterSmem / sizeof(float2));
        const uint32_t q0 = __ldg(A.starts + A.nfull), qend = __ldg(A.starts + A.npass);
        uint32_t qnext = 0;
        if (lead) qnext = q0 + atomicAdd(A.ctr + 1, 1u);
        for (;;) {
            if (lead) s_item[unit] = qnext;
            unit_sync<kPersistUnit>();
            const uint32_t g = s_item[unit];
            if (g >= qend) break;
            if (lead) qnext = q0 + atomicAdd(A.ctr + 1, 1u);
            const int p = (int)__ldg(A.pass_of + g);
            copy_pass(A.passes + p, s_pp + unit, (int)(threadIdx.x % kPersistUnit), kPersistUnit);
            if (lead) wait_dep(A, A.passes[p]);
            unit_sync<kPersistUnit>();
            const PersistPass& pp = s_pp[unit];
            run_shape<true>(pp.shape, pp, g - __ldg(A.starts + p), su);
            unit_sync<kPersistUnit>();
            if (lead) red_release_add(A.ctr + 3 + p, 1u);
        }
    }
    // the last CTA out resets the counters for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's completion adds are performed before it counts itself out
        s_last = atomicAdd(A.ctr + 2, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = (int)threadIdx.x; i < 3 + A.npass; i += kPersistThreads) A.ctr[i] = 0u;
    }
}

}  // namespace

// CTAs of the persistent kernel resident at once (one per SM at most; 0: none fits)
int persist_grid(int dev, int smem) {
    static std::atomic<int> dyn_max[64];  // per device: the dynamic shared memory the kernel may take
    if (dev < 0 || dev >= 64) return 0;
    int lim = dyn_max[dev].load(std::memory_order_relaxed);
    if (lim == 0) {
        // what a CTA may take in all, less the kernel's static shared memory
        cudaFuncAttributes fa;
        int optin = 0;
        if (cudaFuncGetAttributes(&fa, persist_kernel) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();  // leave no error for a later launch check to find
            return 0;
        }
        lim = optin - (int)fa.sharedSizeBytes;
        if (lim <= 0 || cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) !=
                            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        dyn_max[dev].store(lim, std::memory_order_relaxed);
    }
    if (smem > lim) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persist_kernel, kPersistThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb > 0 ? device_sm_count(dev) : 0;
}

cudaError_t launch_persist(const PersistArgs& A, int grid, int smem, cudaStream_t s) {
    persist_kernel<<<grid, kPersistThreads, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace pac
