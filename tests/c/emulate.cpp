// CPU emulation of the pass kernels for the CPU tests: the kernels' own code
// (csrc/fft_device.cuh: run_phase, the rounds, the placement and the
// spectrum order) built for the host, one CTA of NT host threads per pass
// (thread-local threadIdx, __syncthreads as a barrier of the CTA's threads,
// the exchange buffer in host memory), driven by the step records of
// pac_test_host_steps (libpac: the plan's groups and tables).
//   emulate <dtype 0|1|2> <radix> <cap> <flags> <ndim> <d0> [d1] [d2] <h file> <x file> <y file>
// (flags bit 0: the plane pass, one CTA per plane, where the shape has one;
// bit 1: groups spanning prime bases with compiled kernels; bit 2: groups
// spanning bases in the runtime-radix kernel)
// h and x: N complex elements (complex64 for dtype 0, complex128 otherwise);
// y is written in the same format.
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __uint_as_float(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline uint32_t __float_as_uint(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
static inline int __double2hiint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)(b >> 32); }
static inline int __double2loint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)b; }
static inline double __hiloint2double(int hi, int lo) {
    const uint64_t b = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}
static inline float __uint2float_rn(uint32_t u) { return (float)u; }
template <typename T> static inline T __ldg(const T* p) { return *p; }
static thread_local uint3 threadIdx, blockIdx;
static thread_local dim3 blockDim, gridDim;
static thread_local std::barrier<>* g_cta_barrier = nullptr;
static inline void __syncthreads() { g_cta_barrier->arrive_and_wait(); }
static inline void __threadfence() {}
static inline unsigned atomicAdd(unsigned* p, unsigned v) { const unsigned o = *p; *p += v; return o; }
static inline unsigned atomicExch(unsigned* p, unsigned v) { const unsigned o = *p; *p = v; return o; }
static inline long long clock64() { return 0; }
static inline void __nanosleep(unsigned) {}
#define __launch_bounds__(...)

#include "fft_device.cuh"
#include "mix.cuh"
#include "pac.h"

using namespace pac;

// one pass: a single CTA of NT host threads walks every tile (run_phase's
// loop over blockIdx.x, +gridDim.x with a grid of one)
template <typename V, int M, bool LINES> static void run_pass(const PassArgs& a) {
    using SH = Shape<V, M, LINES, 0>;
    const int nt = SH::NT;
    std::vector<unsigned char> smem(pass_smem_bytes<V, M, 0>(LINES) + 16);
    V* s = reinterpret_cast<V*>((reinterpret_cast<uintptr_t>(smem.data()) + 15) & ~uintptr_t(15));
    std::barrier<> bar(nt);
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i)
        th.emplace_back([&, i] {
            threadIdx = uint3{(unsigned)i, 0u, 0u};
            blockIdx = uint3{0u, 0u, 0u};
            blockDim = dim3((unsigned)nt);
            gridDim = dim3(1u);
            g_cta_barrier = &bar;
            run_phase<V, M, LINES, 0>(a, s);
        });
    for (auto& t : th) t.join();
}

template <typename V, int M> static bool pass_m(const HostStep& st) {
    if (st.lines)
        run_pass<V, M, true>(st.a);
    else
        run_pass<V, M, false>(st.a);
    return true;
}

// a pass of the runtime-radix kernel: one CTA of kMixThreads host threads walks every tile
template <typename V, bool LINES> static void run_mix(const PassArgs& a) {
    const int nt = kMixThreads;
    std::vector<unsigned char> smem(mix_smem_bytes(a.mix_m, (int)sizeof(V)) + 16);
    V* s = reinterpret_cast<V*>((reinterpret_cast<uintptr_t>(smem.data()) + 15) & ~uintptr_t(15));
    std::barrier<> bar(nt);
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i)
        th.emplace_back([&, i] {
            threadIdx = uint3{(unsigned)i, 0u, 0u};
            blockIdx = uint3{0u, 0u, 0u};
            blockDim = dim3((unsigned)nt);
            gridDim = dim3(1u);
            g_cta_barrier = &bar;
            for (uint32_t t = 0; t < (uint32_t)a.tiles; ++t) {
                mix_tile<V, LINES>(a, s, t);
                __syncthreads();
            }
        });
    for (auto& t : th) t.join();
}

template <typename V> static bool dispatch(const HostStep& st) {
    if (st.a.mix_nr > 0) {
        if constexpr (std::is_same<V, dfloat2>::value) {
            return false;
        } else {
            if (st.lines)
                run_mix<V, true>(st.a);
            else
                run_mix<V, false>(st.a);
            return true;
        }
    }
    switch (st.M) {
        case 2: return pass_m<V, 2>(st);
        case 3: return pass_m<V, 3>(st);
        case 4: return pass_m<V, 4>(st);
        case 5: return pass_m<V, 5>(st);
        case 8: return pass_m<V, 8>(st);
        case 9: return pass_m<V, 9>(st);
        case 16: return pass_m<V, 16>(st);
        case 25: return pass_m<V, 25>(st);
        case 27: return pass_m<V, 27>(st);
        case 32: return pass_m<V, 32>(st);
        case 64: return pass_m<V, 64>(st);
        case 81: return pass_m<V, 81>(st);
        case 125: return pass_m<V, 125>(st);
        case 128: return pass_m<V, 128>(st);
        case 48: return pass_m<V, 48>(st);
        case 120: return pass_m<V, 120>(st);
        case 1000: return pass_m<V, 1000>(st);
        case 2048: return pass_m<V, 2048>(st);
        default: return false;
    }
}

// a plane pass: one CTA of NT host threads walks every plane (plane_kernel's
// loop with a grid of one, K = 1)
template <typename V, int M1, int M2> static bool run_plane(const PlaneArgs& pa) {
    using PS = PlaneShape<V, M1, M2, 1>;
    const int nt = PS::NT;
    std::vector<unsigned char> smem(PS::SMEM + 16);
    V* s = reinterpret_cast<V*>((reinterpret_cast<uintptr_t>(smem.data()) + 15) & ~uintptr_t(15));
    std::barrier<> bar(nt);
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i)
        th.emplace_back([&, i] {
            threadIdx = uint3{(unsigned)i, 0u, 0u};
            blockIdx = uint3{0u, 0u, 0u};
            blockDim = dim3((unsigned)nt);
            gridDim = dim3(1u);
            g_cta_barrier = &bar;
            for (uint32_t p = 0; p < (uint32_t)pa.planes; ++p) {
                plane_run<V, M1, M2, 1>(pa, p, 0u, s);
                __syncthreads();
            }
        });
    for (auto& t : th) t.join();
    return true;
}

template <typename V> static bool dispatch_plane(const HostStep& st);
template <> bool dispatch_plane<float2>(const HostStep& st) {
    if (st.M == 64 && st.lines == 64) return run_plane<float2, 64, 64>(st.pa);
    if (st.M == 128 && st.lines == 128) return run_plane<float2, 128, 128>(st.pa);
    if (st.M == 27 && st.lines == 27) return run_plane<float2, 27, 27>(st.pa);
    if (st.M == 25 && st.lines == 25) return run_plane<float2, 25, 25>(st.pa);
    if (st.M == 128 && st.lines == 2) return run_plane<float2, 128, 2>(st.pa);
    return false;
}
template <> bool dispatch_plane<double2>(const HostStep& st) {
    if (st.M == 64 && st.lines == 64) return run_plane<double2, 64, 64>(st.pa);
    if (st.M == 27 && st.lines == 27) return run_plane<double2, 27, 27>(st.pa);
    if (st.M == 25 && st.lines == 25) return run_plane<double2, 25, 25>(st.pa);
    if (st.M == 128 && st.lines == 2) return run_plane<double2, 128, 2>(st.pa);
    return false;
}

template <typename V, typename T> static void reorder(const HostStep& st, T scale) {
    const V* src = static_cast<const V*>(st.src);
    V* dst = static_cast<V*>(st.dst);
    for (uint32_t e = 0; e < (uint32_t)st.n; ++e) dst[spec_slot(st.o, e)] = cscale(src[e], scale);
}

static void* aligned(size_t bytes) {
    void* p = std::aligned_alloc(256, (bytes + 255) / 256 * 256);
    std::memset(p, 0, (bytes + 255) / 256 * 256);
    return p;
}

int main(int argc, char** argv) {
    if (argc < 10) return 2;
    const int dtype = std::atoi(argv[1]), radix = std::atoi(argv[2]), cap = std::atoi(argv[3]);
    const int flags = std::atoi(argv[4]), ndim = std::atoi(argv[5]);
    if (ndim < 1 || ndim > 3 || argc != 6 + ndim + 3) return 2;
    int64_t dims[3] = {1, 1, 1};
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= (dims[a] = std::atoll(argv[6 + a]));
    const size_t es = dtype == 0 ? 8 : 16;
    void* h = aligned(n * es);
    void* x = aligned(n * es);
    void* y = aligned(n * es);
    void* scratch = aligned(n * es);
    for (int k = 0; k < 2; ++k) {
        FILE* f = std::fopen(argv[6 + ndim + k], "rb");
        if (!f || std::fread(k == 0 ? h : x, es, (size_t)n, f) != (size_t)n) return 3;
        std::fclose(f);
    }
    int64_t tb = 0, se = 0;
    int ns = 0;
    if (pac_test_host_steps(ndim, dims, radix, (pac_dtype)dtype, cap, flags, h, x, y, nullptr, scratch, nullptr, &tb,
                            &se, nullptr, &ns) != 0) {
        std::fprintf(stderr, "%s\n", pac_last_error());
        return 4;
    }
    void* tables = aligned((size_t)tb);
    void* spec = aligned((size_t)se * es);
    std::vector<HostStep> steps(ns);
    if (pac_test_host_steps(ndim, dims, radix, (pac_dtype)dtype, cap, flags, h, x, y, spec, scratch, tables, &tb, &se,
                            steps.data(), &ns) != 0) {
        std::fprintf(stderr, "%s\n", pac_last_error());
        return 4;
    }
    for (const HostStep& st : steps) {
        if (st.kind == 1) {
            if (dtype == 0)
                reorder<float2>(st, (float)st.scale);
            else if (dtype == 1)
                reorder<double2>(st, st.scale);
            else
                reorder<dfloat2>(st, dfloat((float)st.scale, (float)(st.scale - (double)(float)st.scale)));
            continue;
        }
        bool ok;
        if (st.kind == 2)
            ok = dtype == 0 ? dispatch_plane<float2>(st) : dtype == 1 ? dispatch_plane<double2>(st) : false;
        else
            ok = dtype == 0 ? dispatch<float2>(st) : dtype == 1 ? dispatch<double2>(st) : dispatch<dfloat2>(st);
        if (!ok) {
            std::fprintf(stderr, "no emulated kernel for group size %d (%d)\n", st.M, st.lines);
            return 5;
        }
    }
    FILE* f = std::fopen(argv[6 + ndim + 2], "wb");
    if (!f || std::fwrite(y, es, (size_t)n, f) != (size_t)n) return 6;
    std::fclose(f);
    return 0;
}
