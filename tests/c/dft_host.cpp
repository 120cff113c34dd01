// Host build of the kernels' in-register DFTs (csrc/fft_device.cuh: dft<R, INV, V>
// with its factored twiddles and stage-2 butterflies) for the CPU tests: the
// device intrinsics and built-in variables the header names get host
// definitions (IEEE single / double precision, round to nearest, no
// contraction), and only the DFT templates are instantiated.  Reads lines
// "type R inv v0.re v0.im ... v(R-1).im" (type 0: complex FP32, 1: complex
// FP64, 2: double-float; values as hex doubles) and prints the R outputs.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

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
static uint3 threadIdx, blockIdx;
static dim3 blockDim, gridDim;
static inline void __syncthreads() {}
static inline void __threadfence() {}
static inline unsigned atomicAdd(unsigned* p, unsigned v) { const unsigned o = *p; *p += v; return o; }
static inline unsigned atomicExch(unsigned* p, unsigned v) { const unsigned o = *p; *p = v; return o; }
static inline long long clock64() { return 0; }
static inline void __nanosleep(unsigned) {}
#define __launch_bounds__(...)

#include "fft_device.cuh"

using namespace pac;

template <typename V> V from(double re, double im);
template <> float2 from<float2>(double re, double im) { return float2{(float)re, (float)im}; }
template <> double2 from<double2>(double re, double im) { return double2{re, im}; }
template <> dfloat2 from<dfloat2>(double re, double im) { return dfloat2{df_from_double(re), df_from_double(im)}; }
static void out(float2 v) { std::printf(" %a %a", (double)v.x, (double)v.y); }
static void out(double2 v) { std::printf(" %a %a", v.x, v.y); }
static void out(dfloat2 v) { std::printf(" %a %a", df_to_double(v.x), df_to_double(v.y)); }

template <typename V, int R> static void run(int inv, const double* in) {
    V v[R];
    for (int k = 0; k < R; ++k) v[k] = from<V>(in[2 * k], in[2 * k + 1]);
    if (inv)
        dft<R, true>(v);
    else
        dft<R, false>(v);
    for (int k = 0; k < R; ++k) out(v[k]);
    std::printf("\n");
}

template <typename V> static bool dispatch(int R, int inv, const double* in) {
    switch (R) {
        case 2: run<V, 2>(inv, in); return true;
        case 3: run<V, 3>(inv, in); return true;
        case 4: run<V, 4>(inv, in); return true;
        case 5: run<V, 5>(inv, in); return true;
        case 8: run<V, 8>(inv, in); return true;
        case 9: run<V, 9>(inv, in); return true;
        case 16: run<V, 16>(inv, in); return true;
        case 25: run<V, 25>(inv, in); return true;
        case 27: run<V, 27>(inv, in); return true;
        case 32: run<V, 32>(inv, in); return true;
        default: return false;
    }
}

int main() {
    int type, R, inv;
    while (std::scanf("%d %d %d", &type, &R, &inv) == 3) {
        double in[64];
        if (R < 1 || R > 32) return 2;
        for (int k = 0; k < 2 * R; ++k)
            if (std::scanf("%la", &in[k]) != 1) return 2;
        const bool ok = type == 0 ? dispatch<float2>(R, inv, in)
                        : type == 1 ? dispatch<double2>(R, inv, in)
                                    : dispatch<dfloat2>(R, inv, in);
        if (!ok) return 3;
    }
    return 0;
}
