// Host build of the double-float arithmetic (csrc/df.cuh) for the CPU tests:
// the device intrinsics it calls are given host definitions with the same
// rounding (IEEE single precision, round to nearest; no contraction), so the
// header's own code runs on the CPU.  Reads lines "op a b" (hex doubles / the
// two FP32 parts as hex) on stdin and prints the results as hex.
//   split d         -> hi lo             (df_from_double)
//   widen d         -> hi lo D           (df_to_double of the split: D as FP64)
//   add ahi alo bhi blo -> hi lo         (operator+)
//   mul ahi alo bhi blo -> hi lo         (operator*)
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

#include "df.cuh"

using namespace pac;

int main() {
    char op[16];
    while (std::scanf("%15s", op) == 1) {
        if (!std::strcmp(op, "split") || !std::strcmp(op, "widen")) {
            double d;
            if (std::scanf("%la", &d) != 1) return 2;
            const dfloat r = df_from_double(d);
            if (op[0] == 's')
                std::printf("%a %a\n", (double)r.hi, (double)r.lo);
            else
                std::printf("%a %a %a\n", (double)r.hi, (double)r.lo, df_to_double(r));
        } else {
            double a0, a1, b0, b1;
            if (std::scanf("%la %la %la %la", &a0, &a1, &b0, &b1) != 4) return 2;
            const dfloat a((float)a0, (float)a1), b((float)b0, (float)b1);
            const dfloat r = op[0] == 'a' ? a + b : a * b;
            std::printf("%a %a\n", (double)r.hi, (double)r.lo);
        }
    }
    return 0;
}
