// Auxiliary kernels: the index-reversal permutation of the comparator
// (Algorithm 1, a gather through per-axis index tables, optionally fused with
// the Hadamard product; one block per row, or one thread per element for
// short rows), the one-time reordering of a filter spectrum into
// its storage order, and a pointwise product for the degenerate N = 1 plan.
#include <algorithm>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

// out[i0,i1,i2] = in[t0[i0], t1[i1], t2[i2]] (* mul[i0,i1,i2]) (* scale); a null table is the identity.
// 32-bit index arithmetic (a plan keeps N < 2^31): a 64-bit division would
// run on the FP64 pipe, which is narrow on this GPU.
template <typename V>
__global__ void permute_kernel(uint32_t d0, uint32_t d1, uint32_t d2, const int64_t* __restrict__ t0,
                               const int64_t* __restrict__ t1, const int64_t* __restrict__ t2, const V* src,
                               V* dst, const V* __restrict__ mul, typename Real<V>::T scale, int do_scale) {
    const uint32_t rows = d0 * d1;
    for (uint32_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const uint32_t i0 = row / d1, i1 = row - i0 * d1;
        const uint32_t s0 = t0 ? (uint32_t)__ldg(t0 + i0) : i0;
        const uint32_t s1 = t1 ? (uint32_t)__ldg(t1 + i1) : i1;
        const V* srow = src + (size_t)(s0 * d1 + s1) * d2;
        V* drow = dst + (size_t)row * d2;
        const V* mrow = mul ? mul + (size_t)row * d2 : nullptr;
        for (uint32_t i2 = blockIdx.x * blockDim.x + threadIdx.x; i2 < d2; i2 += gridDim.x * blockDim.x) {
            V v = srow[t2 ? (uint32_t)__ldg(t2 + i2) : i2];
            if (mrow) v = cmul(v, __ldg(mrow + i2));
            if (do_scale) v = cscale(v, scale);
            drow[i2] = v;
        }
    }
}

// The same gather for short rows (d2 small: one block per row would leave
// most of its threads idle): one thread per output element, grid-stride,
// 32-bit indices (a plan keeps N < 2^31).
template <typename V>
__global__ void permute_flat_kernel(uint32_t n, uint32_t d1, uint32_t d2, const int64_t* __restrict__ t0,
                                    const int64_t* __restrict__ t1, const int64_t* __restrict__ t2, const V* src,
                                    V* dst, const V* __restrict__ mul, typename Real<V>::T scale, int do_scale) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t row = e / d2, i2 = e - row * d2;
        const uint32_t i0 = row / d1, i1 = row - i0 * d1;
        const uint32_t s0 = t0 ? (uint32_t)__ldg(t0 + i0) : i0;
        const uint32_t s1 = t1 ? (uint32_t)__ldg(t1 + i1) : i1;
        const uint32_t s2 = t2 ? (uint32_t)__ldg(t2 + i2) : i2;
        V v = src[(s0 * d1 + s1) * d2 + s2];
        if (mul) v = cmul(v, __ldg(mul + e));
        if (do_scale) v = cscale(v, scale);
        dst[e] = v;
    }
}

template <typename V>
__global__ void pointwise_kernel(int64_t n, const V* a, const V* __restrict__ b, V* out, typename Real<V>::T scale,
                                 int do_scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        V v = a[i];
        if (b) v = cmul(v, __ldg(b + i));
        if (do_scale) v = cscale(v, scale);
        out[i] = v;
    }
}

// Between the plain index-reversed order of a spectrum and its storage order
// (see SpecOrder): to_kernel ? dst[slot(e)] = src[e] : dst[e] = src[slot(e)],
// times `scale` (the filter spectrum's 1/N, applied here once).
template <typename V>
__global__ void spec_order_kernel(const SpecOrder o, uint32_t n, const V* __restrict__ src, V* __restrict__ dst,
                                  int to_kernel, typename Real<V>::T scale) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t k = spec_slot(o, e);
        if (to_kernel)
            dst[k] = cscale(src[e], scale);
        else
            dst[e] = cscale(src[k], scale);
    }
}

cudaError_t launch_spec_order_df(const SpecOrder& o, int64_t n, const void* src, void* dst, cudaStream_t s,
                                 double scale) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 8192);
    const float hi = (float)scale;
    const dfloat sc(hi, (float)(scale - (double)hi));
    spec_order_kernel<dfloat2><<<(unsigned)blocks, threads, 0, s>>>(o, (uint32_t)n, (const dfloat2*)src, (dfloat2*)dst,
                                                                    1, sc);
    return cudaGetLastError();
}

cudaError_t launch_spec_order(int esize, const SpecOrder& o, int64_t n, const void* src, void* dst, bool to_kernel,
                              cudaStream_t s, double scale) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 8192);
    if (esize == 8)
        spec_order_kernel<float2><<<(unsigned)blocks, threads, 0, s>>>(o, (uint32_t)n, (const float2*)src,
                                                                      (float2*)dst, to_kernel ? 1 : 0, (float)scale);
    else
        spec_order_kernel<double2><<<(unsigned)blocks, threads, 0, s>>>(o, (uint32_t)n, (const double2*)src,
                                                                       (double2*)dst, to_kernel ? 1 : 0, scale);
    return cudaGetLastError();
}

cudaError_t launch_permute(int esize, int ndim, const int64_t* dims, const int64_t* const* idx_dev,
                           const void* src, void* dst, const void* mul, cudaStream_t s, double scale) {
    int64_t d[3] = {1, 1, 1};
    const int64_t* t[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < ndim; ++a) {
        d[3 - ndim + a] = dims[a];
        t[3 - ndim + a] = idx_dev[a];
    }
    const int64_t rows = d[0] * d[1];
    if (d[2] < 64) {  // short rows: one thread per element
        int dev = 0;
        cudaGetDevice(&dev);
        const int64_t n = rows * d[2];
        const unsigned blocks =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count(dev) * 16));
        if (esize == 8)
            permute_flat_kernel<float2><<<blocks, 256, 0, s>>>((uint32_t)n, (uint32_t)d[1], (uint32_t)d[2], t[0], t[1],
                                                               t[2], (const float2*)src, (float2*)dst,
                                                               (const float2*)mul, (float)scale, scale != 1.0);
        else
            permute_flat_kernel<double2><<<blocks, 256, 0, s>>>((uint32_t)n, (uint32_t)d[1], (uint32_t)d[2], t[0],
                                                                t[1], t[2], (const double2*)src, (double2*)dst,
                                                                (const double2*)mul, scale, scale != 1.0);
        return cudaGetLastError();
    }
    const int threads = (int)std::min<int64_t>(256, ((d[2] + 31) / 32) * 32);
    const int64_t gx = std::min<int64_t>((d[2] + threads - 1) / threads, 4096);
    const int64_t gy = std::min<int64_t>(rows, 65535);
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (esize == 8)
        permute_kernel<float2><<<grid, threads, 0, s>>>((uint32_t)d[0], (uint32_t)d[1], (uint32_t)d[2], t[0], t[1],
                                                         t[2], (const float2*)src, (float2*)dst, (const float2*)mul,
                                                         (float)scale, scale != 1.0);
    else
        permute_kernel<double2><<<grid, threads, 0, s>>>((uint32_t)d[0], (uint32_t)d[1], (uint32_t)d[2], t[0], t[1],
                                                          t[2], (const double2*)src, (double2*)dst,
                                                          (const double2*)mul, scale, scale != 1.0);
    return cudaGetLastError();
}

cudaError_t launch_pointwise_mul(int esize, int64_t n, const void* a, const void* b, void* out, double scale,
                                 cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 65535);
    if (esize == 8)
        pointwise_kernel<float2><<<(unsigned)blocks, threads, 0, s>>>(n, (const float2*)a, (const float2*)b,
                                                                     (float2*)out, (float)scale, scale != 1.0);
    else
        pointwise_kernel<double2><<<(unsigned)blocks, threads, 0, s>>>(n, (const double2*)a, (const double2*)b,
                                                                      (double2*)out, scale, scale != 1.0);
    return cudaGetLastError();
}

}  // namespace pac

// ---------------------------------------------------------------- FMA probe
//
// Peak fused multiply-add throughput of the device for one precision: every
// thread runs 8 independent chains of dependent FMAs, enough warps per SM to
// cover the pipe latency.  Used as the ALU roofline of FP64 passes, which
// on this GPU are bound by the FP64 pipe rather than by HBM.
namespace pac {

template <typename T>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // never true in practice; keeps the chains live
}

}  // namespace pac

extern "C" int pac_measure_fma_peak(int dtype, double* gflops) {
    using namespace pac;
    if (!gflops || (dtype != PAC_C64 && dtype != PAC_C128)) return fail(PAC_ERR_ARG, "bad arguments");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const int blocks = device_sm_count(dev) * 8, threads = 256, iters = 4096;
    void* out = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * 16);
    if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "probe buffer: %s", cudaGetErrorString(e));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a, 0);
        if (dtype == PAC_C64)
            fma_probe_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.999f, 0.001f);
        else
            fma_probe_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999, 0.001);
        cudaEventRecord(b, 0);
        e = cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;  // the first run warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "FMA probe");
    *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
    return PAC_OK;
}
