// Auxiliary kernels: the index-reversal permutation of the comparator
// (Algorithm 1, a gather through per-axis index tables, optionally fused with
// the Hadamard product), the one-time reordering of a filter spectrum into
// its storage order, and a pointwise product for the degenerate N = 1 plan.
#include <algorithm>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

// out[i0,i1,i2] = in[t0[i0], t1[i1], t2[i2]] (* mul[i0,i1,i2]); a null table is the identity
template <typename V>
__global__ void permute_kernel(int64_t d0, int64_t d1, int64_t d2, const int64_t* __restrict__ t0,
                               const int64_t* __restrict__ t1, const int64_t* __restrict__ t2, const V* src,
                               V* dst, const V* __restrict__ mul) {
    const int64_t rows = d0 * d1;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int64_t i0 = row / d1, i1 = row - (row / d1) * d1;
        const int64_t s0 = t0 ? __ldg(t0 + i0) : i0;
        const int64_t s1 = t1 ? __ldg(t1 + i1) : i1;
        const V* srow = src + (s0 * d1 + s1) * d2;
        V* drow = dst + row * d2;
        for (int64_t i2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i2 < d2;
             i2 += (int64_t)gridDim.x * blockDim.x) {
            V v = srow[t2 ? __ldg(t2 + i2) : i2];
            if (mul) v = cmul(v, __ldg(mul + row * d2 + i2));
            drow[i2] = v;
        }
    }
}

template <typename V>
__global__ void pointwise_kernel(int64_t n, const V* a, const V* __restrict__ b, V* out, double scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        V v = a[i];
        if (b) v = cmul(v, __ldg(b + i));
        if (scale != 1.0) v = cscale(v, (typename Real<V>::T)scale);
        out[i] = v;
    }
}

// Between the plain index-reversed order of a spectrum and its storage order
// (see SpecOrder): to_kernel ? dst[slot(e)] = src[e] : dst[e] = src[slot(e)].
template <typename V>
__global__ void spec_order_kernel(const SpecOrder o, uint32_t n, const V* __restrict__ src, V* __restrict__ dst,
                                  int to_kernel) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t k = spec_slot(o, e);
        if (to_kernel)
            dst[k] = src[e];
        else
            dst[e] = src[k];
    }
}

cudaError_t launch_spec_order(int esize, const SpecOrder& o, int64_t n, const void* src, void* dst, bool to_kernel,
                              cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 8192);
    if (esize == 8)
        spec_order_kernel<float2><<<(unsigned)blocks, threads, 0, s>>>(o, (uint32_t)n, (const float2*)src,
                                                                      (float2*)dst, to_kernel ? 1 : 0);
    else
        spec_order_kernel<double2><<<(unsigned)blocks, threads, 0, s>>>(o, (uint32_t)n, (const double2*)src,
                                                                       (double2*)dst, to_kernel ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_permute(int esize, int ndim, const int64_t* dims, const int64_t* const* idx_dev,
                           const void* src, void* dst, const void* mul, cudaStream_t s) {
    int64_t d[3] = {1, 1, 1};
    const int64_t* t[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < ndim; ++a) {
        d[3 - ndim + a] = dims[a];
        t[3 - ndim + a] = idx_dev[a];
    }
    const int64_t rows = d[0] * d[1];
    const int threads = (int)std::min<int64_t>(256, ((d[2] + 31) / 32) * 32);
    const int64_t gx = std::min<int64_t>((d[2] + threads - 1) / threads, 4096);
    const int64_t gy = std::min<int64_t>(rows, 65535);
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (esize == 8)
        permute_kernel<float2><<<grid, threads, 0, s>>>(d[0], d[1], d[2], t[0], t[1], t[2], (const float2*)src,
                                                         (float2*)dst, (const float2*)mul);
    else
        permute_kernel<double2><<<grid, threads, 0, s>>>(d[0], d[1], d[2], t[0], t[1], t[2], (const double2*)src,
                                                          (double2*)dst, (const double2*)mul);
    return cudaGetLastError();
}

cudaError_t launch_pointwise_mul(int esize, int64_t n, const void* a, const void* b, void* out, double scale,
                                 cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 65535);
    if (esize == 8)
        pointwise_kernel<float2><<<(unsigned)blocks, threads, 0, s>>>(n, (const float2*)a, (const float2*)b,
                                                                     (float2*)out, scale);
    else
        pointwise_kernel<double2><<<(unsigned)blocks, threads, 0, s>>>(n, (const double2*)a, (const double2*)b,
                                                                      (double2*)out, scale);
    return cudaGetLastError();
}

}  // namespace pac
