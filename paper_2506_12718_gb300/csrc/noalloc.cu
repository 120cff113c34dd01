// pac_convolve_permuted_noalloc: the permuted (comparator) convolution for
// callers that cannot allocate device memory.
//
// Who needs it: a process whose device memory is owned by another allocator
// (a framework that reserves nearly all of the GPU up front for its own
// caching pool), a service running under a hard device-memory quota that
// forbids growth after start-up, or a latency-critical path that cannot
// afford cudaMalloc's implicit synchronisation and unpredictable cost.  The
// ordinary pac_convolve_permuted obtains its N-element intermediate buffer
// (and its index tables and natural-order spectrum) with cudaMalloc on first
// use; this variant allocates nothing.
//
// Its only scratch is the file-scope array g_noalloc_scratch below, a fixed
// PAC_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU which loads this library
// keeps until the process exits.  The index-reversal positions are computed
// from the plan's stage lists inside the kernel instead of read from tables,
// and the natural-order spectrum is gathered from the stored one on the fly
// (through its storage order, spec_slot, and the plan's placement table).  Every scratch element is written before it is read, so the
// array needs no clearing between calls; it keeps the last call's contents.
// All calls share the one array: two calls whose kernels overlap on the GPU
// (on different streams, or on different threads without ordering) race on it.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address once with cudaGetSymbolAddress (host code must not
// use the array's name as an address).  Make that first call before any
// stream capture begins.
#include <mutex>

#include "fft_device.cuh"
#include "pac_internal.h"

using namespace pac;

#define PAC_NOALLOC_SCRATCH_BYTES (8u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxStages = 32;

// Stage lists of the (up to 3, padded to 3 with length-1) axes.
struct DigitPlan {
    int64_t dims[3];
    int nst[3];
    int st[3][kMaxStages];
};

// Position (in the index-reversed order) of frequency k along one axis:
// k = k_1 + s_1 k_2 + ... lands at p = sum_i k_i prod_{j>i} s_j.
__device__ __forceinline__ int64_t pos_of_freq(const int* st, int T, int64_t k) {
    int64_t pos = 0;
    for (int i = 0; i < T; ++i) {
        pos = pos * st[i] + k % st[i];
        k /= st[i];
    }
    return pos;
}

// Frequency held at position p along one axis (inverse of pos_of_freq).
__device__ __forceinline__ int64_t freq_of_pos(const int* st, int T, int64_t p) {
    int64_t f = 0;
    for (int i = T - 1; i >= 0; --i) {
        f = f * st[i] + p % st[i];
        p /= st[i];
    }
    return f;
}

// out[i] = in[src(i)] (* mul[src(i)]), i a row-major multi-index; src maps
// each axis index through pos_of_freq (to_natural) or freq_of_pos.
template <typename V>
__global__ void permute_digits_kernel(const DigitPlan dp, bool to_natural, const V* in, V* out, const V* mul,
                                      const SpecOrder so) {
    const int64_t n = dp.dims[0] * dp.dims[1] * dp.dims[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i, src = 0, stride = 1;
        for (int a = 2; a >= 0; --a) {
            const int64_t k = rem % dp.dims[a];
            rem /= dp.dims[a];
            const int64_t m = to_natural ? pos_of_freq(dp.st[a], dp.nst[a], k) : freq_of_pos(dp.st[a], dp.nst[a], k);
            src += m * stride;
            stride *= dp.dims[a];
        }
        V v = in[src];
        if (mul) v = cmul(v, __ldg(mul + spec_slot(so, (uint32_t)src)));  // the stored spectrum's slot
        out[i] = v;
    }
}

std::mutex g_mu;
void* g_ptr[64];
bool g_ready[64];

// Device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process.  A device reset destroys
// the primary context and reloads the module at another address, so the
// cached address (like every plan's device memory) is stale after one: the
// library is not used across a device reset.
int scratch_address(int device, void** out) {
    if (device < 0 || device >= 64) return fail(PAC_ERR_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_ptr[device] = p;
        g_ready[device] = true;
    }
    *out = g_ptr[device];
    return PAC_OK;
}

template <typename V>
cudaError_t launch_digits(const DigitPlan& dp, bool to_natural, const void* in, void* out, const void* mul,
                          const SpecOrder& so, int64_t n, cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 4096);
    permute_digits_kernel<V><<<(unsigned)blocks, threads, 0, s>>>(dp, to_natural, static_cast<const V*>(in),
                                                                   static_cast<V*>(out), static_cast<const V*>(mul), so);
    return cudaGetLastError();
}

}  // namespace

extern "C" int pac_convolve_permuted_noalloc(pac_plan p, const void* x_dev, void* y_dev, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (!x_dev || !y_dev) return fail(PAC_ERR_ARG, "null array");
    if (reinterpret_cast<uintptr_t>(x_dev) % 16 || reinterpret_cast<uintptr_t>(y_dev) % 16)
        return fail(PAC_ERR_ARG, "arrays must be 16-byte aligned");
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_filter_spectrum was not called for this plan");
    if (int rc = df_unsupported(p, "pac_convolve_permuted_noalloc")) return rc;
    const uint64_t need = (uint64_t)p->N * (uint64_t)p->esize;
    if (need > PAC_NOALLOC_SCRATCH_BYTES)
        return fail(PAC_ERR_SIZE,
                    "pac_convolve_permuted_noalloc: the array needs %llu bytes of scratch, more than the fixed "
                    "%u-byte static buffer (at most %u complex64 or %u complex128 elements)",
                    (unsigned long long)need, PAC_NOALLOC_SCRATCH_BYTES, PAC_NOALLOC_SCRATCH_BYTES / 8,
                    PAC_NOALLOC_SCRATCH_BYTES / 16);
    for (int a = 0; a < p->ndim; ++a)
        if ((int)p->stages[a].size() > kMaxStages) return fail(PAC_ERR_SIZE, "too many stages on axis %d", a);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(PAC_ERR_ARG, "the plan belongs to device %d, current device is %d", p->device, dev);
    void* scratch = nullptr;
    if (int rc = scratch_address(dev, &scratch)) return rc;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int G = (int)p->groups.size();
    if (G == 0) {  // N = 1: a plain product
        e = launch_pointwise_mul(p->esize, p->N, x_dev, p->d_spec, y_dev, 1.0, s);
        return e == cudaSuccess ? PAC_OK : cuda_fail(e, "pointwise kernel");
    }
    DigitPlan dp;
    for (int a = 0; a < 3; ++a) {
        dp.dims[a] = 1;
        dp.nst[a] = 0;
    }
    for (int a = 0; a < p->ndim; ++a) {
        const int b = 3 - p->ndim + a;
        dp.dims[b] = p->dims[a];
        dp.nst[b] = (int)p->stages[a].size();
        for (int i = 0; i < dp.nst[b]; ++i) dp.st[b][i] = p->stages[a][i];
    }
    // FFT2 = permute o uFFT2 (Algorithm 5): DIF passes one launch per group
    for (int i = 0; i < G; ++i) {
        int rc = run_pass(p, p->groups[i], kFwd, i == 0 ? x_dev : y_dev, y_dev, s);
        if (rc) return rc;
    }
    // natural order with the product (spectrum gathered at the same positions), into the static scratch
    const SpecOrder so = spec_order_of(p);
    e = p->esize == 8 ? launch_digits<float2>(dp, true, y_dev, scratch, p->d_spec, so, p->N, s)
                      : launch_digits<double2>(dp, true, y_dev, scratch, p->d_spec, so, p->N, s);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    // back to the index-reversed order for the inverse (iFFT = uiFFT o permute, Algorithm 9)
    e = p->esize == 8 ? launch_digits<float2>(dp, false, scratch, y_dev, nullptr, so, p->N, s)
                      : launch_digits<double2>(dp, false, scratch, y_dev, nullptr, so, p->N, s);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    for (int i = G - 1; i >= 0; --i) {
        int rc = run_pass(p, p->groups[i], kInv, y_dev, y_dev, s);
        if (rc) return rc;
    }
    return PAC_OK;
}
