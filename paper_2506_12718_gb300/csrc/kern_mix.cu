// Launchers of the runtime-radix kernel for mixed groups (mix.cuh).
#include <atomic>

#include "mix.cuh"
#include "pac_internal.h"

namespace pac {

namespace {

template <typename K> cudaError_t mix_setup(K kernel, std::atomic<int>* ready, int dev, int* per_sm, int smem) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (ready[dev].load(std::memory_order_relaxed) == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMixSmemMax);
        if (e != cudaSuccess) return e;
        ready[dev].store(1, std::memory_order_relaxed);
    }
    if (per_sm) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kMixThreads, smem);
        if (e != cudaSuccess) return e;
        *per_sm = nb > 0 ? nb : 1;
    }
    return cudaSuccess;
}

template <typename V, bool LINES> cudaError_t launch_mix_variant(const PassArgs& a, cudaStream_t s) {
    static std::atomic<int> ready[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = mix_setup(mix_kernel<V, LINES>, ready, dev, nullptr, 0);
    if (e != cudaSuccess) return e;
    if (a.tiles <= 0) return cudaSuccess;
    if (a.tiles > 0x7fffffffLL || a.mix_nr < 1 || a.mix_nr > kMixMaxRounds) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.tiles);
    cfg.blockDim = dim3(kMixThreads);
    cfg.dynamicSmemBytes = mix_smem_bytes(a.mix_m, (int)sizeof(V));
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mix_kernel<V, LINES>, a);
}

template <typename V, bool LINES>
cudaError_t launch_mix_multi_variant(int M, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                                     cudaStream_t s) {
    static std::atomic<int> ready[64];
    int dev = 0, per_sm = 1;
    const int smem = mix_smem_bytes(M, (int)sizeof(V));
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = mix_setup(mix_multi_kernel<V, LINES>, ready, dev, &per_sm, smem);
    if (e != cudaSuccess) return e;
    if (total <= 0 || n <= 0) return cudaSuccess;
    if (total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)per_sm * device_sm_count(dev);
    const int64_t grid = total < cap ? total : cap;
    mix_multi_kernel<V, LINES><<<(unsigned)grid, kMixThreads, smem, s>>>(list, starts, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mix(int esize, bool lines, const PassArgs& a, cudaStream_t s) {
    if (esize == 8) return lines ? launch_mix_variant<float2, true>(a, s) : launch_mix_variant<float2, false>(a, s);
    return lines ? launch_mix_variant<double2, true>(a, s) : launch_mix_variant<double2, false>(a, s);
}

cudaError_t launch_mix_multi(int esize, int M, bool lines, const PassArgs* list, const uint32_t* starts, int n,
                             int64_t total, cudaStream_t s) {
    if (esize == 8)
        return lines ? launch_mix_multi_variant<float2, true>(M, list, starts, n, total, s)
                     : launch_mix_multi_variant<float2, false>(M, list, starts, n, total, s);
    return lines ? launch_mix_multi_variant<double2, true>(M, list, starts, n, total, s)
                 : launch_mix_multi_variant<double2, false>(M, list, starts, n, total, s);
}

}  // namespace pac
