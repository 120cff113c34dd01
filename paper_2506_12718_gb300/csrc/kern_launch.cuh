// Launch helper for the pass kernels: one instantiation per (element type,
// group size M).  Grid = one CTA per tile for single passes; the batched and
// single-launch forms use resident CTAs walking the tiles.
#pragma once
#include <atomic>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

template <typename V, int M, bool LINES, int NV = 0>
cudaError_t launch_variant(const PassArgs& a, cudaStream_t s) {
    using SH = Shape<V, M, LINES, NV>;
    constexpr int smem = pass_smem_bytes<V, M, NV>(LINES);
    static std::atomic<int> resident[64];  // per device: CTAs per SM; 0 = not set up
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = resident[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        e = cudaFuncSetAttribute(pass_kernel<V, M, LINES, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_kernel<V, M, LINES, NV>, SH::NT, smem);
        if (e != cudaSuccess) return e;
        per_sm = nb > 0 ? nb : 1;
        resident[dev].store(per_sm, std::memory_order_relaxed);
    }
    if (a.tiles <= 0) return cudaSuccess;
    if (a.tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    // one CTA per tile: the hardware fills the SMs wave after wave, and CTAs
    // end every few microseconds, so kernels of other streams (higher
    // priority requests of a serving queue) get SMs between them
    const int64_t grid = a.tiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SH::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pass_kernel<V, M, LINES, NV>, a);
}

// Batched form: n passes of this shape, their arguments and tile starts in
// device memory; grid = resident CTAs, capped by the total tile count.
template <typename V, int M, bool LINES, int NV = 0>
cudaError_t launch_multi_variant(const PassArgs* list, const uint32_t* starts, int n, int64_t total_tiles,
                                 cudaStream_t s) {
    using SH = Shape<V, M, LINES, NV>;
    constexpr int smem = pass_smem_bytes<V, M, NV>(LINES);
    static std::atomic<int> resident[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = resident[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        e = cudaFuncSetAttribute(pass_multi_kernel<V, M, LINES, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_multi_kernel<V, M, LINES, NV>, SH::NT, smem);
        if (e != cudaSuccess) return e;
        per_sm = nb > 0 ? nb : 1;
        resident[dev].store(per_sm, std::memory_order_relaxed);
    }
    if (total_tiles <= 0 || n <= 0) return cudaSuccess;
    if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)per_sm * device_sm_count(dev);
    const int64_t grid = total_tiles < cap ? total_tiles : cap;
    pass_multi_kernel<V, M, LINES, NV><<<(unsigned)grid, SH::NT, smem, s>>>(list, starts, n);
    return cudaGetLastError();
}

// nv = 1: the narrow tile variant where the group has one (has_narrow), else the default tile
template <typename V, int M>
cudaError_t launch_multi_M(bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                           cudaStream_t s) {
    if constexpr (has_narrow(M, sizeof(V))) {
        if (nv)
            return lines ? launch_multi_variant<V, M, true, 1>(list, starts, n, total, s)
                         : launch_multi_variant<V, M, false, 1>(list, starts, n, total, s);
    }
    return lines ? launch_multi_variant<V, M, true>(list, starts, n, total, s)
                 : launch_multi_variant<V, M, false>(list, starts, n, total, s);
}

template <typename V, int M>
cudaError_t launch_M(const PassArgs& a, cudaStream_t s) {
    if constexpr (has_narrow(M, sizeof(V))) {
        if (a.nv) return a.C == 1 ? launch_variant<V, M, true, 1>(a, s) : launch_variant<V, M, false, 1>(a, s);
    }
    return a.C == 1 ? launch_variant<V, M, true>(a, s) : launch_variant<V, M, false>(a, s);
}

// Co-resident grid size of the cooperative convolution kernel (0 on error).
template <typename V, int M>
int conv_grid(int dev) {
    using SH = Shape<V, M>;
    constexpr int smem = pass_smem_bytes<V, M>(true) > pass_smem_bytes<V, M>(false) ? pass_smem_bytes<V, M>(true)
                                                                                      : pass_smem_bytes<V, M>(false);
    static std::atomic<int> resident[64];
    if (dev < 0 || dev >= 64) return 0;
    int per_sm = resident[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if (cudaFuncSetAttribute(conv_kernel<V, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, conv_kernel<V, M>, SH::NT, smem) != cudaSuccess || nb < 1)
            return 0;
        per_sm = nb;
        resident[dev].store(per_sm, std::memory_order_relaxed);
    }
    return per_sm * device_sm_count(dev);
}

template <typename V, int M>
cudaError_t launch_conv_M(ConvArgs& args, int grid, cudaStream_t s) {
    using SH = Shape<V, M>;
    constexpr int smem = pass_smem_bytes<V, M>(true) > pass_smem_bytes<V, M>(false) ? pass_smem_bytes<V, M>(true)
                                                                                      : pass_smem_bytes<V, M>(false);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SH::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, conv_kernel<V, M>, args);
}

}  // namespace pac
