// Instantiations and launchers of the TMA-fed lines kernel (lines_tma.cuh):
// complex FP32 lines groups of 1024, 2048, 4096, 2187 and 3125 points.
#include <atomic>

#include "lines_tma.cuh"
#include "pac_internal.h"

namespace pac {

namespace {

template <typename V, int M>
cudaError_t launch_tma_M(const LinesTmaArgs& ta, bool pdl, cudaStream_t s) {
    using TS = TmaShape<V, M>;
    static std::atomic<int> resident[64][2];  // per device and spectrum staging: CTAs per SM
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int st = ta.stage_spec ? 1 : 0;
    const int smem = tma_smem_bytes(M, (int)sizeof(V), st != 0);
    int per_sm = resident[dev][st].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        e = cudaFuncSetAttribute(lines_tma_kernel<V, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tma_smem_bytes(M, (int)sizeof(V), true));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lines_tma_kernel<V, M>, TS::NT, smem);
        if (e != cudaSuccess) return e;
        per_sm = nb > 0 ? nb : 1;
        resident[dev][st].store(per_sm, std::memory_order_relaxed);
    }
    if (ta.total == 0) return cudaSuccess;
    const int64_t cap = (int64_t)per_sm * device_sm_count(dev);
    const int64_t grid = (int64_t)ta.total < cap ? (int64_t)ta.total : cap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TS::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, lines_tma_kernel<V, M>, ta);
}

cudaError_t launch_tma(int esize, int M, const LinesTmaArgs& ta, bool pdl, cudaStream_t s) {
    if (esize != 8) return cudaErrorInvalidValue;
    switch (M) {
        case 1024: return launch_tma_M<float2, 1024>(ta, pdl, s);
        case 2048: return launch_tma_M<float2, 2048>(ta, pdl, s);
        case 4096: return launch_tma_M<float2, 4096>(ta, pdl, s);
        case 2187: return launch_tma_M<float2, 2187>(ta, pdl, s);
        case 3125: return launch_tma_M<float2, 3125>(ta, pdl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int tma_lines_supported(int M, int esize) {
    if (esize != 8 || !tma_group(M, esize)) return 0;
    switch (M) {
        case 1024: case 2048: case 4096: case 2187: case 3125: return 1;
        default: return 0;
    }
}

cudaError_t launch_lines_tma(int esize, int M, const PassArgs& a, cudaStream_t s) {
    LinesTmaArgs ta = {};
    ta.one = a;
    ta.list = nullptr;
    ta.starts = nullptr;
    ta.n = 1;
    if (a.tiles < 0 || a.tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    ta.total = (uint32_t)a.tiles;
    ta.stage_spec = a.mode == kFused ? 1 : 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (device_error_word(dev, &ta.error) != PAC_OK) return cudaErrorMemoryAllocation;
    return launch_tma(esize, M, ta, true, s);
}

cudaError_t launch_lines_tma_multi(int esize, int M, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                                   int stage_spec, cudaStream_t s) {
    LinesTmaArgs ta = {};
    ta.list = list;
    ta.starts = starts;
    ta.n = n;
    if (total < 0 || total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    ta.total = n > 0 ? (uint32_t)total : 0u;
    ta.stage_spec = stage_spec;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (device_error_word(dev, &ta.error) != PAC_OK) return cudaErrorMemoryAllocation;
    return launch_tma(esize, M, ta, false, s);
}

}  // namespace pac
