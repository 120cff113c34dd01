// Launch helper for the pass kernels: one instantiation per (element type,
// group size M).  Grid = resident CTAs of the whole GPU (persistent loop over
// tiles), capped by the tile count.
#pragma once
#include <atomic>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

template <typename V, int M>
cudaError_t launch_M(const PassArgs& a, cudaStream_t s) {
    constexpr int smem = tile_smem_bytes(M, sizeof(V));
    static std::atomic<int> resident[64];  // CTAs per SM, per device; 0 = not set up
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = resident[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        e = cudaFuncSetAttribute(pass_kernel<V, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_kernel<V, M>, kThreads, smem);
        if (e != cudaSuccess) return e;
        per_sm = nb > 0 ? nb : 1;
        resident[dev].store(per_sm, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)per_sm * device_sm_count(dev);
    const int64_t grid = a.tiles < cap ? a.tiles : cap;
    if (grid <= 0) return cudaSuccess;
    pass_kernel<V, M><<<(unsigned)grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pac
