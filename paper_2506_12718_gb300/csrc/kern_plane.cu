// Plane-pass instantiations (the last two axes of whole planes in one CTA)
// and their launchers.
#include <atomic>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

namespace {

template <typename V, int M1, int M2, bool MULTI>
cudaError_t prepare(int dev) {
    static std::atomic<int> ready[64];
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (ready[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    constexpr int smem = PlaneShape<V, M1, M2>::SMEM;
    cudaError_t e = MULTI ? cudaFuncSetAttribute(plane_multi_kernel<V, M1, M2>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                          : cudaFuncSetAttribute(plane_kernel<V, M1, M2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem);
    if (e == cudaSuccess) ready[dev].store(1, std::memory_order_relaxed);
    return e;
}

template <typename V, int M1, int M2>
cudaError_t launch_one(const PlaneArgs& pa, cudaStream_t s) {
    using PS = PlaneShape<V, M1, M2>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = prepare<V, M1, M2, false>(dev);
    if (e != cudaSuccess) return e;
    if (pa.planes <= 0) return cudaSuccess;
    const int64_t cap = device_sm_count(dev);  // one CTA per SM (the plane fills most of its shared memory)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(pa.planes < cap ? pa.planes : cap));
    cfg.blockDim = dim3(PS::NT);
    cfg.dynamicSmemBytes = PS::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, plane_kernel<V, M1, M2>, pa);
}

template <typename V, int M1, int M2>
cudaError_t launch_many(const PlaneArgs* list, const uint32_t* starts, int n, int64_t total, cudaStream_t s) {
    using PS = PlaneShape<V, M1, M2>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = prepare<V, M1, M2, true>(dev);
    if (e != cudaSuccess) return e;
    if (n <= 0 || total <= 0) return cudaSuccess;
    const int64_t cap = device_sm_count(dev);
    plane_multi_kernel<V, M1, M2><<<(unsigned)(total < cap ? total : cap), PS::NT, PS::SMEM, s>>>(list, starts, n);
    return cudaGetLastError();
}

}  // namespace

int plane_supported(int M1, int M2, int esize) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128) return 1;
        if (M1 == 64 && M2 == 64) return 1;
        if (M1 == 32 && M2 == 32) return 1;
        if (M1 == 16 && M2 == 16) return 1;
        if (M1 == 64 && M2 == 128) return 1;
        if (M1 == 128 && M2 == 64) return 1;
        if (M1 == 81 && M2 == 81) return 1;
        if (M1 == 27 && M2 == 27) return 1;
        if (M1 == 9 && M2 == 9) return 1;
        if (M1 == 25 && M2 == 25) return 1;
        if (M1 == 125 && M2 == 125) return 1;
        return 0;
    }
    if (M1 == 64 && M2 == 64) return 1;
    if (M1 == 32 && M2 == 32) return 1;
    if (M1 == 16 && M2 == 16) return 1;
    if (M1 == 27 && M2 == 27) return 1;
    if (M1 == 81 && M2 == 81) return 1;
    if (M1 == 25 && M2 == 25) return 1;
    if (M1 == 9 && M2 == 9) return 1;
    return 0;
}

cudaError_t launch_plane(int esize, int M1, int M2, const PlaneArgs& pa, cudaStream_t s) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128) return launch_one<float2, 128, 128>(pa, s);
        if (M1 == 64 && M2 == 64) return launch_one<float2, 64, 64>(pa, s);
        if (M1 == 32 && M2 == 32) return launch_one<float2, 32, 32>(pa, s);
        if (M1 == 16 && M2 == 16) return launch_one<float2, 16, 16>(pa, s);
        if (M1 == 64 && M2 == 128) return launch_one<float2, 64, 128>(pa, s);
        if (M1 == 128 && M2 == 64) return launch_one<float2, 128, 64>(pa, s);
        if (M1 == 81 && M2 == 81) return launch_one<float2, 81, 81>(pa, s);
        if (M1 == 27 && M2 == 27) return launch_one<float2, 27, 27>(pa, s);
        if (M1 == 9 && M2 == 9) return launch_one<float2, 9, 9>(pa, s);
        if (M1 == 25 && M2 == 25) return launch_one<float2, 25, 25>(pa, s);
        if (M1 == 125 && M2 == 125) return launch_one<float2, 125, 125>(pa, s);
    } else {
        if (M1 == 64 && M2 == 64) return launch_one<double2, 64, 64>(pa, s);
        if (M1 == 32 && M2 == 32) return launch_one<double2, 32, 32>(pa, s);
        if (M1 == 16 && M2 == 16) return launch_one<double2, 16, 16>(pa, s);
        if (M1 == 27 && M2 == 27) return launch_one<double2, 27, 27>(pa, s);
        if (M1 == 81 && M2 == 81) return launch_one<double2, 81, 81>(pa, s);
        if (M1 == 25 && M2 == 25) return launch_one<double2, 25, 25>(pa, s);
        if (M1 == 9 && M2 == 9) return launch_one<double2, 9, 9>(pa, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_plane_multi(int esize, int M1, int M2, const PlaneArgs* list, const uint32_t* starts, int n,
                               int64_t total, cudaStream_t s) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128) return launch_many<float2, 128, 128>(list, starts, n, total, s);
        if (M1 == 64 && M2 == 64) return launch_many<float2, 64, 64>(list, starts, n, total, s);
        if (M1 == 32 && M2 == 32) return launch_many<float2, 32, 32>(list, starts, n, total, s);
        if (M1 == 16 && M2 == 16) return launch_many<float2, 16, 16>(list, starts, n, total, s);
        if (M1 == 64 && M2 == 128) return launch_many<float2, 64, 128>(list, starts, n, total, s);
        if (M1 == 128 && M2 == 64) return launch_many<float2, 128, 64>(list, starts, n, total, s);
        if (M1 == 81 && M2 == 81) return launch_many<float2, 81, 81>(list, starts, n, total, s);
        if (M1 == 27 && M2 == 27) return launch_many<float2, 27, 27>(list, starts, n, total, s);
        if (M1 == 9 && M2 == 9) return launch_many<float2, 9, 9>(list, starts, n, total, s);
        if (M1 == 25 && M2 == 25) return launch_many<float2, 25, 25>(list, starts, n, total, s);
        if (M1 == 125 && M2 == 125) return launch_many<float2, 125, 125>(list, starts, n, total, s);
    } else {
        if (M1 == 64 && M2 == 64) return launch_many<double2, 64, 64>(list, starts, n, total, s);
        if (M1 == 32 && M2 == 32) return launch_many<double2, 32, 32>(list, starts, n, total, s);
        if (M1 == 16 && M2 == 16) return launch_many<double2, 16, 16>(list, starts, n, total, s);
        if (M1 == 27 && M2 == 27) return launch_many<double2, 27, 27>(list, starts, n, total, s);
        if (M1 == 81 && M2 == 81) return launch_many<double2, 81, 81>(list, starts, n, total, s);
        if (M1 == 25 && M2 == 25) return launch_many<double2, 25, 25>(list, starts, n, total, s);
        if (M1 == 9 && M2 == 9) return launch_many<double2, 9, 9>(list, starts, n, total, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pac
