// Plane-pass instantiations (the last two axes of whole planes, in one CTA
// or split over a K-CTA cluster) and their launchers.
#include <atomic>
#include <cstdlib>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

namespace {

template <typename V, int M1, int M2, int K, bool MULTI>
cudaError_t prepare(int dev) {
    static std::atomic<int> ready[64];
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (ready[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    constexpr int smem = PlaneShape<V, M1, M2, K>::SMEM;
    cudaError_t e = MULTI ? cudaFuncSetAttribute(plane_multi_kernel<V, M1, M2, K>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                          : cudaFuncSetAttribute(plane_kernel<V, M1, M2, K>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && K > 1)
        e = MULTI ? cudaFuncSetAttribute(plane_multi_kernel<V, M1, M2, K>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 0)
                  : cudaFuncSetAttribute(plane_kernel<V, M1, M2, K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    if (e == cudaSuccess) ready[dev].store(1, std::memory_order_relaxed);
    return e;
}

// clusters to launch: at most the planes, at most two resident rounds of the GPU
int64_t cluster_grid(int dev, int64_t planes, int k) {
    const int64_t cap = 2 * (int64_t)device_sm_count(dev) * (k > 1 ? 2 : 1) / k;
    return planes < cap ? planes : cap;
}

template <typename V, int M1, int M2, int K>
cudaError_t launch_one(const PlaneArgs& pa, cudaStream_t s) {
    using PS = PlaneShape<V, M1, M2, K>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = prepare<V, M1, M2, K, false>(dev);
    if (e != cudaSuccess) return e;
    if (pa.planes <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(K * pa.planes));  // one cluster per plane (CTAs end often; see kern_launch.cuh)
    cfg.blockDim = dim3(PS::NT);
    cfg.dynamicSmemBytes = PS::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = K;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, plane_kernel<V, M1, M2, K>, pa);
}

template <typename V, int M1, int M2, int K>
cudaError_t launch_many(const PlaneArgs* list, const uint32_t* starts, int n, int64_t total, cudaStream_t s) {
    using PS = PlaneShape<V, M1, M2, K>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = prepare<V, M1, M2, K, true>(dev);
    if (e != cudaSuccess) return e;
    if (n <= 0 || total <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(K * cluster_grid(dev, total, K)));
    cfg.blockDim = dim3(PS::NT);
    cfg.dynamicSmemBytes = PS::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, plane_multi_kernel<V, M1, M2, K>, list, starts, n);
}

}  // namespace

// CTAs per plane for a plane shape and plane count (0: no plane kernel).
// Enough planes to give every SM one (planes >= SMs / 2): one CTA per plane
// (a cluster's barriers and remote accesses only cost time then); fewer
// planes: the split form where one exists (measured faster for 81^2 and
// 125^2; a 128^2 FP64 plane exists only split).  PAC_PLANE_K in the
// environment forces a cluster size where that form exists.
int plane_cluster(int M1, int M2, int esize, int64_t planes, int device) {
    const char* f = std::getenv("PAC_PLANE_K");
    const int want = f ? std::atoi(f) : 0;
    if (want > 0 && plane_supported_k(M1, M2, esize, want)) return want;
    if (2 * planes >= device_sm_count(device) && plane_supported_k(M1, M2, esize, 1)) return 1;
    if (esize == 8) {
        if (M1 == 128 && M2 == 128) return 1;
        if (M1 == 64 && M2 == 64) return 1;
        if (M1 == 32 && M2 == 32) return 1;
        if (M1 == 16 && M2 == 16) return 1;
        if (M1 == 64 && M2 == 128) return 1;
        if (M1 == 128 && M2 == 64) return 1;
        if (M1 == 81 && M2 == 81) return 3;
        if (M1 == 27 && M2 == 27) return 1;
        if (M1 == 9 && M2 == 9) return 1;
        if (M1 == 25 && M2 == 25) return 1;
        if (M1 == 125 && M2 == 125) return 5;
        if (M1 == 128 && M2 == 2) return 1;
        if (M1 == 256 && M2 == 2) return 1;
        if (M1 == 512 && M2 == 2) return 1;
        if (M1 == 1024 && M2 == 2) return 1;
        if (M1 == 2048 && M2 == 2) return 1;
        if (M1 == 4096 && M2 == 2) return 1;
        if (M1 == 256 && M2 == 4) return 1;
        if (M1 == 1024 && M2 == 4) return 1;
        return 0;
    }
    if (M1 == 64 && M2 == 64) return 1;
    if (M1 == 32 && M2 == 32) return 1;
    if (M1 == 16 && M2 == 16) return 1;
    if (M1 == 27 && M2 == 27) return 1;
    if (M1 == 81 && M2 == 81) return 1;
    if (M1 == 25 && M2 == 25) return 1;
    if (M1 == 9 && M2 == 9) return 1;
    if (M1 == 128 && M2 == 128) return 2;
    if (M1 == 128 && M2 == 2) return 1;
    if (M1 == 256 && M2 == 2) return 1;
    if (M1 == 512 && M2 == 2) return 1;
    if (M1 == 1024 && M2 == 2) return 1;
    if (M1 == 2048 && M2 == 2) return 1;
    return 0;
}

int plane_supported_k(int M1, int M2, int esize, int K) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128 && K == 1) return 1;
        if (M1 == 64 && M2 == 64 && K == 1) return 1;
        if (M1 == 32 && M2 == 32 && K == 1) return 1;
        if (M1 == 16 && M2 == 16 && K == 1) return 1;
        if (M1 == 64 && M2 == 128 && K == 1) return 1;
        if (M1 == 128 && M2 == 64 && K == 1) return 1;
        if (M1 == 81 && M2 == 81 && K == 1) return 1;
        if (M1 == 81 && M2 == 81 && K == 3) return 1;
        if (M1 == 27 && M2 == 27 && K == 1) return 1;
        if (M1 == 9 && M2 == 9 && K == 1) return 1;
        if (M1 == 25 && M2 == 25 && K == 1) return 1;
        if (M1 == 125 && M2 == 125 && K == 1) return 1;
        if (M1 == 125 && M2 == 125 && K == 5) return 1;
        if (M1 == 128 && M2 == 2 && K == 1) return 1;
        if (M1 == 256 && M2 == 2 && K == 1) return 1;
        if (M1 == 512 && M2 == 2 && K == 1) return 1;
        if (M1 == 1024 && M2 == 2 && K == 1) return 1;
        if (M1 == 2048 && M2 == 2 && K == 1) return 1;
        if (M1 == 4096 && M2 == 2 && K == 1) return 1;
        if (M1 == 256 && M2 == 4 && K == 1) return 1;
        if (M1 == 1024 && M2 == 4 && K == 1) return 1;
        return 0;
    }
    if (M1 == 64 && M2 == 64 && K == 1) return 1;
    if (M1 == 32 && M2 == 32 && K == 1) return 1;
    if (M1 == 16 && M2 == 16 && K == 1) return 1;
    if (M1 == 27 && M2 == 27 && K == 1) return 1;
    if (M1 == 81 && M2 == 81 && K == 1) return 1;
    if (M1 == 25 && M2 == 25 && K == 1) return 1;
    if (M1 == 9 && M2 == 9 && K == 1) return 1;
    if (M1 == 128 && M2 == 128 && K == 2) return 1;
    if (M1 == 128 && M2 == 2 && K == 1) return 1;
    if (M1 == 256 && M2 == 2 && K == 1) return 1;
    if (M1 == 512 && M2 == 2 && K == 1) return 1;
    if (M1 == 1024 && M2 == 2 && K == 1) return 1;
    if (M1 == 2048 && M2 == 2 && K == 1) return 1;
    return 0;
}

int plane_supported(int M1, int M2, int esize) { return plane_cluster(M1, M2, esize, 0, 0) > 0; }

cudaError_t launch_plane(int esize, int M1, int M2, int K, const PlaneArgs& pa, cudaStream_t s) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128 && K == 1) return launch_one<float2, 128, 128, 1>(pa, s);
        if (M1 == 64 && M2 == 64 && K == 1) return launch_one<float2, 64, 64, 1>(pa, s);
        if (M1 == 32 && M2 == 32 && K == 1) return launch_one<float2, 32, 32, 1>(pa, s);
        if (M1 == 16 && M2 == 16 && K == 1) return launch_one<float2, 16, 16, 1>(pa, s);
        if (M1 == 64 && M2 == 128 && K == 1) return launch_one<float2, 64, 128, 1>(pa, s);
        if (M1 == 128 && M2 == 64 && K == 1) return launch_one<float2, 128, 64, 1>(pa, s);
        if (M1 == 81 && M2 == 81 && K == 1) return launch_one<float2, 81, 81, 1>(pa, s);
        if (M1 == 81 && M2 == 81 && K == 3) return launch_one<float2, 81, 81, 3>(pa, s);
        if (M1 == 27 && M2 == 27 && K == 1) return launch_one<float2, 27, 27, 1>(pa, s);
        if (M1 == 9 && M2 == 9 && K == 1) return launch_one<float2, 9, 9, 1>(pa, s);
        if (M1 == 25 && M2 == 25 && K == 1) return launch_one<float2, 25, 25, 1>(pa, s);
        if (M1 == 125 && M2 == 125 && K == 1) return launch_one<float2, 125, 125, 1>(pa, s);
        if (M1 == 125 && M2 == 125 && K == 5) return launch_one<float2, 125, 125, 5>(pa, s);
        if (M1 == 128 && M2 == 2 && K == 1) return launch_one<float2, 128, 2, 1>(pa, s);
        if (M1 == 256 && M2 == 2 && K == 1) return launch_one<float2, 256, 2, 1>(pa, s);
        if (M1 == 512 && M2 == 2 && K == 1) return launch_one<float2, 512, 2, 1>(pa, s);
        if (M1 == 1024 && M2 == 2 && K == 1) return launch_one<float2, 1024, 2, 1>(pa, s);
        if (M1 == 2048 && M2 == 2 && K == 1) return launch_one<float2, 2048, 2, 1>(pa, s);
        if (M1 == 4096 && M2 == 2 && K == 1) return launch_one<float2, 4096, 2, 1>(pa, s);
        if (M1 == 256 && M2 == 4 && K == 1) return launch_one<float2, 256, 4, 1>(pa, s);
        if (M1 == 1024 && M2 == 4 && K == 1) return launch_one<float2, 1024, 4, 1>(pa, s);
    } else {
        if (M1 == 64 && M2 == 64 && K == 1) return launch_one<double2, 64, 64, 1>(pa, s);
        if (M1 == 32 && M2 == 32 && K == 1) return launch_one<double2, 32, 32, 1>(pa, s);
        if (M1 == 16 && M2 == 16 && K == 1) return launch_one<double2, 16, 16, 1>(pa, s);
        if (M1 == 27 && M2 == 27 && K == 1) return launch_one<double2, 27, 27, 1>(pa, s);
        if (M1 == 81 && M2 == 81 && K == 1) return launch_one<double2, 81, 81, 1>(pa, s);
        if (M1 == 25 && M2 == 25 && K == 1) return launch_one<double2, 25, 25, 1>(pa, s);
        if (M1 == 9 && M2 == 9 && K == 1) return launch_one<double2, 9, 9, 1>(pa, s);
        if (M1 == 128 && M2 == 128 && K == 2) return launch_one<double2, 128, 128, 2>(pa, s);
        if (M1 == 128 && M2 == 2 && K == 1) return launch_one<double2, 128, 2, 1>(pa, s);
        if (M1 == 256 && M2 == 2 && K == 1) return launch_one<double2, 256, 2, 1>(pa, s);
        if (M1 == 512 && M2 == 2 && K == 1) return launch_one<double2, 512, 2, 1>(pa, s);
        if (M1 == 1024 && M2 == 2 && K == 1) return launch_one<double2, 1024, 2, 1>(pa, s);
        if (M1 == 2048 && M2 == 2 && K == 1) return launch_one<double2, 2048, 2, 1>(pa, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_plane_multi(int esize, int M1, int M2, int K, const PlaneArgs* list, const uint32_t* starts, int n,
                               int64_t total, cudaStream_t s) {
    if (esize == 8) {
        if (M1 == 128 && M2 == 128 && K == 1) return launch_many<float2, 128, 128, 1>(list, starts, n, total, s);
        if (M1 == 64 && M2 == 64 && K == 1) return launch_many<float2, 64, 64, 1>(list, starts, n, total, s);
        if (M1 == 32 && M2 == 32 && K == 1) return launch_many<float2, 32, 32, 1>(list, starts, n, total, s);
        if (M1 == 16 && M2 == 16 && K == 1) return launch_many<float2, 16, 16, 1>(list, starts, n, total, s);
        if (M1 == 64 && M2 == 128 && K == 1) return launch_many<float2, 64, 128, 1>(list, starts, n, total, s);
        if (M1 == 128 && M2 == 64 && K == 1) return launch_many<float2, 128, 64, 1>(list, starts, n, total, s);
        if (M1 == 81 && M2 == 81 && K == 1) return launch_many<float2, 81, 81, 1>(list, starts, n, total, s);
        if (M1 == 81 && M2 == 81 && K == 3) return launch_many<float2, 81, 81, 3>(list, starts, n, total, s);
        if (M1 == 27 && M2 == 27 && K == 1) return launch_many<float2, 27, 27, 1>(list, starts, n, total, s);
        if (M1 == 9 && M2 == 9 && K == 1) return launch_many<float2, 9, 9, 1>(list, starts, n, total, s);
        if (M1 == 25 && M2 == 25 && K == 1) return launch_many<float2, 25, 25, 1>(list, starts, n, total, s);
        if (M1 == 125 && M2 == 125 && K == 1) return launch_many<float2, 125, 125, 1>(list, starts, n, total, s);
        if (M1 == 125 && M2 == 125 && K == 5) return launch_many<float2, 125, 125, 5>(list, starts, n, total, s);
        if (M1 == 128 && M2 == 2 && K == 1) return launch_many<float2, 128, 2, 1>(list, starts, n, total, s);
        if (M1 == 256 && M2 == 2 && K == 1) return launch_many<float2, 256, 2, 1>(list, starts, n, total, s);
        if (M1 == 512 && M2 == 2 && K == 1) return launch_many<float2, 512, 2, 1>(list, starts, n, total, s);
        if (M1 == 1024 && M2 == 2 && K == 1) return launch_many<float2, 1024, 2, 1>(list, starts, n, total, s);
        if (M1 == 2048 && M2 == 2 && K == 1) return launch_many<float2, 2048, 2, 1>(list, starts, n, total, s);
        if (M1 == 4096 && M2 == 2 && K == 1) return launch_many<float2, 4096, 2, 1>(list, starts, n, total, s);
        if (M1 == 256 && M2 == 4 && K == 1) return launch_many<float2, 256, 4, 1>(list, starts, n, total, s);
        if (M1 == 1024 && M2 == 4 && K == 1) return launch_many<float2, 1024, 4, 1>(list, starts, n, total, s);
    } else {
        if (M1 == 64 && M2 == 64 && K == 1) return launch_many<double2, 64, 64, 1>(list, starts, n, total, s);
        if (M1 == 32 && M2 == 32 && K == 1) return launch_many<double2, 32, 32, 1>(list, starts, n, total, s);
        if (M1 == 16 && M2 == 16 && K == 1) return launch_many<double2, 16, 16, 1>(list, starts, n, total, s);
        if (M1 == 27 && M2 == 27 && K == 1) return launch_many<double2, 27, 27, 1>(list, starts, n, total, s);
        if (M1 == 81 && M2 == 81 && K == 1) return launch_many<double2, 81, 81, 1>(list, starts, n, total, s);
        if (M1 == 25 && M2 == 25 && K == 1) return launch_many<double2, 25, 25, 1>(list, starts, n, total, s);
        if (M1 == 9 && M2 == 9 && K == 1) return launch_many<double2, 9, 9, 1>(list, starts, n, total, s);
        if (M1 == 128 && M2 == 128 && K == 2) return launch_many<double2, 128, 128, 2>(list, starts, n, total, s);
        if (M1 == 128 && M2 == 2 && K == 1) return launch_many<double2, 128, 2, 1>(list, starts, n, total, s);
        if (M1 == 256 && M2 == 2 && K == 1) return launch_many<double2, 256, 2, 1>(list, starts, n, total, s);
        if (M1 == 512 && M2 == 2 && K == 1) return launch_many<double2, 512, 2, 1>(list, starts, n, total, s);
        if (M1 == 1024 && M2 == 2 && K == 1) return launch_many<double2, 1024, 2, 1>(list, starts, n, total, s);
        if (M1 == 2048 && M2 == 2 && K == 1) return launch_many<double2, 2048, 2, 1>(list, starts, n, total, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pac
