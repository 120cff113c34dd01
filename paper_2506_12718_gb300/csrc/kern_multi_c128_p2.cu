// Batched pass-kernel instantiations: double2, group sizes that are powers of 2.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_multi_c128_p2(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                                 int64_t total, cudaStream_t s) {
    switch (M) {
        case 2: return launch_multi_M<double2, 2>(lines, nv, list, starts, n, total, s);
        case 4: return launch_multi_M<double2, 4>(lines, nv, list, starts, n, total, s);
        case 8: return launch_multi_M<double2, 8>(lines, nv, list, starts, n, total, s);
        case 16: return launch_multi_M<double2, 16>(lines, nv, list, starts, n, total, s);
        case 32: return launch_multi_M<double2, 32>(lines, nv, list, starts, n, total, s);
        case 64: return launch_multi_M<double2, 64>(lines, nv, list, starts, n, total, s);
        case 128: return launch_multi_M<double2, 128>(lines, nv, list, starts, n, total, s);
        case 256: return launch_multi_M<double2, 256>(lines, nv, list, starts, n, total, s);
        case 512: return launch_multi_M<double2, 512>(lines, nv, list, starts, n, total, s);
        case 1024: return launch_multi_M<double2, 1024>(lines, nv, list, starts, n, total, s);
        case 2048: return launch_multi_M<double2, 2048>(lines, nv, list, starts, n, total, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
