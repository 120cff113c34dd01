// Batched pass-kernel instantiations: double2, group sizes that are powers of 3 or 5.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_multi_c128_p35(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                                 int64_t total, cudaStream_t s) {
    switch (M) {
        case 3: return launch_multi_M<double2, 3>(lines, nv, list, starts, n, total, s);
        case 9: return launch_multi_M<double2, 9>(lines, nv, list, starts, n, total, s);
        case 27: return launch_multi_M<double2, 27>(lines, nv, list, starts, n, total, s);
        case 81: return launch_multi_M<double2, 81>(lines, nv, list, starts, n, total, s);
        case 243: return launch_multi_M<double2, 243>(lines, nv, list, starts, n, total, s);
        case 729: return launch_multi_M<double2, 729>(lines, nv, list, starts, n, total, s);
        case 2187: return launch_multi_M<double2, 2187>(lines, nv, list, starts, n, total, s);
        case 5: return launch_multi_M<double2, 5>(lines, nv, list, starts, n, total, s);
        case 25: return launch_multi_M<double2, 25>(lines, nv, list, starts, n, total, s);
        case 125: return launch_multi_M<double2, 125>(lines, nv, list, starts, n, total, s);
        case 625: return launch_multi_M<double2, 625>(lines, nv, list, starts, n, total, s);
        case 3125: return launch_multi_M<double2, 3125>(lines, nv, list, starts, n, total, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
