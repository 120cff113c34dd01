// Pass-kernel instantiations of the compiled mixed groups (groups spanning
// prime bases, mixed_compiled in config.h), single and batched forms, both
// element types.  Their rounds are config.h's mixed round lists.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_pass_mixc(int esize, int M, const PassArgs& a, cudaStream_t s) {
    if (esize == 8) {
        switch (M) {
            case 48: return launch_M<float2, 48>(a, s);
            case 120: return launch_M<float2, 120>(a, s);
            case 1000: return launch_M<float2, 1000>(a, s);
            case 6000: return launch_M<float2, 6000>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (M) {
        case 48: return launch_M<double2, 48>(a, s);
        case 120: return launch_M<double2, 120>(a, s);
        case 1000: return launch_M<double2, 1000>(a, s);
        case 6000: return launch_M<double2, 6000>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_multi_mixc(int esize, int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                              int64_t total, cudaStream_t s) {
    if (esize == 8) {
        switch (M) {
            case 48: return launch_multi_M<float2, 48>(lines, nv, list, starts, n, total, s);
            case 120: return launch_multi_M<float2, 120>(lines, nv, list, starts, n, total, s);
            case 1000: return launch_multi_M<float2, 1000>(lines, nv, list, starts, n, total, s);
            case 6000: return launch_multi_M<float2, 6000>(lines, nv, list, starts, n, total, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (M) {
        case 48: return launch_multi_M<double2, 48>(lines, nv, list, starts, n, total, s);
        case 120: return launch_multi_M<double2, 120>(lines, nv, list, starts, n, total, s);
        case 1000: return launch_multi_M<double2, 1000>(lines, nv, list, starts, n, total, s);
        case 6000: return launch_multi_M<double2, 6000>(lines, nv, list, starts, n, total, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
