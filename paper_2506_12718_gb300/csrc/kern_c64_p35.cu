// Pass-kernel instantiations: float2, group sizes that are powers of 35.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_pass_c64_p35(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 3: return launch_M<float2, 3>(a, s);
        case 9: return launch_M<float2, 9>(a, s);
        case 27: return launch_M<float2, 27>(a, s);
        case 81: return launch_M<float2, 81>(a, s);
        case 243: return launch_M<float2, 243>(a, s);
        case 729: return launch_M<float2, 729>(a, s);
        case 2187: return launch_M<float2, 2187>(a, s);
        case 5: return launch_M<float2, 5>(a, s);
        case 25: return launch_M<float2, 25>(a, s);
        case 125: return launch_M<float2, 125>(a, s);
        case 625: return launch_M<float2, 625>(a, s);
        case 3125: return launch_M<float2, 3125>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
