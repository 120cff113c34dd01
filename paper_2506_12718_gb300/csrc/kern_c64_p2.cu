// Pass-kernel instantiations: float2, group sizes that are powers of 2.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_pass_c64_p2(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 2: return launch_M<float2, 2>(a, s);
        case 4: return launch_M<float2, 4>(a, s);
        case 8: return launch_M<float2, 8>(a, s);
        case 16: return launch_M<float2, 16>(a, s);
        case 32: return launch_M<float2, 32>(a, s);
        case 64: return launch_M<float2, 64>(a, s);
        case 128: return launch_M<float2, 128>(a, s);
        case 256: return launch_M<float2, 256>(a, s);
        case 512: return launch_M<float2, 512>(a, s);
        case 1024: return launch_M<float2, 1024>(a, s);
        case 2048: return launch_M<float2, 2048>(a, s);
        case 4096: return launch_M<float2, 4096>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
