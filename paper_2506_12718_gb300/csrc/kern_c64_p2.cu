// Pass-kernel and convolution-kernel instantiations: float2, group sizes that are powers of 2.
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

int conv_grid_c64_p2(int M, int dev) {
    switch (M) {
        case 2: return conv_grid<float2, 2>(dev);
        case 4: return conv_grid<float2, 4>(dev);
        case 8: return conv_grid<float2, 8>(dev);
        case 16: return conv_grid<float2, 16>(dev);
        case 32: return conv_grid<float2, 32>(dev);
        case 64: return conv_grid<float2, 64>(dev);
        case 128: return conv_grid<float2, 128>(dev);
        case 256: return conv_grid<float2, 256>(dev);
        case 512: return conv_grid<float2, 512>(dev);
        case 1024: return conv_grid<float2, 1024>(dev);
        case 2048: return conv_grid<float2, 2048>(dev);
        case 4096: return conv_grid<float2, 4096>(dev);
        default: return 0;
    }
}

cudaError_t launch_conv_c64_p2(int M, ConvArgs& args, int grid, cudaStream_t s) {
    switch (M) {
        case 2: return launch_conv_M<float2, 2>(args, grid, s);
        case 4: return launch_conv_M<float2, 4>(args, grid, s);
        case 8: return launch_conv_M<float2, 8>(args, grid, s);
        case 16: return launch_conv_M<float2, 16>(args, grid, s);
        case 32: return launch_conv_M<float2, 32>(args, grid, s);
        case 64: return launch_conv_M<float2, 64>(args, grid, s);
        case 128: return launch_conv_M<float2, 128>(args, grid, s);
        case 256: return launch_conv_M<float2, 256>(args, grid, s);
        case 512: return launch_conv_M<float2, 512>(args, grid, s);
        case 1024: return launch_conv_M<float2, 1024>(args, grid, s);
        case 2048: return launch_conv_M<float2, 2048>(args, grid, s);
        case 4096: return launch_conv_M<float2, 4096>(args, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
