// Pass-kernel and convolution-kernel instantiations: double2, group sizes that are powers of 3 or 5.
#include "kern_launch.cuh"

namespace pac {

cudaError_t launch_pass_c128_p35(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 3: return launch_M<double2, 3>(a, s);
        case 9: return launch_M<double2, 9>(a, s);
        case 27: return launch_M<double2, 27>(a, s);
        case 81: return launch_M<double2, 81>(a, s);
        case 243: return launch_M<double2, 243>(a, s);
        case 729: return launch_M<double2, 729>(a, s);
        case 2187: return launch_M<double2, 2187>(a, s);
        case 5: return launch_M<double2, 5>(a, s);
        case 25: return launch_M<double2, 25>(a, s);
        case 125: return launch_M<double2, 125>(a, s);
        case 625: return launch_M<double2, 625>(a, s);
        case 3125: return launch_M<double2, 3125>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

int conv_grid_c128_p35(int M, int dev) {
    switch (M) {
        case 3: return conv_grid<double2, 3>(dev);
        case 9: return conv_grid<double2, 9>(dev);
        case 27: return conv_grid<double2, 27>(dev);
        case 81: return conv_grid<double2, 81>(dev);
        case 243: return conv_grid<double2, 243>(dev);
        case 729: return conv_grid<double2, 729>(dev);
        case 2187: return conv_grid<double2, 2187>(dev);
        case 5: return conv_grid<double2, 5>(dev);
        case 25: return conv_grid<double2, 25>(dev);
        case 125: return conv_grid<double2, 125>(dev);
        case 625: return conv_grid<double2, 625>(dev);
        case 3125: return conv_grid<double2, 3125>(dev);
        default: return 0;
    }
}

cudaError_t launch_conv_c128_p35(int M, ConvArgs& args, int grid, cudaStream_t s) {
    switch (M) {
        case 3: return launch_conv_M<double2, 3>(args, grid, s);
        case 9: return launch_conv_M<double2, 9>(args, grid, s);
        case 27: return launch_conv_M<double2, 27>(args, grid, s);
        case 81: return launch_conv_M<double2, 81>(args, grid, s);
        case 243: return launch_conv_M<double2, 243>(args, grid, s);
        case 729: return launch_conv_M<double2, 729>(args, grid, s);
        case 2187: return launch_conv_M<double2, 2187>(args, grid, s);
        case 5: return launch_conv_M<double2, 5>(args, grid, s);
        case 25: return launch_conv_M<double2, 25>(args, grid, s);
        case 125: return launch_conv_M<double2, 125>(args, grid, s);
        case 625: return launch_conv_M<double2, 625>(args, grid, s);
        case 3125: return launch_conv_M<double2, 3125>(args, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
