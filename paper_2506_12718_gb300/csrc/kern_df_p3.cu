// Pass-kernel instantiations of the double-float element type (df.cuh): group sizes that are powers of 3.
#include "kern_launch.cuh"

namespace pac {

namespace {
template <int M> cudaError_t launch_df_M(const PassArgs& a, cudaStream_t s) {
    return a.C == 1 ? launch_variant<dfloat2, M, true>(a, s) : launch_variant<dfloat2, M, false>(a, s);
}
}  // namespace

cudaError_t launch_pass_df_p3(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 3: return launch_df_M<3>(a, s);
        case 9: return launch_df_M<9>(a, s);
        case 27: return launch_df_M<27>(a, s);
        case 81: return launch_df_M<81>(a, s);
        case 243: return launch_df_M<243>(a, s);
        case 729: return launch_df_M<729>(a, s);
        case 2187: return launch_df_M<2187>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
