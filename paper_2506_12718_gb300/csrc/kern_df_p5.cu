// Pass-kernel instantiations of the double-float element type (df.cuh): group sizes that are powers of 5.
#include "kern_launch.cuh"

namespace pac {

namespace {
template <int M> cudaError_t launch_df_M(const PassArgs& a, cudaStream_t s) {
    return a.C == 1 ? launch_variant<dfloat2, M, true>(a, s) : launch_variant<dfloat2, M, false>(a, s);
}
}  // namespace

cudaError_t launch_pass_df_p5(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 5: return launch_df_M<5>(a, s);
        case 25: return launch_df_M<25>(a, s);
        case 125: return launch_df_M<125>(a, s);
        case 625: return launch_df_M<625>(a, s);
        case 3125: return launch_df_M<3125>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
