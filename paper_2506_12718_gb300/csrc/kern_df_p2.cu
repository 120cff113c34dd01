// Pass-kernel instantiations of the double-float element type (df.cuh): group sizes that are powers of 2.
#include "kern_launch.cuh"

namespace pac {

namespace {
template <int M> cudaError_t launch_df_M(const PassArgs& a, cudaStream_t s) {
    return a.C == 1 ? launch_variant<dfloat2, M, true>(a, s) : launch_variant<dfloat2, M, false>(a, s);
}
}  // namespace

cudaError_t launch_pass_df_p2(int M, const PassArgs& a, cudaStream_t s) {
    switch (M) {
        case 2: return launch_df_M<2>(a, s);
        case 4: return launch_df_M<4>(a, s);
        case 8: return launch_df_M<8>(a, s);
        case 16: return launch_df_M<16>(a, s);
        case 32: return launch_df_M<32>(a, s);
        case 64: return launch_df_M<64>(a, s);
        case 128: return launch_df_M<128>(a, s);
        case 256: return launch_df_M<256>(a, s);
        case 512: return launch_df_M<512>(a, s);
        case 1024: return launch_df_M<1024>(a, s);
        case 2048: return launch_df_M<2048>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pac
