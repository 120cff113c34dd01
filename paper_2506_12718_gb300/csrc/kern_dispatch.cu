// Dispatch of a pass (a whole single-launch convolution, or a batch of
// passes of one shape) to its instantiation by element type and group size.
#include "pac_internal.h"

namespace pac {

cudaError_t launch_pass_c64_p2(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c64_p35(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c128_p2(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c128_p35(int M, const PassArgs& a, cudaStream_t s);
int conv_grid_c64_p2(int M, int dev);
int conv_grid_c64_p35(int M, int dev);
int conv_grid_c128_p2(int M, int dev);
int conv_grid_c128_p35(int M, int dev);
cudaError_t launch_conv_c64_p2(int M, ConvArgs& args, int grid, cudaStream_t s);
cudaError_t launch_conv_c64_p35(int M, ConvArgs& args, int grid, cudaStream_t s);
cudaError_t launch_conv_c128_p2(int M, ConvArgs& args, int grid, cudaStream_t s);
cudaError_t launch_conv_c128_p35(int M, ConvArgs& args, int grid, cudaStream_t s);

cudaError_t launch_mix(int esize, bool lines, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_mixc(int esize, int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_multi_mixc(int esize, int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts,
                              int n, int64_t total, cudaStream_t s);
cudaError_t launch_mix_multi(int esize, int M, bool lines, const PassArgs* list, const uint32_t* starts, int n,
                             int64_t total, cudaStream_t s);

cudaError_t launch_pass_df_p2(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_df_p3(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_df_p5(int M, const PassArgs& a, cudaStream_t s);

cudaError_t launch_pass(int esize, int M, const PassArgs& a, cudaStream_t s) {
    if (a.df & kDfKernel) {  // double-float plans: one-base groups only
        if (a.mix_nr > 0 || is_mixed(M)) return cudaErrorInvalidValue;
        return (M % 2 == 0) ? launch_pass_df_p2(M, a, s)
                            : (M % 3 == 0 ? launch_pass_df_p3(M, a, s) : launch_pass_df_p5(M, a, s));
    }
    if (a.mix_nr > 0) return launch_mix(esize, a.C == 1, a, s);
    if (is_mixed(M)) return launch_pass_mixc(esize, M, a, s);
    if (esize == 8) return (M % 2 == 0) ? launch_pass_c64_p2(M, a, s) : launch_pass_c64_p35(M, a, s);
    return (M % 2 == 0) ? launch_pass_c128_p2(M, a, s) : launch_pass_c128_p35(M, a, s);
}

int conv_grid(int esize, int M, int dev) {
    if (is_mixed(M)) return 0;  // no single-launch form of the mixed groups
    if (esize == 8) return (M % 2 == 0) ? conv_grid_c64_p2(M, dev) : conv_grid_c64_p35(M, dev);
    return (M % 2 == 0) ? conv_grid_c128_p2(M, dev) : conv_grid_c128_p35(M, dev);
}

cudaError_t launch_conv(int esize, int M, ConvArgs& args, int grid, cudaStream_t s) {
    if (is_mixed(M)) return cudaErrorInvalidValue;
    if (esize == 8) return (M % 2 == 0) ? launch_conv_c64_p2(M, args, grid, s) : launch_conv_c64_p35(M, args, grid, s);
    return (M % 2 == 0) ? launch_conv_c128_p2(M, args, grid, s) : launch_conv_c128_p35(M, args, grid, s);
}

cudaError_t launch_multi_c64_p2(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                               cudaStream_t s);
cudaError_t launch_multi_c64_p35(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                                cudaStream_t s);
cudaError_t launch_multi_c128_p2(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n, int64_t total,
                                cudaStream_t s);
cudaError_t launch_multi_c128_p35(int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                                 int64_t total, cudaStream_t s);

cudaError_t launch_multi(int esize, int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                         int64_t total, cudaStream_t s) {
    if (M < 0) return launch_mix_multi(esize, -M, lines, list, starts, n, total, s);  // mixed groups of size -M
    if (is_mixed(M)) return launch_multi_mixc(esize, M, lines, nv, list, starts, n, total, s);
    if (esize == 8)
        return (M % 2 == 0) ? launch_multi_c64_p2(M, lines, nv, list, starts, n, total, s)
                            : launch_multi_c64_p35(M, lines, nv, list, starts, n, total, s);
    return (M % 2 == 0) ? launch_multi_c128_p2(M, lines, nv, list, starts, n, total, s)
                        : launch_multi_c128_p35(M, lines, nv, list, starts, n, total, s);
}

int pass_kernel_supported(int M, int esize) {
    if (is_mixed(M)) return mixed_compiled(M) ? 1 : 0;
    int b = base_of(M);
    if (b == 1 || M < 2) return 0;
    int m = M;
    while (m % b == 0) m /= b;
    if (m != 1) return 0;
    return M <= group_mmax(b, esize) ? 1 : 0;
}

}  // namespace pac
