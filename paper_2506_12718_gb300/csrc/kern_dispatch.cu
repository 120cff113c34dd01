// Dispatch of a pass to its instantiation by element type and group size.
#include "pac_internal.h"

namespace pac {

cudaError_t launch_pass_c64_p2(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c64_p35(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c128_p2(int M, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_c128_p35(int M, const PassArgs& a, cudaStream_t s);

cudaError_t launch_pass_c64(int M, const PassArgs& a, cudaStream_t s) {
    return (M % 2 == 0) ? launch_pass_c64_p2(M, a, s) : launch_pass_c64_p35(M, a, s);
}

cudaError_t launch_pass_c128(int M, const PassArgs& a, cudaStream_t s) {
    return (M % 2 == 0) ? launch_pass_c128_p2(M, a, s) : launch_pass_c128_p35(M, a, s);
}

int pass_kernel_supported(int M, int esize) {
    int b = base_of(M);
    if (b == 1 || M < 2) return 0;
    int m = M;
    while (m % b == 0) m /= b;
    if (m != 1) return 0;
    return M <= group_mmax(b, esize) ? 1 : 0;
}

}  // namespace pac
