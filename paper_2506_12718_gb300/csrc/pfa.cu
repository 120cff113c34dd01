// Prime factor convolution (Section 7.2).
//
// A 1-D length n = n_1 ... n_t with pairwise coprime factors (the prime
// powers 2^a, 3^b, 5^c of n, ascending) is convolved as a t-D
// permutation-avoiding convolution of shape (n_t, ..., n_1) between two
// index maps.  Gamma^T gathers a length-n vector into the tensor: entry
// (i_t, ..., i_1) is element i with i = i_q mod n_q for every q (Chinese
// remainders, i = sum_q i_q e_q mod n with e_q = 1 mod n_q and 0 mod the
// other factors).  Gamma gathers it back: output k is tensor entry
// (k mod n_t, ..., k mod n_1).  The map is additive, so a cyclic convolution
// of length n is the t-D cyclic convolution of the gathered arrays.  Three
// permutations in all: Gamma^T h once per filter, Gamma^T x and Gamma y per
// call (against six with ordered transforms).  The t-D convolution is an
// ordinary plan (one prime base per axis, no twiddles between factors).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "fft_device.cuh"
#include "pac_internal.h"

struct pac_pfa_s {
    int64_t n = 1;
    int t = 0;                       // number of factors
    int64_t dims[3] = {1, 1, 1};     // tensor shape (n_t, ..., n_1), the last index fastest
    int64_t crt[3] = {0, 0, 0};      // e_q per tensor axis
    pac_dtype dtype = PAC_C64;
    int esize = 8;
    pac_plan inner = nullptr;        // the t-D convolution
    void* d_scratch = nullptr;       // the gathered tensor, n elements
    bool has_spec = false;
    std::mutex mu;
};

namespace pac {

// Gamma^T: tensor entry t = (i_0, i_1, i_2) (i_2 fastest) = src[k], k = (i_0 e_0 + i_1 e_1 + i_2 e_2) mod n.
// A thread walks t, t + S, t + 2S, ... (S the grid's thread count) and keeps
// the digits of t and k up to date with 32-bit additions: adding the digits
// (s_0, s_1, s_2) of S adds delta = (s_0 e_0 + s_1 e_1 + s_2 e_2) mod n to k,
// and a carry out of digit q adds e_{q-1}, because d_q e_q = 0 mod n (e_q is
// 0 modulo every other factor and d_q e_q is 0 modulo d_q).  No 64-bit
// division per element (a 64-bit modulo runs on the FP64 pipe, which is
// narrow on this GPU).
template <typename V>
__global__ void pfa_to_tensor_kernel(uint32_t n, uint32_t d1, uint32_t d2, uint32_t e0, uint32_t e1, uint32_t e2,
                                     uint32_t s0, uint32_t s1, uint32_t s2, uint32_t delta,
                                     const V* __restrict__ src, V* __restrict__ dst) {
    const uint32_t S = gridDim.x * blockDim.x;
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t i2 = t % d2, r = t / d2, i1 = r % d1, i0 = r / d1;
    uint32_t k = (uint32_t)(((uint64_t)i0 * e0 + (uint64_t)i1 * e1 + (uint64_t)i2 * e2) % n);
    const auto addmod = [n](uint32_t a, uint32_t b) { const uint32_t c = a + b; return c >= n ? c - n : c; };
    for (;;) {
        dst[t] = __ldg(src + k);
        t += S;
        if (t >= n) break;
        i2 += s2;
        const bool c2 = i2 >= d2;
        if (c2) i2 -= d2;
        i1 += s1 + (c2 ? 1u : 0u);
        const bool c1 = i1 >= d1;
        if (c1) i1 -= d1;
        i0 += s0 + (c1 ? 1u : 0u);
        k = addmod(k, delta);
        if (c2) k = addmod(k, e1);
        if (c1) k = addmod(k, e0);
    }
}

// Gamma: dst[k] = tensor entry (k mod d_0, k mod d_1, k mod d_2); a thread
// walks k, k + S, ... keeping the three residues with 32-bit additions of
// S mod d_q.
template <typename V>
__global__ void pfa_from_tensor_kernel(uint32_t n, uint32_t d0, uint32_t d1, uint32_t d2, uint32_t m0, uint32_t m1,
                                       uint32_t m2, const V* __restrict__ src, V* __restrict__ dst) {
    const uint32_t S = gridDim.x * blockDim.x;
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t r0 = k % d0, r1 = k % d1, r2 = k % d2;
    for (;;) {
        dst[k] = __ldg(src + (r0 * d1 + r1) * d2 + r2);
        k += S;
        if (k >= n) break;
        r0 += m0;
        if (r0 >= d0) r0 -= d0;
        r1 += m1;
        if (r1 >= d1) r1 -= d1;
        r2 += m2;
        if (r2 >= d2) r2 -= d2;
    }
}

static cudaError_t launch_pfa_map(const pac_pfa_s* p, bool to_tensor, const void* src, void* dst, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int64_t want = (p->n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count(dev) * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const uint64_t n = (uint64_t)p->n;  // < 2^31
    const uint64_t S = (uint64_t)grid * threads;
    const uint64_t d0 = (uint64_t)p->dims[0], d1 = (uint64_t)p->dims[1], d2 = (uint64_t)p->dims[2];
    if (to_tensor) {
        // digits of the stride S (mod n) in the tensor's mixed radix, and the k increment they give
        const uint64_t sm = S % n;
        const uint64_t s2 = sm % d2, s1 = (sm / d2) % d1, s0 = sm / (d1 * d2);
        const uint64_t delta = (s0 * ((uint64_t)p->crt[0] % n) % n + s1 * ((uint64_t)p->crt[1] % n) % n +
                                s2 * ((uint64_t)p->crt[2] % n) % n) % n;
        const uint32_t a[10] = {(uint32_t)n, (uint32_t)d1, (uint32_t)d2, (uint32_t)(p->crt[0] % (int64_t)n),
                                (uint32_t)(p->crt[1] % (int64_t)n), (uint32_t)(p->crt[2] % (int64_t)n),
                                (uint32_t)s0, (uint32_t)s1, (uint32_t)s2, (uint32_t)delta};
        if (p->esize == 8)
            pfa_to_tensor_kernel<float2><<<grid, threads, 0, s>>>(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8],
                                                                  a[9], static_cast<const float2*>(src),
                                                                  static_cast<float2*>(dst));
        else
            pfa_to_tensor_kernel<double2><<<grid, threads, 0, s>>>(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8],
                                                                   a[9], static_cast<const double2*>(src),
                                                                   static_cast<double2*>(dst));
    } else {
        const uint32_t m0 = (uint32_t)(S % d0), m1 = (uint32_t)(S % d1), m2 = (uint32_t)(S % d2);
        if (p->esize == 8)
            pfa_from_tensor_kernel<float2><<<grid, threads, 0, s>>>((uint32_t)n, (uint32_t)d0, (uint32_t)d1,
                                                                    (uint32_t)d2, m0, m1, m2,
                                                                    static_cast<const float2*>(src),
                                                                    static_cast<float2*>(dst));
        else
            pfa_from_tensor_kernel<double2><<<grid, threads, 0, s>>>((uint32_t)n, (uint32_t)d0, (uint32_t)d1,
                                                                     (uint32_t)d2, m0, m1, m2,
                                                                     static_cast<const double2*>(src),
                                                                     static_cast<double2*>(dst));
    }
    return cudaGetLastError();
}

// a^{-1} mod m (a and m coprime, m >= 1)
static int64_t inverse_mod(int64_t a, int64_t m) {
    int64_t r0 = m, r1 = a % m, s0 = 0, s1 = 1;
    while (r1 != 0) {
        const int64_t q = r0 / r1;
        int64_t t = r0 - q * r1;
        r0 = r1;
        r1 = t;
        t = s0 - q * s1;
        s0 = s1;
        s1 = t;
    }
    s0 %= m;
    return s0 < 0 ? s0 + m : s0;
}

}  // namespace pac

using namespace pac;

static int check_dev_ptr(const void* ptr, const char* name) {
    if (!ptr) return fail(PAC_ERR_ARG, "%s is null", name);
    if (reinterpret_cast<uintptr_t>(ptr) % 16) return fail(PAC_ERR_ARG, "%s is not 16-byte aligned", name);
    return PAC_OK;
}

extern "C" int pac_pfa_create(int64_t n, pac_dtype dtype, pac_pfa* out) {
    if (!out) return fail(PAC_ERR_ARG, "null out");
    *out = nullptr;
    if (dtype != PAC_C64 && dtype != PAC_C128) return fail(PAC_ERR_ARG, "bad dtype %d", (int)dtype);
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(PAC_ERR_SIZE, "length %lld out of range", (long long)n);
    int64_t f[3];
    int t = 0;
    int64_t m = n;
    for (int q : {2, 3, 5}) {
        int64_t pq = 1;
        while (m % q == 0) {
            m /= q;
            pq *= q;
        }
        if (pq > 1) f[t++] = pq;
    }
    if (m != 1) return fail(PAC_ERR_SIZE, "length %lld is not of the form 2^a 3^b 5^c", (long long)n);
    for (int i = 1; i < t; ++i)  // ascending: n_1 <= ... <= n_t
        for (int j = i; j > 0 && f[j - 1] > f[j]; --j) std::swap(f[j - 1], f[j]);
    pac_pfa p = new (std::nothrow) pac_pfa_s();
    if (!p) return fail(PAC_ERR_NOMEM, "host allocation failed");
    p->n = n;
    p->t = t;
    p->dtype = dtype;
    p->esize = dtype == PAC_C64 ? 8 : 16;
    // tensor axes (n_t, ..., n_1) padded on the left with 1s to three axes
    for (int a = 0; a < 3; ++a) {
        const int q = 2 - a;  // axis a holds factor n_{q+1} (zero-based f[q])
        p->dims[a] = q < t ? f[q] : 1;
        const int64_t d = p->dims[a];
        p->crt[a] = d == 1 ? 0 : (n / d) * inverse_mod((n / d) % d, d) % n;
    }
    const int ndim = t > 0 ? t : 1;
    const int64_t* inner_dims = p->dims + (3 - ndim);
    int rc = pac_plan_create(ndim, inner_dims, 0, dtype, &p->inner);
    if (rc) {
        delete p;
        return rc;
    }
    cudaError_t e = cudaMalloc(&p->d_scratch, (size_t)n * p->esize);
    if (e != cudaSuccess) {
        pac_plan_destroy(p->inner);
        delete p;
        return fail(PAC_ERR_NOMEM, "prime factor scratch: %s", cudaGetErrorString(e));
    }
    *out = p;
    return PAC_OK;
}

extern "C" int pac_pfa_destroy(pac_pfa p) {
    if (!p) return PAC_OK;
    cudaDeviceSynchronize();
    if (p->d_scratch) cudaFree(p->d_scratch);
    int rc = p->inner ? pac_plan_destroy(p->inner) : PAC_OK;
    delete p;
    return rc;
}

extern "C" int pac_pfa_filter_spectrum(pac_pfa p, const void* h_dev) {
    if (!p) return fail(PAC_ERR_ARG, "null object");
    if (int rc = check_dev_ptr(h_dev, "h_dev")) return rc;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaError_t e = cudaDeviceSynchronize();  // h may come from any stream
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    e = launch_pfa_map(p, true, h_dev, p->d_scratch, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "prime factor map of h");
    int rc = pac_filter_spectrum(p->inner, p->d_scratch);
    if (rc == PAC_OK) p->has_spec = true;
    return rc;
}

extern "C" int pac_pfa_convolve(pac_pfa p, const void* x_dev, void* y_dev, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null object");
    if (int rc = check_dev_ptr(x_dev, "x_dev")) return rc;
    if (int rc = check_dev_ptr(y_dev, "y_dev")) return rc;
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_pfa_filter_spectrum was not called for this object");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pfa_map(p, true, x_dev, p->d_scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "prime factor map of x");
    int rc = pac_convolve(p->inner, p->d_scratch, p->d_scratch, stream);
    if (rc) return rc;
    e = launch_pfa_map(p, false, p->d_scratch, y_dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "prime factor map of y");
    return PAC_OK;
}

extern "C" int pac_pfa_shape(pac_pfa p, int* t, int64_t* dims) {
    if (!p || !t || !dims) return fail(PAC_ERR_ARG, "null argument");
    *t = p->t;
    for (int a = 0; a < 3; ++a) dims[a] = p->dims[a];
    return PAC_OK;
}

extern "C" int pac_pfa_query(pac_pfa p, int key, int64_t* value) {
    if (!p || !value) return fail(PAC_ERR_ARG, "null argument");
    switch (key) {
        case PAC_Q_NDIM: *value = p->t; return PAC_OK;
        case PAC_Q_N_TOTAL: *value = p->n; return PAC_OK;
        case PAC_Q_ELEM_BYTES: *value = p->esize; return PAC_OK;
        case PAC_Q_HAS_SPECTRUM: *value = p->has_spec ? 1 : 0; return PAC_OK;
        case PAC_Q_LAUNCHES_CONVOLVE: {
            int64_t v = 0;
            if (int rc = pac_plan_query(p->inner, key, &v)) return rc;
            *value = v + 2;
            return PAC_OK;
        }
        case PAC_Q_DEVICE_BYTES: {
            int64_t v = 0;
            if (int rc = pac_plan_query(p->inner, key, &v)) return rc;
            *value = v + p->n * p->esize;
            return PAC_OK;
        }
        default: return pac_plan_query(p->inner, key, value);
    }
}

extern "C" int pac_pfa_plan(pac_pfa p, pac_plan* inner) {
    if (!p || !inner) return fail(PAC_ERR_ARG, "null argument");
    *inner = p->inner;
    return PAC_OK;
}
