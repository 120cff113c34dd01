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
#include <vector>

#include "fft_device.cuh"
#include "pac_internal.h"

namespace pac {

// The maps in tiles.  Write the tensor as m = d_0 d_1 rows of d_2 elements,
// row rho(s) = (s mod d_0) d_1 + (s mod d_1) holding the residues of s.
// Output k has row residue s = k mod m and column c = k mod d_2 (m and d_2
// coprime), k = (s E_m + c E_2) mod n with the idempotents E_m (1 mod m,
// 0 mod d_2) and E_2 (0 mod m, 1 mod d_2).  In the sheared coordinates
// u = s, v = (c - s) mod d_2 a tile is u in [u_0, u_0 + 32), v in
// [v_0, v_0 + 32); its element (p, q) is
//   tensor row rho(u_0 + p), column (u_0 + p + v_0 + q) mod d_2, and
//   output k = K_0 + q E_2 + p (mod n), K_0 = (u_0 E_m + ((u_0 + v_0) mod d_2) E_2) mod n,
// because adding p to both residues adds p to k.  So for fixed p the tile's
// tensor elements are consecutive (a row segment), for fixed q its outputs
// are consecutive: the tile moves through shared memory with 32-element
// runs on both sides.  K_0 per tile and q E_2 mod n per q come from host
// tables (no 64-bit division on the device).
struct PfaMapArgs {
    uint32_t n, m, d0, d1, d2;
    uint32_t tiles_v;          // ceil(d_2 / 32)
    uint32_t tiles;            // ceil(m / 32) * tiles_v
    const uint32_t* k0;        // [tiles] K_0 of each tile
    const uint32_t* qe2;       // [32] q E_2 mod n
};
}  // namespace pac

struct pac_pfa_s {
    int64_t n = 1;
    int t = 0;                       // number of factors
    int64_t dims[3] = {1, 1, 1};     // tensor shape (n_t, ..., n_1), the last index fastest
    pac_dtype dtype = PAC_C64;
    int esize = 8;
    pac_plan inner = nullptr;        // the t-D convolution
    void* d_scratch = nullptr;       // the gathered tensor, n elements
    uint32_t* d_maptab = nullptr;    // tables of the tiled maps (pfa_build_map)
    pac::PfaMapArgs map = {};
    bool has_spec = false;
    std::mutex mu;
};

namespace pac {




// tensor offset of element (p, lane) of a tile: row rho(u_0 + p), column (u_0 + p + v_0 + lane) mod d_2
__device__ __forceinline__ size_t pfa_tensor_off(const PfaMapArgs& a, uint32_t u0, uint32_t v0, int p, int lane) {
    const uint32_t s = u0 + (uint32_t)p;
    const uint32_t row = (s % a.d0) * a.d1 + s % a.d1;
    uint32_t c = (s + v0) % a.d2 + (uint32_t)lane;
    if (c >= a.d2) c -= a.d2;
    return (size_t)row * a.d2 + c;
}

// output index of element (lane, q) of a tile: K_0 + q E_2 + lane (mod n)
__device__ __forceinline__ uint32_t pfa_vector_idx(const PfaMapArgs& a, uint32_t K0, int q, int lane) {
    uint32_t k = K0 + __ldg(a.qe2 + q);
    if (k >= a.n) k -= a.n;
    k += (uint32_t)lane;
    if (k >= a.n) k -= a.n;
    return k;
}

// TO_TENSOR: Gamma^T (tensor entry of k = src[k]); else Gamma (dst[k] = tensor entry of k).
// Each warp moves row segments (lane = q) on the tensor side and output runs
// (lane = p) on the vector side; the 32 x 33 buffer keeps both conflict-free.
template <typename V, bool TO_TENSOR>
__global__ void __launch_bounds__(256) pfa_map_kernel(const PfaMapArgs a, const V* __restrict__ src,
                                                      V* __restrict__ dst) {
    __shared__ V tile[32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t tix = blockIdx.x; tix < a.tiles; tix += gridDim.x) {
        const uint32_t tu = tix / a.tiles_v, tv = tix - tu * a.tiles_v;
        const uint32_t u0 = tu * 32, v0 = tv * 32;
        const int pn = (int)min(32u, a.m - u0), qn = (int)min(32u, a.d2 - v0);
        const uint32_t K0 = __ldg(a.k0 + tix);
        if constexpr (TO_TENSOR) {
            for (int q = warp; q < qn; q += 8)
                if (lane < pn) tile[lane][q] = __ldg(src + pfa_vector_idx(a, K0, q, lane));
            __syncthreads();
            for (int p = warp; p < pn; p += 8)
                if (lane < qn) dst[pfa_tensor_off(a, u0, v0, p, lane)] = tile[p][lane];
        } else {
            for (int p = warp; p < pn; p += 8)
                if (lane < qn) tile[p][lane] = __ldg(src + pfa_tensor_off(a, u0, v0, p, lane));
            __syncthreads();
            for (int q = warp; q < qn; q += 8)
                if (lane < pn) dst[pfa_vector_idx(a, K0, q, lane)] = tile[lane][q];
        }
        __syncthreads();  // the next tile reuses the buffer
    }
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

// a * b mod n without overflow (a, b < n < 2^31)
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t n) { return (a % n) * (b % n) % n; }

// Host tables of the tiled maps: K_0 of every tile and q E_2 mod n (q < 32).
static int pfa_build_map(pac_pfa_s* p, PfaMapArgs* out, uint32_t** d_tab) {
    const uint64_t n = (uint64_t)p->n, d0 = (uint64_t)p->dims[0], d1 = (uint64_t)p->dims[1], d2 = (uint64_t)p->dims[2];
    const uint64_t m = d0 * d1;
    PfaMapArgs a = {};
    a.n = (uint32_t)n;
    a.m = (uint32_t)m;
    a.d0 = (uint32_t)d0;
    a.d1 = (uint32_t)d1;
    a.d2 = (uint32_t)d2;
    a.tiles_v = (uint32_t)((d2 + 31) / 32);
    a.tiles = (uint32_t)((m + 31) / 32) * a.tiles_v;
    // idempotents of the coprime pair (m, d_2)
    const uint64_t Em = d2 == 1 ? 1 % n : mulmod(d2, (uint64_t)inverse_mod((int64_t)(d2 % m), (int64_t)m), n);
    const uint64_t E2 = m == 1 ? 1 % n : mulmod(m, (uint64_t)inverse_mod((int64_t)(m % d2), (int64_t)d2), n);
    std::vector<uint32_t> tab((size_t)a.tiles + 32);
    for (uint32_t tu = 0, i = 0; tu * 32ull < m; ++tu)
        for (uint32_t tv = 0; tv < a.tiles_v; ++tv, ++i) {
            const uint64_t u0 = tu * 32ull, v0 = tv * 32ull;
            tab[i] = (uint32_t)((mulmod(u0, Em, n) + mulmod((u0 + v0) % d2, E2, n)) % n);
        }
    for (uint32_t q = 0; q < 32; ++q) tab[a.tiles + q] = (uint32_t)mulmod(q, E2, n);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d_tab), tab.size() * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "prime factor map tables: %s", cudaGetErrorString(e));
    e = cudaMemcpy(*d_tab, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(*d_tab);
        *d_tab = nullptr;
        return cuda_fail(e, "prime factor map tables");
    }
    a.k0 = *d_tab;
    a.qe2 = *d_tab + a.tiles;
    *out = a;
    return PAC_OK;
}

// Gamma^T (to_tensor) or Gamma; a single factor (or n = 1) is the identity: a copy
static cudaError_t launch_pfa_map(const pac_pfa_s* p, bool to_tensor, const void* src, void* dst, cudaStream_t s) {
    if (p->t <= 1)
        return cudaMemcpyAsync(dst, src, (size_t)p->n * p->esize, cudaMemcpyDeviceToDevice, s);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)device_sm_count(dev) * 8;
    const unsigned grid = (unsigned)std::min<int64_t>(p->map.tiles, cap);
    if (p->esize == 8) {
        if (to_tensor)
            pfa_map_kernel<float2, true><<<grid, 256, 0, s>>>(p->map, (const float2*)src, (float2*)dst);
        else
            pfa_map_kernel<float2, false><<<grid, 256, 0, s>>>(p->map, (const float2*)src, (float2*)dst);
    } else {
        if (to_tensor)
            pfa_map_kernel<double2, true><<<grid, 256, 0, s>>>(p->map, (const double2*)src, (double2*)dst);
        else
            pfa_map_kernel<double2, false><<<grid, 256, 0, s>>>(p->map, (const double2*)src, (double2*)dst);
    }
    return cudaGetLastError();
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
    if (t >= 2) {
        rc = pfa_build_map(p, &p->map, &p->d_maptab);
        if (rc) {
            cudaFree(p->d_scratch);
            pac_plan_destroy(p->inner);
            delete p;
            return rc;
        }
    }
    *out = p;
    return PAC_OK;
}

extern "C" int pac_pfa_destroy(pac_pfa p) {
    if (!p) return PAC_OK;
    cudaDeviceSynchronize();
    if (p->d_scratch) cudaFree(p->d_scratch);
    if (p->d_maptab) cudaFree(p->d_maptab);
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
