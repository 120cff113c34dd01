/*
 * Oracle: plain, slow, FP64 CPU implementations of what the convolution path
 * computes.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * bench's CPU-baseline leg call it; the CUDA library never does.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Every route works on interleaved complex doubles (C99 double complex, the
 * memory layout of numpy complex128) in row-major order, last index fastest
 * (the row-major vec of Section 4 of the paper).
 *
 *   oracle_conv_direct         y[k] = sum_j h[j] x[(k - j) mod n]   (O1)
 *   oracle_conv_direct_points  the same at chosen output indices     (O1)
 *   oracle_conv_separable      axis-by-axis 1-D definition for       (O2)
 *                              h = h_1 (x) h_2 (x) ... (outer product)
 *   oracle_dft                 naive per-axis DFT, w = exp(-+2 pi i/n) (O3)
 *
 * The convolution operator is the paper's F_h(x) = DFT^-1(DFT(h) o DFT(x))
 * (Section 2, eq. "convolution"; d-D form, Section 4), which equals the
 * circular convolution written above; O1 is that definition literally.
 * Sums use Neumaier compensated summation so the oracle's own rounding error
 * stays far below the FP64 tolerance (1e-12 relative L2) it is used with.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* compensated accumulator for one complex sum */
typedef struct {
    double sr, cr, si, ci;
} acc_t;

static void acc_init(acc_t* a) { a->sr = a->cr = a->si = a->ci = 0.0; }

static void neumaier(double* s, double* c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *c += (*s - t) + v;
    else
        *c += (v - t) + *s;
    *s = t;
}

static void acc_add(acc_t* a, cplx v) {
    neumaier(&a->sr, &a->cr, creal(v));
    neumaier(&a->si, &a->ci, cimag(v));
}

static cplx acc_get(const acc_t* a) { return (a->sr + a->cr) + I * (a->si + a->ci); }

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int64_t total_size(int ndim, const int64_t* dims) {
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= dims[a];
    return n;
}

/* one output point of the d-D circular convolution, straight from the definition */
static cplx conv_point(int ndim, const int64_t* dims, const cplx* h, const cplx* x, int64_t k_lin) {
    int64_t k[8], j[8];
    int64_t rem = k_lin;
    for (int a = ndim - 1; a >= 0; --a) {
        k[a] = rem % dims[a];
        rem /= dims[a];
        j[a] = 0;
    }
    int64_t n = total_size(ndim, dims);
    acc_t acc;
    acc_init(&acc);
    for (int64_t jl = 0; jl < n; ++jl) {
        /* linear index of (k - j) mod n, per axis */
        int64_t src = 0;
        for (int a = 0; a < ndim; ++a) {
            int64_t d = k[a] - j[a];
            if (d < 0) d += dims[a];
            src = src * dims[a] + d;
        }
        acc_add(&acc, h[jl] * x[src]);
        /* advance the multi-index j (last axis fastest) */
        for (int a = ndim - 1; a >= 0; --a) {
            if (++j[a] < dims[a]) break;
            j[a] = 0;
        }
    }
    return acc_get(&acc);
}

/* O1: the whole output from the definition; O(N^2). Returns 0, or -1 on bad args. */
int oracle_conv_direct(int ndim, const int64_t* dims, const cplx* h, const cplx* x, cplx* y) {
    if (ndim < 1 || ndim > 8) return -1;
    int64_t n = total_size(ndim, dims);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) y[k] = conv_point(ndim, dims, h, x, k);
    return 0;
}

/* O1 at npts chosen output linear indices idx[0..npts) -> y_pts[0..npts). */
int oracle_conv_direct_points(int ndim, const int64_t* dims, const cplx* h, const cplx* x,
                              int64_t npts, const int64_t* idx, cplx* y_pts) {
    if (ndim < 1 || ndim > 8) return -1;
    int64_t n = total_size(ndim, dims);
    for (int64_t p = 0; p < npts; ++p)
        if (idx[p] < 0 || idx[p] >= n) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < npts; ++p) y_pts[p] = conv_point(ndim, dims, h, x, idx[p]);
    return 0;
}

/*
 * 1-D circular convolution along axis `a` of a row-major array:
 * out[.., k, ..] = sum_j f[j] in[.., (k - j) mod n_a, ..].
 */
static void conv_axis(int ndim, const int64_t* dims, int a, const cplx* f, const cplx* in, cplx* out) {
    int64_t na = dims[a];
    int64_t inner = 1, outer = 1;
    for (int b = a + 1; b < ndim; ++b) inner *= dims[b];
    for (int b = 0; b < a; ++b) outer *= dims[b];
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t o = 0; o < outer; ++o)
        for (int64_t i = 0; i < inner; ++i) {
            const cplx* line = in + o * na * inner + i;
            cplx* oline = out + o * na * inner + i;
            for (int64_t k = 0; k < na; ++k) {
                acc_t acc;
                acc_init(&acc);
                for (int64_t j = 0; j < na; ++j) {
                    int64_t d = k - j;
                    if (d < 0) d += na;
                    acc_add(&acc, f[j] * line[d * inner]);
                }
                oline[k * inner] = acc_get(&acc);
            }
        }
}

/*
 * O2: convolution with a separable filter h = f_0 (x) f_1 (x) ... (x) f_{d-1}
 * (outer product, f_a of length dims[a]).  Circular convolution with an outer
 * product factorises into one 1-D circular convolution per axis, each taken
 * from the definition: N * sum(n_a) multiply-adds.  `work` holds N elements.
 */
int oracle_conv_separable(int ndim, const int64_t* dims, const cplx* const* factors, const cplx* x,
                          cplx* y, cplx* work) {
    if (ndim < 1 || ndim > 8) return -1;
    int64_t n = total_size(ndim, dims);
    /* ping-pong so that the last axis lands in y */
    const cplx* src = x;
    for (int a = 0; a < ndim; ++a) {
        cplx* dst = ((ndim - 1 - a) % 2 == 0) ? y : work;
        conv_axis(ndim, dims, a, factors[a], src, dst);
        src = dst;
    }
    (void)n;
    return 0;
}

/* w_n^m = exp(sign * 2 pi i m / n) with m reduced exactly in integers first */
static cplx root_of_unity(int64_t m, int64_t n, int sign) {
    m %= n;
    if (m < 0) m += n;
    const double two_pi = 6.283185307179586476925286766559;
    double ang = two_pi * (double)m / (double)n;
    return cos(ang) + I * (sign * sin(ang));
}

/*
 * O3: naive multi-dimensional DFT, one axis at a time (the Kronecker form of
 * Section 4): X[k] = sum_j x[j] exp(sign 2 pi i j k / n) along each axis.
 * sign = -1 is the paper's forward DFT (w_n = exp(-2 pi i / n), Section 2);
 * sign = +1 is the unnormalised inverse.  O(N * sum(n_a)), not an FFT.
 * `work` holds N elements.
 */
int oracle_dft(int ndim, const int64_t* dims, const cplx* x, cplx* X, int sign, cplx* work) {
    if (ndim < 1 || ndim > 8 || (sign != 1 && sign != -1)) return -1;
    int64_t n = total_size(ndim, dims);
    memcpy(X, x, sizeof(cplx) * (size_t)n);
    for (int a = 0; a < ndim; ++a) {
        int64_t na = dims[a];
        int64_t inner = 1, outer = 1;
        for (int b = a + 1; b < ndim; ++b) inner *= dims[b];
        for (int b = 0; b < a; ++b) outer *= dims[b];
        cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)na);
        if (!tw) return -2;
        for (int64_t m = 0; m < na; ++m) tw[m] = root_of_unity(m, na, sign);
#pragma omp parallel for collapse(2) schedule(static)
        for (int64_t o = 0; o < outer; ++o)
            for (int64_t i = 0; i < inner; ++i) {
                const cplx* line = X + o * na * inner + i;
                cplx* oline = work + o * na * inner + i;
                for (int64_t k = 0; k < na; ++k) {
                    acc_t acc;
                    acc_init(&acc);
                    for (int64_t j = 0; j < na; ++j) acc_add(&acc, line[j * inner] * tw[(j * k) % na]);
                    oline[k * inner] = acc_get(&acc);
                }
            }
        memcpy(X, work, sizeof(cplx) * (size_t)n);
        free(tw);
    }
    return 0;
}
