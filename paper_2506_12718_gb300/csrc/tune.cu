// Autotuner of pass schedules (pac_tune).
//
// A schedule fixes how many DIF stages one pass fuses (the largest group
// size, as a cap on its exponent), whether the last two axes may run as one
// plane pass, and the plane pass' tile (a whole plane per CTA or a plane split
// over a K-CTA cluster).  Large groups mean few passes over HBM but narrow tiles
// and few resident CTAs; small groups the opposite, so the best choice
// depends on the shape and the GPU and is measured, not guessed: every
// candidate that gives a different split is built, run on scratch data and
// timed with CUDA events, and the fastest is remembered per
// (dims, radix, dtype).  For stage lists of several prime bases (radix 0)
// the candidates also include one-base groups only against groups spanning
// bases.  With PAC_TUNE_FILE set, schedules persist in that file as lines
// "ndim n0 n1 n2 radix dtype cap flags us", flags bit 0 = plane pass allowed,
// bit 1 = groups may not span bases, bits 4-7 = CTAs per plane (0: the
// default rule).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "pac_internal.h"

using namespace pac;

namespace {

struct Key {
    int ndim;
    int64_t d[3];
    int radix, dtype;
    bool operator<(const Key& o) const {
        if (ndim != o.ndim) return ndim < o.ndim;
        for (int a = 0; a < 3; ++a)
            if (d[a] != o.d[a]) return d[a] < o.d[a];
        if (radix != o.radix) return radix < o.radix;
        return dtype < o.dtype;
    }
};

struct Tuned {
    Schedule sch;
    double us = 0;
};

std::mutex g_mu;
std::map<Key, Tuned> g_tuned;
bool g_loaded = false;

Key make_key(int ndim, const int64_t* dims, int radix, pac_dtype dtype) {
    Key k;
    k.ndim = ndim;
    for (int a = 0; a < 3; ++a) k.d[a] = a < ndim ? dims[a] : 1;
    k.radix = radix;
    k.dtype = (int)dtype;
    return k;
}

void load_file_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = std::getenv("PAC_TUNE_FILE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    Key k;
    long long n0, n1, n2;
    int cap, plane;
    double us;
    while (std::fscanf(f, "%d %lld %lld %lld %d %d %d %d %lf", &k.ndim, &n0, &n1, &n2, &k.radix, &k.dtype, &cap,
                       &plane, &us) == 9) {
        k.d[0] = n0;
        k.d[1] = n1;
        k.d[2] = n2;
        Tuned t;
        t.sch.cap = cap;
        t.sch.plane = (plane & 1) != 0;
        t.sch.mixed = (plane & 2) == 0;
        t.sch.plane_k = (plane >> 4) & 15;
        t.sch.nv = (plane >> 2) & 1;
        t.us = us;
        g_tuned[k] = t;  // later lines win
    }
    std::fclose(f);
}

void append_file(const Key& k, const Tuned& t) {
    const char* path = std::getenv("PAC_TUNE_FILE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %lld %lld %lld %d %d %d %d %.3f\n", k.ndim, (long long)k.d[0], (long long)k.d[1],
                 (long long)k.d[2], k.radix, k.dtype, t.sch.cap,
                 (t.sch.plane ? 1 : 0) | (t.sch.mixed ? 0 : 2) | (t.sch.nv ? 4 : 0) | ((t.sch.plane_k & 15) << 4),
                 t.us);
    std::fclose(f);
}

// Median time (us) of `reps` convolutions of plan p on scratch arrays.
int time_plan(pac_plan p, void* x, void* y, int reps, double* us) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    std::vector<cudaEvent_t> ev(2 * reps, nullptr);
    int rc = PAC_OK;
    for (auto& x_ : ev)
        if (cudaEventCreate(&x_) != cudaSuccess) rc = PAC_ERR_CUDA;
    for (int w = 0; w < 2 && rc == PAC_OK; ++w) rc = pac_convolve(p, x, y, s);
    for (int r = 0; r < reps && rc == PAC_OK; ++r) {
        cudaEventRecord(ev[2 * r], s);
        rc = pac_convolve(p, x, y, s);
        cudaEventRecord(ev[2 * r + 1], s);
    }
    e = cudaStreamSynchronize(s);
    if (rc == PAC_OK && e != cudaSuccess) rc = cuda_fail(e, "tuning run");
    std::vector<float> ms;
    if (rc == PAC_OK) {
        for (int r = 0; r < reps; ++r) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[2 * r], ev[2 * r + 1]);
            ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        *us = 1e3 * ms[ms.size() / 2];
    }
    for (auto x_ : ev)
        if (x_) cudaEventDestroy(x_);
    cudaStreamDestroy(s);
    return rc;
}

}  // namespace

namespace pac {

bool tuned_schedule(int ndim, const int64_t* dims, int radix, pac_dtype dtype, Schedule* out) {
    *out = Schedule();
    if (ndim < 1 || ndim > 3 || !dims) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    auto it = g_tuned.find(make_key(ndim, dims, radix, dtype));
    if (it == g_tuned.end()) return false;
    *out = it->second.sch;
    return true;
}

}  // namespace pac

extern "C" int pac_tune(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int reps, double* best_us) {
    if (ndim < 1 || ndim > 3 || !dims || reps < 1) return fail(PAC_ERR_ARG, "bad arguments");
    // candidates: every group cap that changes the split, plane on and off,
    // groups spanning prime bases or not, the plane tile, the default or the
    // narrow tile of the group passes
    std::vector<Schedule> cands;
    std::vector<std::vector<int>> seen;
    for (int mixed = 1; mixed >= 0; --mixed) {
        for (int cap = 12; cap >= 1; --cap) {
            for (int plane = 1; plane >= 0; --plane) {
                Schedule sch;
                sch.cap = cap;
                sch.plane = plane != 0;
                sch.mixed = mixed != 0;
                pac_plan p = nullptr;
                if (plan_build(ndim, dims, radix, dtype, sch, &p) != PAC_OK) continue;
                // the plane tile: every supported split of the plane (0 = the default rule first)
                std::vector<int> ks = {0};
                if (p->plane) {
                    const int m1 = p->groups[p->plane_g1].M, m2 = p->groups[p->plane_g1 + 1].M;
                    for (int k = 1; k <= 5; ++k)
                        if (plane_supported_k(m1, m2, p->esize, k)) ks.push_back(k);
                }
                pac_plan_destroy(p);
                for (int k : ks) {
                    for (int nv = 0; nv <= 1; ++nv) {
                        Schedule sk = sch;
                        sk.plane_k = k;
                        sk.nv = nv;
                        if (plan_build(ndim, dims, radix, dtype, sk, &p) != PAC_OK) continue;
                        std::vector<int> sig;  // the resulting pass structure
                        for (const GroupPlan& g : p->groups)
                            sig.push_back(g.mix_nr > 0 ? -2 * g.M : 2 * g.M + g.nv);
                        sig.push_back(p->plane ? -p->plane_k : 0);
                        pac_plan_destroy(p);
                        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
                        seen.push_back(sig);
                        cands.push_back(sk);
                    }
                }
            }
        }
    }
    if (cands.empty()) return fail(PAC_ERR_SIZE, "no schedule builds for this problem");
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= dims[a];
    const size_t bytes = (size_t)n * (dtype == PAC_C64 ? 8 : 16);
    void *x = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&x, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&y, bytes);
    if (e == cudaSuccess) e = cudaMemset(x, 0, bytes);
    if (e != cudaSuccess) {
        if (x) cudaFree(x);
        return fail(PAC_ERR_NOMEM, "tuning buffers: %s", cudaGetErrorString(e));
    }
    Tuned best;
    best.us = -1;
    int rc = PAC_OK;
    for (const Schedule& sch : cands) {
        pac_plan p = nullptr;
        rc = plan_build(ndim, dims, radix, dtype, sch, &p);
        if (rc == PAC_OK) rc = pac_filter_spectrum(p, x);
        double us = 0;
        if (rc == PAC_OK) rc = time_plan(p, x, y, reps, &us);
        if (p) pac_plan_destroy(p);
        if (rc != PAC_OK) break;
        if (best.us < 0 || us < best.us) {
            best.sch = sch;
            best.us = us;
        }
    }
    cudaFree(x);
    cudaFree(y);
    if (rc != PAC_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_file_locked();
        const Key k = make_key(ndim, dims, radix, dtype);
        g_tuned[k] = best;
        append_file(k, best);
    }
    if (best_us) *best_us = best.us;
    return PAC_OK;
}
