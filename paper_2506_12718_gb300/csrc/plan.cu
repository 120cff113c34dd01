// Plan builder and the plan-level C-ABI entry points.
//
// A plan fixes, per axis, the decimation-in-frequency stage list (Section 2.1
// for a uniform radix; the mixed-radix framework of Section 7.1 for the
// leftover stage), splits it into groups that one CTA can transform in shared
// memory, and builds every table the pass kernels read: round twiddles
// w_M^u, the two-level external twiddles w_L^e, and per group the placement
// of each frequency (the digit-reversed position of the group's stages).
// Twiddles are computed in FP64 on the host and rounded once to the plan's
// precision.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>

#include "pac_internal.h"

namespace pac {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return PAC_ERR_CUDA;
}

void root_fp64(int64_t e, int64_t L, double* re, double* im) {
    e %= L;
    if (e < 0) e += L;
    bool conj = false;
    if (2 * e > L) {  // w^e = conj(w^(L-e))
        e = L - e;
        conj = true;
    }
    const double two_pi = 6.283185307179586476925286766559;
    double c, s;
    if (8 * e <= L) {
        const double a = two_pi * (double)e / (double)L;
        c = std::cos(a);
        s = std::sin(a);
    } else if (8 * e <= 3 * L) {  // cos(2 pi f) = sin(2 pi (1/4 - f))
        const double a = two_pi * (double)(L - 4 * e) / (double)(4 * L);
        c = std::sin(a);
        s = std::cos(a);
    } else {  // cos(2 pi f) = -cos(2 pi (1/2 - f))
        const double a = two_pi * (double)(L - 2 * e) / (double)(2 * L);
        c = -std::cos(a);
        s = std::sin(a);
    }
    *re = c;
    *im = conj ? s : -s;
}

int device_sm_count(int device) {
    static int cache[64] = {0};
    if (device < 0 || device >= 64) return 132;
    if (cache[device] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 132;
        cache[device] = v;
    }
    return cache[device];
}

static int prime_of(int radix) {
    switch (radix) {
        case 2: case 4: case 8: return 2;
        case 3: return 3;
        case 5: return 5;
        default: return 0;
    }
}

static int exact_log(int64_t n, int p) {
    int e = 0;
    while (n > 1 && n % p == 0) {
        n /= p;
        ++e;
    }
    return n == 1 ? e : -1;
}

// Prime base of a stage radix (a power of 2, 3 or 5 that a kernel round
// takes whole), 0 for anything else.
static int stage_base(int r) {
    if (r < 2 || r > 32) return 0;
    for (int p : {2, 3, 5})
        if (exact_log(r, p) >= 1) return p;
    return 0;
}

// DIF stage list of an axis.  radix in {2,3,4,5,8}: [r]*(e/f) then a
// leftover stage p^(e mod f).  radix 0, the mixed-radix framework of
// Section 7.1 for n = 2^a 3^b 5^c: the factor 2^a as radix-4 stages (a
// leftover 2 last), then b stages of 3, then c stages of 5.
static int stage_list(int64_t n, int radix, std::vector<int>& out) {
    out.clear();
    if (n < 1) return fail(PAC_ERR_SIZE, "dimension %lld < 1", (long long)n);
    if (radix == 0) {
        int64_t m = n;
        int e[3] = {0, 0, 0};
        const int ps[3] = {2, 3, 5};
        for (int i = 0; i < 3; ++i)
            while (m % ps[i] == 0) {
                m /= ps[i];
                ++e[i];
            }
        if (m != 1) return fail(PAC_ERR_SIZE, "dimension %lld is not of the form 2^a 3^b 5^c", (long long)n);
        for (int i = 0; i < e[0] / 2; ++i) out.push_back(4);
        if (e[0] % 2) out.push_back(2);
        for (int i = 0; i < e[1]; ++i) out.push_back(3);
        for (int i = 0; i < e[2]; ++i) out.push_back(5);
        return PAC_OK;
    }
    const int p = prime_of(radix);
    if (p == 0) return fail(PAC_ERR_ARG, "radix %d not in {0,2,3,4,5,8}", radix);
    const int e = exact_log(n, p);
    if (e < 0) return fail(PAC_ERR_SIZE, "dimension %lld is not a power of %d (radix %d)", (long long)n, p, radix);
    const int f = exact_log(radix, p);
    for (int i = 0; i < e / f; ++i) out.push_back(radix);
    if (e % f) out.push_back(ipow(p, e % f));
    return PAC_OK;
}

// Position -> frequency of a DIF stage list s_1..s_T: frequency
// k = k_1 + s_1 k_2 + s_1 s_2 k_3 + ... sits at p = sum_i k_i prod_{j>i} s_j.
static void reverse_table(const int* st, int T, int64_t* p2f) {
    int64_t n = 1;
    for (int i = 0; i < T; ++i) n *= st[i];
    std::vector<int64_t> suffix(T + 1, 1);
    for (int i = T - 1; i >= 0; --i) suffix[i] = suffix[i + 1] * st[i];
    for (int64_t k = 0; k < n; ++k) {
        int64_t rem = k, pos = 0;
        for (int i = 0; i < T; ++i) {
            pos += (rem % st[i]) * suffix[i + 1];
            rem /= st[i];
        }
        p2f[pos] = k;
    }
}

// Split stages [lo, hi) of an axis' stage list, all of prime base p, into
// consecutive groups with product <= the largest column one CTA handles (or
// p^cap, a schedule's cap), balanced in size.
static void split_run(const std::vector<int>& st, int lo, int hi, int p, int esize, int cap,
                      std::vector<std::pair<int, int>>& out) {
    const int T = hi;
    std::vector<int> ex(T, 0);
    int etot = 0;
    for (int i = lo; i < T; ++i) {
        ex[i] = exact_log(st[i], p);
        etot += ex[i];
    }
    int emax = exact_log(group_mmax(p, esize), p);
    if (cap > 0 && cap < emax) emax = cap;  // a schedule's smaller group cap (more, smaller passes)
    for (int i = lo; i < T; ++i) emax = std::max(emax, ex[i]);  // a single stage is never split
    int ngroups = (etot + emax - 1) / emax;
    int i = lo, erem = etot;
    for (int gi = 0; gi < ngroups && i < T; ++gi) {
        const int target = (erem + (ngroups - gi) - 1) / (ngroups - gi);
        int acc = 0, first = i;
        while (i < T && (acc == 0 || acc + ex[i] <= std::min(target, emax))) {
            acc += ex[i];
            ++i;
        }
        if (gi == ngroups - 1) {  // the last group takes the rest
            while (i < T) acc += ex[i++];
        }
        out.push_back({first, i - first});
        erem -= acc;
    }
    while (i < T) {  // defensive: any leftover becomes one more group
        out.push_back({i, T - i});
        i = T;
    }
}

// Groups of a stage list that may span prime bases (the runtime-radix
// kernel): the fewest groups with product <= kMixMmax (a stage is never
// split), balanced in size: a group takes the next stage while that brings
// its size closer to the geometric mean of what is left.  Falls back to
// greedy packing if balancing leaves the last group too large.
static std::vector<std::pair<int, int>> split_mixed(const std::vector<int>& st) {
    const int T = (int)st.size();
    std::vector<std::pair<int, int>> greedy;
    for (int i = 0; i < T;) {
        int64_t acc = 1;
        const int first = i;
        while (i < T && (acc == 1 || acc * st[i] <= kMixMmax)) acc *= st[i++];
        greedy.push_back({first, i - first});
    }
    const int ng = (int)greedy.size();
    std::vector<std::pair<int, int>> out;
    double rem = 0;
    for (int r : st) rem += std::log((double)r);
    int i = 0;
    for (int gi = 0; gi < ng && i < T; ++gi) {
        const int first = i;
        if (gi == ng - 1) {
            int64_t acc = 1;
            for (int k = i; k < T; ++k) acc *= st[k];
            if (acc > kMixMmax) return greedy;
            out.push_back({i, T - i});
            i = T;
            break;
        }
        const double target = rem / (ng - gi);
        int64_t acc = 1;
        double lacc = 0;
        while (i < T && (acc == 1 || (acc * st[i] <= kMixMmax &&
                                      std::fabs(lacc + std::log((double)st[i]) - target) < std::fabs(lacc - target)))) {
            acc *= st[i];
            lacc += std::log((double)st[i]);
            ++i;
        }
        out.push_back({first, i - first});
        rem -= lacc;
    }
    if (i < T) return greedy;
    return out;
}

// Groups of an axis' stage list.  One-base groups (a CTA's in-register rounds
// of the one-base kernels take one base): each maximal run of equal base is
// split on its own (one run for a uniform radix).  With several bases and
// sch.mixed, groups spanning bases (split_mixed) are taken instead when they
// are fewer; by default (sch.mixed < 0) only when each of them has a compiled
// kernel (mixed_compiled), since the runtime-radix kernel costs 2-3x a
// compiled pass.
static std::vector<std::pair<int, int>> split_groups(const std::vector<int>& st, int esize, const Schedule& sch) {
    std::vector<std::pair<int, int>> out;
    const int T = (int)st.size();
    int i = 0, runs = 0;
    while (i < T) {
        const int p = stage_base(st[i]);
        int j = i;
        while (j < T && stage_base(st[j]) == p) ++j;
        split_run(st, i, j, p, esize, sch.cap, out);
        ++runs;
        i = j;
    }
    if (runs > 1 && sch.mixed != 0 && !sch.mix_runtime && (sch.cap == 0 || sch.cap >= 12)) {
        // the whole axis as one group when a compiled kernel takes it (6000 = 2^4 3 5^3)
        int64_t n = 1;
        for (int k = 0; k < T; ++k) n *= st[k];
        if (mixed_compiled((int)n) && n > kMixMmax) return {{0, T}};
    }
    if (runs > 1 && sch.mixed != 0) {
        std::vector<std::pair<int, int>> mixed = split_mixed(st);
        bool take = mixed.size() < out.size();
        if (take && sch.mixed < 0) {
            for (auto [first, cnt] : mixed) {
                int m = 1;
                for (int k = 0; k < cnt; ++k) m *= st[first + k];
                if (is_mixed(m) && (!mixed_compiled(m) || sch.mix_runtime)) take = false;
            }
        }
        if (take) return mixed;
    }
    return out;
}

// Round radices of a mixed group of size M for the runtime-radix kernel (the
// rule of config.h, the same rounds a compiled mixed kernel runs).  Returns
// the round count.
static int mix_round_list(int M, int* r) {
    const int n = std::min(mixed_round_count(M), kMixMaxRounds);
    for (int i = 0; i < n; ++i) r[i] = mixed_round_radix(M, i);
    return n;
}

}  // namespace pac

using namespace pac;

// ------------------------------------------------------------- host helpers

extern "C" int pac_stage_list(int64_t n, int radix, int* radices, int* count) {
    if (!count) return fail(PAC_ERR_ARG, "null count");
    std::vector<int> st;
    int rc = stage_list(n, radix, st);
    if (rc) return rc;
    if (radices) {
        if (*count < (int)st.size()) return fail(PAC_ERR_ARG, "radices array too small (%d < %d)", *count, (int)st.size());
        std::copy(st.begin(), st.end(), radices);
    }
    *count = (int)st.size();
    return PAC_OK;
}

extern "C" int pac_reverse_table(int nstages, const int* radices, int64_t* pos_to_freq) {
    if (nstages < 0 || (nstages > 0 && !radices) || !pos_to_freq) return fail(PAC_ERR_ARG, "bad arguments");
    for (int i = 0; i < nstages; ++i)
        if (radices[i] < 2) return fail(PAC_ERR_ARG, "radix %d < 2", radices[i]);
    reverse_table(radices, nstages, pos_to_freq);
    return PAC_OK;
}

extern "C" const char* pac_last_error(void) { return g_err.c_str(); }

extern "C" const char* pac_version(void) { return "pac 0.1 (sm_103a)"; }

// ------------------------------------------------------------------- plans

namespace {

template <typename V, typename T>
void put_root(std::vector<unsigned char>& blob, size_t off, int64_t idx, int64_t e, int64_t L) {
    double re, im;
    root_fp64(e, L, &re, &im);
    V v;
    v.x = (T)re;
    v.y = (T)im;
    std::memcpy(blob.data() + off + idx * sizeof(V), &v, sizeof(V));
}

size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Twiddle table `which` of group g (0: round twiddles w_M^u, u < M; 1: the
// external factor's low table w_L^u, u < T; 2: its high table w_L^{T v},
// v < ceil(L/T)), each root computed in FP64 (root_fp64) and rounded once to
// the plan's precision, written at dst.  The plan builder and the host hook
// pac_plan_twiddles both call this, so the hook returns the uploaded values.
int64_t twiddle_count(const GroupPlan& g, int which) {
    if (which == 0) return g.M;
    if (!g.has_ext) return 0;
    return which == 1 ? g.tw_T : (g.L + g.tw_T - 1) / g.tw_T;
}

// FP64 complex values [off, off + 16 n) of the blob as double-float pairs in
// the same bytes: each double d becomes hi = d rounded to FP32, lo = d - hi
// rounded to FP32
void df_split(std::vector<unsigned char>& blob, size_t off, size_t n) {
    for (size_t i = 0; i < 2 * n; ++i) {
        double d;
        std::memcpy(&d, blob.data() + off + 8 * i, 8);
        const float hl[2] = {(float)d, (float)(d - (double)(float)d)};
        std::memcpy(blob.data() + off + 8 * i, hl, 8);
    }
}

void fill_twiddles(const GroupPlan& g, int esize, int which, std::vector<unsigned char>& blob, size_t off) {
    const int64_t n = twiddle_count(g, which);
    for (int64_t u = 0; u < n; ++u) {
        const int64_t e = which == 2 ? u * g.tw_T : u;
        const int64_t L = which == 0 ? g.M : g.L;
        if (esize == 8) put_root<float2, float>(blob, off, u, e, L);
        else put_root<double2, double>(blob, off, u, e, L);
    }
}

}  // namespace

// Device copies of plan tables (twiddles and placement tables), shared by
// every plan whose tables are the same bytes on the same device, with a
// reference count: plans of one shape, radix, precision and schedule (a
// batch of many instances of one class, the requests of a serving pool)
// upload them once.
namespace {

struct SharedTables {
    void* d = nullptr;
    int refs = 0;
};
using TableKey = std::pair<int, std::vector<unsigned char>>;
std::mutex g_tab_mu;
std::map<TableKey, SharedTables> g_tables;
std::map<void*, std::map<TableKey, SharedTables>::iterator> g_table_of;

int acquire_tables(int device, const std::vector<unsigned char>& blob, void** out) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    TableKey key(device, blob);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
        ++it->second.refs;
        *out = it->second.d;
        return PAC_OK;
    }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, blob.size());
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(PAC_ERR_NOMEM, "device tables: out of memory")
                                              : cuda_fail(e, "cudaMalloc(tables)");
    e = cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy(tables)");
    }
    auto ins = g_tables.emplace(std::move(key), SharedTables{d, 1}).first;
    g_table_of[d] = ins;
    *out = d;
    return PAC_OK;
}

void release_tables(void* d) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto w = g_table_of.find(d);
    if (w == g_table_of.end()) return;
    if (--w->second->second.refs == 0) {
        cudaFree(d);
        g_tables.erase(w->second);
        g_table_of.erase(w);
    }
}

}  // namespace

static void free_plan(pac_plan p) {
    if (!p) return;
    if (p->d_tables) release_tables(p->d_tables);
    if (p->d_spec) cudaFree(p->d_spec);
    if (p->d_spec_nat) cudaFree(p->d_spec_nat);
    if (p->d_scratch) cudaFree(p->d_scratch);
    if (p->d_perm) cudaFree(p->d_perm);
    if (p->d_stage) cudaFree(p->d_stage);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    for (cudaEvent_t ev : p->chunk_ev) cudaEventDestroy(ev);
    delete p;
}

// PAC_LOG=1 in the environment: each plan prints its pass schedule to stderr.
static void log_plan(const pac_plan p) {
    static const bool on = [] {
        const char* e = std::getenv("PAC_LOG");
        return e && e[0] != '0';
    }();
    if (!on) return;
    std::fprintf(stderr, "pac: plan dims");
    for (int a = 0; a < p->ndim; ++a) std::fprintf(stderr, " %lld", (long long)p->dims[a]);
    std::fprintf(stderr, " radix %d %s cap %d:", p->radix, p->esize == 8 ? "c64" : "c128", p->schedule.cap);
    for (const GroupPlan& g : p->groups)
        std::fprintf(stderr, " [axis %d M %d C %lld%s]", g.axis, g.M, (long long)g.C,
                     g.mix_nr > 0 ? " mixed" : (g.nv ? " narrow" : ""));
    if (p->plane) std::fprintf(stderr, " plane %dx%d K=%d", p->groups[p->plane_g1].M, p->groups[p->plane_g1 + 1].M,
                               p->plane_k);
    std::fprintf(stderr, "\n");
}

extern "C" int pac_plan_create(int ndim, const int64_t* dims, int radix, pac_dtype dtype, pac_plan* out) {
    Schedule sch;
    bool have = tuned_schedule(ndim, dims, radix, dtype, &sch);
    // PAC_TUNE=search: tune a problem the first time a plan is made for it
    const char* tune = std::getenv("PAC_TUNE");
    if (!have && tune && std::strcmp(tune, "search") == 0 && ndim >= 1 && ndim <= 3 && dims) {
        double us = 0;
        if (pac_tune(ndim, dims, radix, dtype, 5, &us) == PAC_OK) tuned_schedule(ndim, dims, radix, dtype, &sch);
    }
    int rc = plan_build(ndim, dims, radix, dtype, sch, out);
    if (rc == PAC_OK) log_plan(*out);
    return rc;
}

namespace pac {
static int form_groups(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int esize,
                       const Schedule& sch, std::vector<GroupPlan>& out);
}  // namespace pac

extern "C" int pac_plan_groups(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int flags, int cap,
                               int* axis, int* size, int* rounds, int* count) {
    if (ndim < 1 || ndim > 3 || !dims || !count) return fail(PAC_ERR_ARG, "bad arguments");
    if (dtype != PAC_C64 && dtype != PAC_C128 && dtype != PAC_C128_DF)
        return fail(PAC_ERR_ARG, "bad dtype %d", (int)dtype);
    if (radix != 0 && prime_of(radix) == 0) return fail(PAC_ERR_ARG, "radix %d not in {0,2,3,4,5,8}", radix);
    std::vector<std::vector<int>> st(ndim);
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(PAC_ERR_SIZE, "dimension %lld out of range", (long long)dims[a]);
        if (int rc = stage_list(dims[a], radix, st[a])) return rc;
    }
    Schedule sch;
    sch.cap = cap;
    sch.mixed = (flags & 2) ? -1 : (flags & 1) ? 1 : 0;
    if (dtype == PAC_C128_DF) sch.mixed = 0;  // one-base groups only, as plan_build_stages
    // the tiling rules' key (config.h)
    const int esize = dtype == PAC_C64 ? 8 : (dtype == PAC_C128_DF ? kEsDf : 16);
    std::vector<GroupPlan> gr;
    if (int rc = form_groups(ndim, dims, st, esize, sch, gr)) return rc;
    const int n = (int)gr.size();
    if (axis || size || rounds) {
        if (*count < n) return fail(PAC_ERR_ARG, "room for %d groups, %d needed", *count, n);
        for (int g = 0; g < n; ++g) {
            const GroupPlan& p = gr[g];
            if (axis) axis[g] = p.axis;
            if (size) size[g] = p.M;
            if (rounds) {
                const int nr = p.mix_nr > 0 ? p.mix_nr : round_count(p.M, esize);
                for (int i = 0; i < 8; ++i)
                    rounds[8 * g + i] = i < nr ? (p.mix_nr > 0 ? p.mix_r[i] : round_radix(p.M, esize, i)) : 0;
            }
        }
    }
    *count = n;
    return PAC_OK;
}

extern "C" int pac_plan_twiddles(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int flags, int cap,
                                 int group, int which, void* out, int64_t* count, int64_t* L, int64_t* T) {
    if (ndim < 1 || ndim > 3 || !dims || !count) return fail(PAC_ERR_ARG, "bad arguments");
    if (dtype != PAC_C64 && dtype != PAC_C128 && dtype != PAC_C128_DF)
        return fail(PAC_ERR_ARG, "bad dtype %d", (int)dtype);
    if (radix != 0 && prime_of(radix) == 0) return fail(PAC_ERR_ARG, "radix %d not in {0,2,3,4,5,8}", radix);
    if (which < 0 || which > 2) return fail(PAC_ERR_ARG, "table %d not in {0,1,2}", which);
    std::vector<std::vector<int>> st(ndim);
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(PAC_ERR_SIZE, "dimension %lld out of range", (long long)dims[a]);
        if (int rc = stage_list(dims[a], radix, st[a])) return rc;
    }
    Schedule sch;
    sch.cap = cap;
    sch.mixed = (flags & 2) ? -1 : (flags & 1) ? 1 : 0;
    if (dtype == PAC_C128_DF) sch.mixed = 0;
    std::vector<GroupPlan> gr;
    const int esize = dtype == PAC_C64 ? 8 : 16;  // bytes of an entry (double-float: two FP32 pairs)
    if (int rc = form_groups(ndim, dims, st, dtype == PAC_C128_DF ? kEsDf : esize, sch, gr)) return rc;
    if (group < 0 || group >= (int)gr.size()) return fail(PAC_ERR_ARG, "group %d of %d", group, (int)gr.size());
    const GroupPlan& g = gr[group];
    const int64_t n = twiddle_count(g, which);
    if (L) *L = which == 0 ? g.M : g.L;
    if (T) *T = g.tw_T;
    if (out) {
        if (*count < n) return fail(PAC_ERR_ARG, "room for %lld entries, %lld needed", (long long)*count, (long long)n);
        std::vector<unsigned char> blob((size_t)std::max<int64_t>(n, 1) * esize);
        fill_twiddles(g, esize, which, blob, 0);
        if (dtype == PAC_C128_DF) df_split(blob, 0, (size_t)n);  // the pairs a double-float plan uploads
        std::memcpy(out, blob.data(), (size_t)n * esize);
    }
    *count = n;
    return PAC_OK;
}

extern "C" int pac_plan_create_stages(int ndim, const int64_t* dims, const int* nstages, const int* stages,
                                      pac_dtype dtype, pac_plan* out) {
    if (!out) return fail(PAC_ERR_ARG, "null out");
    *out = nullptr;
    if (ndim < 1 || ndim > 3 || !dims || !nstages) return fail(PAC_ERR_ARG, "ndim must be 1, 2 or 3");
    std::vector<std::vector<int>> st(ndim);
    int at = 0;
    for (int a = 0; a < ndim; ++a) {
        if (nstages[a] < 0 || nstages[a] > 64) return fail(PAC_ERR_ARG, "axis %d: %d stages", a, nstages[a]);
        if (nstages[a] > 0 && !stages) return fail(PAC_ERR_ARG, "null stages");
        st[a].assign(stages + at, stages + at + nstages[a]);
        at += nstages[a];
    }
    int rc = plan_build_stages(ndim, dims, st, -1, dtype, Schedule(), out);
    if (rc == PAC_OK) log_plan(*out);
    return rc;
}

namespace pac {

// The pass groups of a problem, forward order (axis 0 first, the contiguous
// axis last): per axis, the stage list split by split_groups; for each group
// its size, block length L, row stride, columns, external-factor split and,
// for a group spanning prime bases, its round radices.  Host only.
static int form_groups(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int esize,
                       const Schedule& sch, std::vector<GroupPlan>& out) {
    out.clear();
    int64_t N = 1;
    for (int a = 0; a < ndim; ++a) N *= dims[a];
    for (int a = 0; a < ndim; ++a) {
        int64_t inner = 1;
        for (int b = a + 1; b < ndim; ++b) inner *= dims[b];
        int64_t Lcur = dims[a];
        for (auto [first, cnt] : split_groups(stages[a], esize, sch)) {
            GroupPlan g;
            g.axis = a;
            g.first_stage = first;
            g.nstages = cnt;
            g.M = 1;
            for (int i = 0; i < cnt; ++i) g.M *= stages[a][first + i];
            g.L = Lcur;
            g.Lp = Lcur / g.M;
            g.I = inner;
            g.C = g.Lp * inner;
            g.Q = N / g.M;
            g.has_ext = g.Lp > 1;
            bool one_base = true;
            for (int i = 1; i < cnt; ++i)
                if (stage_base(stages[a][first + i]) != stage_base(stages[a][first])) one_base = false;
            if (!one_base) {
                if (g.M > kMixMmax && !mixed_compiled(g.M))
                    return fail(PAC_ERR_SIZE, "mixed group size %d above %d", g.M, kMixMmax);
                // a compiled mixed kernel runs the config.h rounds (mix_nr = 0), else the runtime-radix kernel
                if (!mixed_compiled(g.M) || sch.mix_runtime) g.mix_nr = mix_round_list(g.M, g.mix_r);
            } else if (!pass_kernel_supported(g.M, esize)) {
                return fail(PAC_ERR_SIZE, "no pass kernel for group size %d", g.M);
            }
            // two-level split of the external exponent e = hi T + lo: T = p^ceil(e/2)
            // when L = p^e, else (mixed radix) T = ceil(sqrt(L))
            g.tw_T = 0;
            for (int q : {2, 3, 5}) {
                const int eL = exact_log(g.L, q);
                if (eL >= 0) {
                    g.tw_T = ipow(q, (eL + 1) / 2);
                    g.tw_shift = (q == 2) ? (eL + 1) / 2 : -1;
                    break;
                }
            }
            if (g.tw_T == 0) {
                int64_t T = (int64_t)std::sqrt((double)g.L);
                while (T * T < g.L) ++T;
                g.tw_T = (int)T;
                g.tw_shift = -1;
            }
            out.push_back(g);
            Lcur = g.Lp;
        }
    }
    return PAC_OK;
}

int plan_build(int ndim, const int64_t* dims, int radix, pac_dtype dtype, const Schedule& sch, pac_plan* out) {
    if (!out) return fail(PAC_ERR_ARG, "null out");
    *out = nullptr;
    if (ndim < 1 || ndim > 3 || !dims) return fail(PAC_ERR_ARG, "ndim must be 1, 2 or 3");
    if (radix != 0 && prime_of(radix) == 0) return fail(PAC_ERR_ARG, "radix %d not in {0,2,3,4,5,8}", radix);
    std::vector<std::vector<int>> st(ndim);
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(PAC_ERR_SIZE, "dimension %lld out of range", (long long)dims[a]);
        int rc = stage_list(dims[a], radix, st[a]);
        if (rc) return rc;
    }
    return plan_build_stages(ndim, dims, st, radix, dtype, sch, out);
}

// host_blob != NULL: build the groups and the table blob on the host only (no
// device call: no plane pass, tables and spectrum left to the caller)
static int plan_build_impl(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int radix,
                           pac_dtype dtype, const Schedule& sch, pac_plan* out,
                           std::vector<unsigned char>* host_blob);

int plan_build_stages(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int radix,
                      pac_dtype dtype, const Schedule& sch, pac_plan* out) {
    return plan_build_impl(ndim, dims, stages, radix, dtype, sch, out, nullptr);
}

static int plan_build_impl(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int radix,
                           pac_dtype dtype, const Schedule& sch, pac_plan* out,
                           std::vector<unsigned char>* host_blob) {
    if (!out) return fail(PAC_ERR_ARG, "null out");
    *out = nullptr;
    if (ndim < 1 || ndim > 3 || !dims || (int)stages.size() != ndim) return fail(PAC_ERR_ARG, "ndim must be 1, 2 or 3");
    if (dtype != PAC_C64 && dtype != PAC_C128 && dtype != PAC_C128_DF)
        return fail(PAC_ERR_ARG, "bad dtype %d", (int)dtype);
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(PAC_ERR_SIZE, "dimension %lld out of range", (long long)dims[a]);
        int64_t prod = 1;
        for (int r : stages[a]) {
            if (stage_base(r) == 0)
                return fail(PAC_ERR_SIZE, "stage %d of axis %d is not a power of 2, 3 or 5 in [2, 32]", r, a);
            prod *= r;
            if (prod > dims[a]) break;
        }
        if (prod != dims[a])
            return fail(PAC_ERR_SIZE, "the stages of axis %d do not multiply to %lld", a, (long long)dims[a]);
    }

    // N < 2^31 (32-bit element offsets in the kernels), checked before each
    // multiply so that no product of up to three 2^30 dims can overflow
    int64_t n_total = 1;
    for (int a = 0; a < ndim; ++a) {
        if (n_total > ((int64_t(1) << 31) - 1) / dims[a]) {
            double n = 1.0;  // exact for the message: a product of at most three 2^30 dims
            for (int b = 0; b < ndim; ++b) n *= (double)dims[b];
            return fail(PAC_ERR_SIZE, "N = %.0f too large (the kernels take N < 2^31)", n);
        }
        n_total *= dims[a];
    }

    pac_plan pl = new (std::nothrow) pac_plan_s();
    if (!pl) return fail(PAC_ERR_NOMEM, "host allocation failed");
    pl->ndim = ndim;
    pl->radix = radix;
    pl->dtype = dtype;
    pl->esize = dtype == PAC_C64 ? 8 : 16;
    pl->df = dtype == PAC_C128_DF;
    pl->ces = pl->df ? kEsDf : pl->esize;
    pl->N = n_total;
    for (int a = 0; a < ndim; ++a) pl->dims[a] = dims[a];
    pl->stages = stages;
    pl->pos_to_freq.resize(ndim);
    for (int a = 0; a < ndim; ++a) {
        pl->pos_to_freq[a].resize(dims[a]);
        reverse_table(pl->stages[a].data(), (int)pl->stages[a].size(), pl->pos_to_freq[a].data());
    }

    // groups, forward order: axis 0 (outermost) first, the contiguous axis last;
    // PAC_MIXED=1 / 0 in the environment forces groups spanning prime bases on / off,
    // PAC_MIXED=rt on and every one of them in the runtime-radix kernel
    Schedule gs = sch;
    const char* me = std::getenv("PAC_MIXED");
    if (me && (me[0] == '0' || me[0] == '1')) gs.mixed = me[0] == '1' ? 1 : 0;
    if (me && me[0] == 'r' && me[1] == 't') {
        gs.mixed = 1;
        gs.mix_runtime = true;
    }
    if (pl->df) {  // the double-float kernels are compiled for one-base groups only
        gs.mixed = 0;
        gs.mix_runtime = false;
    }
    if (int rc = form_groups(ndim, dims, pl->stages, pl->ces, gs, pl->groups)) {
        delete pl;
        return rc;
    }
    size_t off = 0;  // the groups' tables in one device allocation
    for (GroupPlan& g : pl->groups) {
        g.off_twi = off;
        off = align16(off + (size_t)g.M * pl->esize);
        if (g.has_ext) {
            g.off_lo = off;
            off = align16(off + (size_t)g.tw_T * pl->esize);
            g.off_hi = off;
            off = align16(off + (size_t)((g.L + g.tw_T - 1) / g.tw_T) * pl->esize);
        }
        g.off_rowmap = off;
        off = align16(off + (size_t)g.M * sizeof(int));
        g.off_freq = off;
        off = align16(off + (size_t)g.M * sizeof(int));
        g.off_r2g = off;
        off = align16(off + (size_t)g.M * sizeof(int));
        g.off_r2f = off;
        off = align16(off + (size_t)g.M * sizeof(int));
    }

    // single-launch (cooperative) form of the pass sequence: opt-in per plan,
    // PAC_SINGLE_LAUNCH=1 in the environment when the plan is created
    const char* sl = std::getenv("PAC_SINGLE_LAUNCH");
    pl->single_launch = sl && sl[0] == '1' && !pl->df;
    // plane pass: axis d-1 one group, a supported shape of (last group of axis d-2) x (axis d-1);
    // PAC_PLANE=0 in the environment keeps per-axis passes instead
    const char* pe = std::getenv("PAC_PLANE");
    if (ndim >= 2 && sch.plane && !pl->df && !(pe && pe[0] == '0')) {
        int g_last = 0, g_prev = 0;
        for (const GroupPlan& g : pl->groups) {
            if (g.axis == ndim - 1) ++g_last;
            if (g.axis == ndim - 2) ++g_prev;
        }
        const int G = (int)pl->groups.size();
        // groups[G-2] is the last group of axis d-2 (no external twiddle), groups[G-1] all of axis d-1
        if (host_blob) {  // host only (the CPU emulation): whole planes in one CTA, where the shape has them
            if (g_last == 1 && g_prev >= 1 && G >= 2 &&
                plane_supported_k(pl->groups[G - 2].M, pl->groups[G - 1].M, pl->esize, 1)) {
                pl->plane = true;
                pl->plane_g1 = G - 2;
                pl->plane_k = 1;
            }
        } else if (g_last == 1 && g_prev >= 1 && G >= 2 &&
                   plane_supported(pl->groups[G - 2].M, pl->groups[G - 1].M, pl->esize)) {
            pl->plane = true;
            pl->plane_g1 = G - 2;
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
            pl->plane_k = plane_cluster(pl->groups[G - 2].M, pl->groups[G - 1].M, pl->esize,
                                        pl->N / ((int64_t)pl->groups[G - 2].M * pl->groups[G - 1].M), dev);
            if (sch.plane_k > 0 && plane_supported_k(pl->groups[G - 2].M, pl->groups[G - 1].M, pl->esize, sch.plane_k))
                pl->plane_k = sch.plane_k;
        }
    }
    // narrow tile variant of the group passes (not the plane pass' groups);
    // PAC_NARROW=1 / 0 in the environment forces it on / off
    int nv = sch.nv;
    const char* ne = std::getenv("PAC_NARROW");
    if (ne && (ne[0] == '0' || ne[0] == '1')) nv = ne[0] == '1' ? 1 : 0;
    if (pl->df) nv = 0;
    for (int i = 0; i < (int)pl->groups.size(); ++i) {
        GroupPlan& g = pl->groups[i];
        const bool in_plane = pl->plane && i >= pl->plane_g1;
        g.nv = nv && !in_plane && g.mix_nr == 0 && has_narrow(g.M, pl->esize) ? 1 : 0;
    }
    pl->uniform_m = 0;
    if (!pl->groups.empty()) {
        pl->uniform_m = pl->groups[0].M;
        for (const GroupPlan& g : pl->groups)
            if (g.M != pl->uniform_m || g.mix_nr > 0 || g.nv) pl->uniform_m = 0;
        if (pl->df) pl->uniform_m = 0;  // no single-launch kernel of the double-float type
    }

    // host blob of every table
    std::vector<unsigned char> blob(std::max<size_t>(off, 16), 0);
    for (const GroupPlan& g : pl->groups) {
        fill_twiddles(g, pl->esize, 0, blob, g.off_twi);
        if (g.has_ext) {
            fill_twiddles(g, pl->esize, 1, blob, g.off_lo);
            fill_twiddles(g, pl->esize, 2, blob, g.off_hi);
        }
        // frequency at each global row: digit reversal over the group's stages
        std::vector<int64_t> f(g.M);
        reverse_table(pl->stages[g.axis].data() + g.first_stage, g.nstages, f.data());
        // shared-memory row of frequency k after the in-place rounds: digit
        // reversal over the round radices (larger rounds first)
        const int nr = g.mix_nr > 0 ? g.mix_nr : round_count(g.M, pl->ces);
        std::vector<int> rr(nr);
        for (int i = 0; i < nr; ++i) rr[i] = g.mix_nr > 0 ? g.mix_r[i] : round_radix(g.M, pl->ces, i);
        std::vector<int64_t> row_freq(g.M);
        reverse_table(rr.data(), nr, row_freq.data());
        std::vector<int> f2r(g.M);
        for (int r = 0; r < g.M; ++r) f2r[row_freq[r]] = r;
        int* rowmap = reinterpret_cast<int*>(blob.data() + g.off_rowmap);
        int* freq = reinterpret_cast<int*>(blob.data() + g.off_freq);
        int* r2g = reinterpret_cast<int*>(blob.data() + g.off_r2g);
        int* r2f = reinterpret_cast<int*>(blob.data() + g.off_r2f);
        for (int gg = 0; gg < g.M; ++gg) {
            freq[gg] = (int)f[gg];
            rowmap[gg] = f2r[f[gg]];
            r2g[rowmap[gg]] = gg;
            r2f[rowmap[gg]] = (int)f[gg];
        }
        if (pl->df) {  // twiddles as double-float pairs: each FP64 value split once into hi + lo
            df_split(blob, g.off_twi, (size_t)g.M);
            if (g.has_ext) {
                df_split(blob, g.off_lo, (size_t)g.tw_T);
                df_split(blob, g.off_hi, (size_t)((g.L + g.tw_T - 1) / g.tw_T));
            }
        }
    }

    if (host_blob) {
        pl->tables_bytes = blob.size();
        pl->spec_elems = pl->N;
        if (!pl->groups.empty() && !pl->plane) {
            const GroupPlan& f = pl->groups.back();
            const int64_t W = group_w(f, pl->ces);
            pl->spec_elems = (f.Q + W - 1) / W * W * f.M;
        }
        pl->schedule = sch;
        *host_blob = std::move(blob);
        *out = pl;
        return PAC_OK;
    }
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "cudaGetDevice");
    }
    pl->tables_bytes = blob.size();
    if (int rc = acquire_tables(pl->device, blob, &pl->d_tables)) {
        free_plan(pl);
        return rc;
    }
    pl->spec_elems = pl->N;
    if (!pl->groups.empty() && !pl->plane) {  // whole tiles of the fused pass (see SpecOrder)
        const GroupPlan& f = pl->groups.back();
        const int64_t W = group_w(f, pl->ces);
        pl->spec_elems = (f.Q + W - 1) / W * W * f.M;
    }
    e = cudaMalloc(&pl->d_spec, (size_t)pl->spec_elems * pl->esize);
    if (e != cudaSuccess) {
        free_plan(pl);
        return e == cudaErrorMemoryAllocation ? fail(PAC_ERR_NOMEM, "filter spectrum: out of memory")
                                              : cuda_fail(e, "cudaMalloc(spectrum)");
    }
    pl->device_bytes = pl->tables_bytes + (size_t)pl->spec_elems * pl->esize;
    pl->schedule = sch;
    *out = pl;
    return PAC_OK;
}

}  // namespace pac

// Test hook (host only): the steps of a plan of this problem with one-base
// groups and per-axis passes, their tables and arrays in host memory, for the
// CPU emulation of the kernels (see pac.h).
extern "C" int pac_test_host_steps(int ndim, const int64_t* dims, int radix, pac_dtype dtype, int cap, int flags,
                                   const void* h, const void* x, void* y, void* spec, void* scratch, void* tables,
                                   int64_t* table_bytes, int64_t* spec_elems, void* steps, int* nsteps) {
    if (ndim < 1 || ndim > 3 || !dims || !table_bytes || !spec_elems || !nsteps) return fail(PAC_ERR_ARG, "bad arguments");
    if (radix != 0 && prime_of(radix) == 0) return fail(PAC_ERR_ARG, "radix %d not in {0,2,3,4,5,8}", radix);
    std::vector<std::vector<int>> st(ndim);
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(PAC_ERR_SIZE, "dimension %lld out of range", (long long)dims[a]);
        if (int rc = stage_list(dims[a], radix, st[a])) return rc;
    }
    Schedule sch;
    sch.cap = cap;
    sch.plane = (flags & 1) != 0;
    sch.mixed = (flags & 4) ? 1 : (flags & 2) ? -1 : 0;  // bit 1: spanning groups with compiled kernels
    sch.mix_runtime = (flags & 4) != 0;                   // bit 2: every spanning group in the runtime-radix kernel
    pac_plan p = nullptr;
    std::vector<unsigned char> blob;
    if (int rc = pac::plan_build_impl(ndim, dims, st, radix, dtype, sch, &p, &blob)) return rc;
    for (const GroupPlan& g : p->groups) {
        if (g.nv || (g.mix_nr > 0 && !(flags & 4))) {  // PAC_NARROW / PAC_MIXED set in the environment
            delete p;
            return fail(PAC_ERR_ARG, "pac_test_host_steps: default tiles and compiled groups only (PAC_NARROW, PAC_MIXED)");
        }
    }
    p->d_tables = tables;  // host memory: the step records point into the caller's buffers
    p->d_spec = spec;
    std::vector<HostStep> out;
    auto pass_step = [&](const Step& s) {
        HostStep r = {};
        r.kind = 0;
        r.M = p->groups[s.group].M;
        r.lines = p->groups[s.group].C == 1 ? 1 : 0;
        r.src = s.src;
        r.dst = s.dst;
        r.a = make_pass(p, p->groups[s.group], s.mode, s.src, s.dst, s.io);
        out.push_back(r);
    };
    const int G = (int)p->groups.size();
    if (G > 0) {
        // the spectrum: forward passes on h, then the reorder with 1/N
        for (int i = 0; i < G; ++i) {
            Step s = {i, kFwd, i == 0 ? h : scratch, scratch};
            if (i == 0) s.io |= kDfSrc64;
            pass_step(s);
        }
        HostStep r = {};
        r.kind = 1;
        r.n = p->N;
        r.scale = 1.0 / (double)p->N;
        r.src = scratch;
        r.dst = spec;
        r.o = spec_order_of(p);
        out.push_back(r);
        std::vector<Step> cs;
        convolve_steps(p, x, y, cs);
        for (const Step& s : cs) {
            if (s.mode != kPlane) {
                pass_step(s);
                continue;
            }
            HostStep r2 = {};
            r2.kind = 2;
            r2.M = p->groups[p->plane_g1].M;
            r2.lines = p->groups[p->plane_g1 + 1].M;
            r2.src = s.src;
            r2.dst = s.dst;
            r2.pa = make_plane(p, s.src, s.dst);
            out.push_back(r2);
        }
    }
    *table_bytes = (int64_t)blob.size();
    *spec_elems = p->spec_elems;
    int rc = PAC_OK;
    if (steps) {
        if (*nsteps < (int)out.size())
            rc = fail(PAC_ERR_ARG, "room for %d steps, %d needed", *nsteps, (int)out.size());
        else
            std::memcpy(steps, out.data(), out.size() * sizeof(HostStep));
    }
    if (rc == PAC_OK && tables) std::memcpy(tables, blob.data(), blob.size());
    if (rc == PAC_OK) *nsteps = (int)out.size();
    p->d_tables = nullptr;
    p->d_spec = nullptr;
    delete p;
    return rc;
}

extern "C" int pac_plan_destroy(pac_plan p) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    cudaDeviceSynchronize();
    batch_forget_plan(p);
    free_plan(p);
    return PAC_OK;
}

// ----------------------------------------------------------------- passes

namespace pac {

// Optional per-launch event recorder of pac_convolve_timed (thread-local, so
// concurrent callers on other threads are unaffected).
struct LaunchTimer {
    std::vector<cudaEvent_t> ev;
    std::vector<int> ids;
    int max = 0;
    bool overflow = false;
};
static thread_local LaunchTimer* t_timer = nullptr;

static void timer_mark(cudaStream_t s, int id, bool before) {
    LaunchTimer* t = t_timer;
    if (!t) return;
    if (before) {
        if ((int)t->ids.size() >= t->max) {
            t->overflow = true;
            return;
        }
        t->ids.push_back(id);
    } else if (t->overflow) {
        return;
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    t->ev.push_back(e);
}

// Storage order of the plan's filter spectrum: the read order of the last
// forward round of its fused pass (the last group).
SpecOrder spec_order_of(pac_plan p) {
    const GroupPlan& f = p->groups.back();
    SpecOrder o;
    o.M2 = 0;
    o.rowmap2 = nullptr;
    if (p->plane) {  // the plane pass: product in the last forward round of axis d-2
        const GroupPlan& g1 = p->groups[p->plane_g1];
        const unsigned char* t = static_cast<const unsigned char*>(p->d_tables);
        o.M = (uint32_t)g1.M;
        o.W = (uint32_t)f.M;
        o.C = (uint32_t)g1.C;
        o.R = (uint32_t)round_radix(g1.M, p->esize, round_count(g1.M, p->esize) - 1);
        o.K = (uint32_t)p->plane_k;
        o.tasks = o.W / o.K * o.M / o.R;
        o.rowmap = reinterpret_cast<const int*>(t + g1.off_rowmap);
        o.M2 = (uint32_t)f.M;
        o.rowmap2 = reinterpret_cast<const int*>(t + f.off_rowmap);
        return o;
    }
    o.K = 1;
    o.M = (uint32_t)f.M;
    o.W = (uint32_t)group_w(f, p->ces);
    o.C = (uint32_t)f.C;
    if (f.mix_nr > 0) {
        o.R = (uint32_t)f.mix_r[f.mix_nr - 1];
    } else {
        const int nr = round_count(f.M, p->ces);
        o.R = (uint32_t)round_radix(f.M, p->ces, nr - 1);
    }
    o.tasks = o.W * o.M / o.R;
    o.rowmap = reinterpret_cast<const int*>(static_cast<const unsigned char*>(p->d_tables) + f.off_rowmap);
    return o;
}

PassArgs make_pass(pac_plan p, const GroupPlan& g, int mode, const void* src, void* dst, int io) {
    PassArgs a;
    const unsigned char* t = static_cast<const unsigned char*>(p->d_tables);
    a.src = src;
    a.dst = dst;
    a.spec = p->d_spec;
    a.tw_int = t + g.off_twi;
    a.tw_lo = g.has_ext ? t + g.off_lo : nullptr;
    a.tw_hi = g.has_ext ? t + g.off_hi : nullptr;
    a.rowmap = reinterpret_cast<const int*>(t + g.off_rowmap);
    a.freq = reinterpret_cast<const int*>(t + g.off_freq);
    a.r2g = reinterpret_cast<const int*>(t + g.off_r2g);
    a.r2f = reinterpret_cast<const int*>(t + g.off_r2f);
    a.Q = g.Q;
    a.C = g.C;
    a.I = g.I;
    const int W = group_w(g, p->ces);
    a.tiles = (g.Q + W - 1) / W;
    a.tile0 = 0;
    a.tw_T = g.tw_T;
    a.tw_shift = g.tw_shift;
    a.mode = mode;
    a.has_ext = g.has_ext ? 1 : 0;
    a.nv = g.nv;
    a.df = p->df ? (kDfKernel | io) : 0;
    a.mix_nr = g.mix_nr;
    a.mix_m = g.M;
    a.mix_w = W;
    for (int i = 0; i < 8; ++i) a.mix_r[i] = i < g.mix_nr ? g.mix_r[i] : 0;
    return a;
}

PlaneArgs make_plane(pac_plan p, const void* src, void* dst) {
    PlaneArgs pa;
    pa.a1 = make_pass(p, p->groups[p->plane_g1], kPlane, src, dst);
    pa.a2 = make_pass(p, p->groups[p->plane_g1 + 1], kPlane, src, dst);
    pa.planes = p->N / ((int64_t)p->groups[p->plane_g1].M * p->groups[p->plane_g1 + 1].M);
    return pa;
}

static int run_plane(pac_plan p, const void* src, void* dst, cudaStream_t s) {
    const PlaneArgs pa = make_plane(p, src, dst);
    timer_mark(s, 6, true);
    cudaError_t e = launch_plane(p->esize, p->groups[p->plane_g1].M, p->groups[p->plane_g1 + 1].M, p->plane_k, pa, s);
    timer_mark(s, 6, false);
    if (e != cudaSuccess) return cuda_fail(e, "plane kernel launch");
    return PAC_OK;
}

int run_pass(pac_plan p, const GroupPlan& g, int mode, const void* src, void* dst, cudaStream_t s, int io) {
    const PassArgs a = make_pass(p, g, mode, src, dst, io);
    const int kid = mode == kFwd ? 0 : (mode == kFused ? 1 : 2);
    timer_mark(s, kid, true);
    cudaError_t e = launch_pass(p->esize, g.M, a, s);
    timer_mark(s, kid, false);
    if (e != cudaSuccess) return cuda_fail(e, "pass kernel launch");
    return PAC_OK;
}


// A pass sequence as one cooperative launch (every group of size uniform_m,
// no plane pass); target_bias and spin_limit as in ConvArgs (0 and 0 except
// from the timeout test hook).
static int run_single(pac_plan p, const std::vector<Step>& steps, int grid, unsigned target_bias, unsigned spin_limit,
                      cudaStream_t s) {
    const int n = (int)steps.size();
    ConvArgs args;
    args.npasses = n;
    for (int i = 0; i < n; ++i) {
        const Step& st = steps[i];
        args.pass[i] = make_pass(p, p->groups[st.group], st.mode, st.src, st.dst);
    }
    int rc = barrier_slot(p->device, &args.barrier, &args.base, (unsigned)((n - 1) * grid), &args.error);
    if (rc) return rc;
    args.target_bias = target_bias;
    args.spin_limit = spin_limit;
    timer_mark(s, 5, true);
    cudaError_t e = launch_conv(p->esize, p->uniform_m, args, grid, s);
    timer_mark(s, 5, false);
    if (e != cudaSuccess) return cuda_fail(e, "convolution kernel launch");
    return PAC_OK;
}

// Run a pass sequence: as one cooperative launch when every group has the
// same size M and single launches are allowed, else one launch per pass.
static int run_steps(pac_plan p, const std::vector<Step>& steps, cudaStream_t s, bool allow_single) {
    const int n = (int)steps.size();
    bool single = allow_single && p->single_launch && !p->plane && n > 1 && n <= kMaxPasses && p->uniform_m > 0;
    int grid = 0;
    if (single) {
        grid = conv_grid(p->esize, p->uniform_m, p->device);
        single = grid > 0;
    }
    if (single) return run_single(p, steps, grid, 0u, 0u, s);
    for (const Step& st : steps) {
        int rc = st.mode == kPlane ? run_plane(p, st.src, st.dst, s)
                                   : run_pass(p, p->groups[st.group], st.mode, st.src, st.dst, s, st.io);
        if (rc) return rc;
    }
    return PAC_OK;
}

static cudaError_t timed_permute(pac_plan p, const int64_t* const* idx, const void* src, void* dst, const void* mul,
                                 cudaStream_t s) {
    timer_mark(s, 3, true);
    cudaError_t e = launch_permute(p->esize, p->ndim, p->dims, idx, src, dst, mul, s);
    timer_mark(s, 3, false);
    return e;
}

// The convolution of Algorithm 11 on device pointers: forward groups (the last fused
// with the product and the first inverse group), then the inverse groups.
int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s, bool allow_single) {
    const int G = (int)p->groups.size();
    if (G == 0) {  // N = 1
        timer_mark(s, 4, true);
        cudaError_t e = launch_pointwise_mul(p->esize, p->N, x, p->d_spec, y, 1.0, s);
        timer_mark(s, 4, false);
        return e == cudaSuccess ? PAC_OK : cuda_fail(e, "pointwise kernel");
    }
    std::vector<Step> steps;
    convolve_steps(p, x, y, steps);
    return run_steps(p, steps, s, allow_single);
}

// The convolution of Algorithm 11 as a pass sequence: forward groups (the last fused
// with the product and the first inverse group), then the inverse groups.
// With a plane pass, the groups of the last two axes are one step.
void convolve_steps(pac_plan p, const void* x, void* y, std::vector<Step>& steps) {
    const int G = (int)p->groups.size();
    steps.clear();
    if (p->plane) {
        const int g1 = p->plane_g1;
        for (int i = 0; i < g1; ++i) steps.push_back({i, kFwd, i == 0 ? x : y, y});
        steps.push_back({g1, kPlane, g1 == 0 ? x : y, y});
        for (int i = g1 - 1; i >= 0; --i) steps.push_back({i, kInv, y, y});
        return;
    }
    for (int i = 0; i < G; ++i) steps.push_back({i, i == G - 1 ? kFused : kFwd, i == 0 ? x : y, y});
    for (int i = G - 2; i >= 0; --i) steps.push_back({i, kInv, y, y});
    if (!steps.empty()) {  // double-float plans: the caller's x and y are complex FP64
        steps.front().io |= kDfSrc64;
        steps.back().io |= kDfDst64;
    }
}

int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s) { return run_convolve(p, x, y, s, true); }

int run_forward(pac_plan p, const void* x, void* xhat, cudaStream_t s) {
    const int G = (int)p->groups.size();
    if (G == 0) {
        cudaError_t e = launch_pointwise_mul(p->esize, p->N, x, nullptr, xhat, 1.0, s);
        return e == cudaSuccess ? PAC_OK : cuda_fail(e, "pointwise kernel");
    }
    std::vector<Step> steps;
    for (int i = 0; i < G; ++i) steps.push_back({i, kFwd, i == 0 ? x : xhat, xhat});
    steps.front().io |= kDfSrc64;  // double-float plans: x is complex FP64, xhat double-float pairs
    return run_steps(p, steps, s, true);
}

}  // namespace pac

namespace pac {
int df_unsupported(pac_plan p, const char* what) {
    return p && p->df ? fail(PAC_ERR_ARG, "%s does not take double-float (PAC_C128_DF) plans", what) : PAC_OK;
}
}  // namespace pac

static int check_ptr(const void* ptr, const char* name) {
    if (!ptr) return fail(PAC_ERR_ARG, "%s is null", name);
    if (reinterpret_cast<uintptr_t>(ptr) % 16) return fail(PAC_ERR_ARG, "%s is not 16-byte aligned", name);
    return PAC_OK;
}

// Test hook of the bounded waits (see pac.h): the convolution's passes as one
// cooperative launch whose barriers wait for one arrival more than the grid
// makes, each wait limited to spin_limit polls.
extern "C" int pac_test_barrier_timeout(pac_plan p, const void* x_dev, void* y_dev, void* stream, int spin_limit) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = df_unsupported(p, "pac_test_barrier_timeout")) return rc;
    if (int rc = check_ptr(x_dev, "x_dev")) return rc;
    if (int rc = check_ptr(y_dev, "y_dev")) return rc;
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_filter_spectrum was not called for this plan");
    if (spin_limit < 1 || spin_limit > (1 << 20)) return fail(PAC_ERR_ARG, "spin_limit %d not in [1, 2^20]", spin_limit);
    const int G = (int)p->groups.size();
    std::vector<Step> steps;
    if (G > 0 && !p->plane) convolve_steps(p, x_dev, y_dev, steps);
    const int n = (int)steps.size();
    if (n < 2 || n > kMaxPasses || p->uniform_m == 0)
        return fail(PAC_ERR_ARG, "the plan has no single-launch form (needs >= 2 passes of one group size, no plane pass)");
    const int grid = conv_grid(p->esize, p->uniform_m, p->device);
    if (grid <= 0) return fail(PAC_ERR_CUDA, "no co-resident grid for the cooperative kernel");
    return run_single(p, steps, grid, 1u, (unsigned)spin_limit, static_cast<cudaStream_t>(stream));
}


// Load and set up (module load, shared-memory attribute, occupancy) every
// kernel the plan's convolution launches, with launches of no work, so that
// the first convolution (a served request, a captured graph) does not pay
// for it.
static int prepare_convolve(pac_plan p) {
    std::vector<Step> steps;
    convolve_steps(p, nullptr, nullptr, steps);
    for (const Step& st : steps) {
        cudaError_t e;
        if (st.mode == kPlane) {
            PlaneArgs pa = make_plane(p, nullptr, nullptr);
            pa.planes = 0;
            e = launch_plane(p->esize, p->groups[p->plane_g1].M, p->groups[p->plane_g1 + 1].M, p->plane_k, pa, 0);
        } else {
            PassArgs a = make_pass(p, p->groups[st.group], st.mode, nullptr, nullptr);
            a.tiles = 0;
            e = launch_pass(p->esize, p->groups[st.group].M, a, 0);
        }
        if (e != cudaSuccess) return cuda_fail(e, "kernel set-up");
    }
    return PAC_OK;
}

extern "C" int pac_filter_spectrum(pac_plan p, const void* h_dev) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = check_ptr(h_dev, "h_dev")) return rc;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaError_t e = cudaDeviceSynchronize();  // h may come from any stream
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    int rc;
    void* tmp = nullptr;
    if (p->groups.empty()) {  // N = 1
        e = launch_pointwise_mul(p->esize, p->N, h_dev, nullptr, p->d_spec, 1.0 / (double)p->N, s);
        rc = e == cudaSuccess ? PAC_OK : cuda_fail(e, "pointwise kernel");
    } else {
        // A^T h in the plain index-reversed order, then once into the order
        // the fused pass reads it, times 1/N (the scale of the inverse)
        e = cudaMalloc(&tmp, (size_t)p->bytes());
        if (e != cudaSuccess) {
            cudaStreamDestroy(s);
            return fail(PAC_ERR_NOMEM, "filter spectrum staging: %s", cudaGetErrorString(e));
        }
        rc = run_forward(p, h_dev, tmp, s);
        if (rc == PAC_OK) {
            e = p->df ? launch_spec_order_df(spec_order_of(p), p->N, tmp, p->d_spec, s, 1.0 / (double)p->N)
                      : launch_spec_order(p->esize, spec_order_of(p), p->N, tmp, p->d_spec, true, s, 1.0 / (double)p->N);
            if (e != cudaSuccess) rc = cuda_fail(e, "spectrum order kernel");
        }
    }
    e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (tmp) cudaFree(tmp);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "filter spectrum");
    if (int prc = prepare_convolve(p)) return prc;
    p->has_spec = true;
    if (p->d_spec_nat) {  // comparator spectrum must follow
        cudaFree(p->d_spec_nat);
        p->d_spec_nat = nullptr;
    }
    return PAC_OK;
}

extern "C" int pac_convolve(pac_plan p, const void* x_dev, void* y_dev, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = check_ptr(x_dev, "x_dev")) return rc;
    if (int rc = check_ptr(y_dev, "y_dev")) return rc;
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_filter_spectrum was not called for this plan");
    return run_convolve(p, x_dev, y_dev, static_cast<cudaStream_t>(stream));
}

extern "C" int pac_forward_unordered(pac_plan p, const void* x_dev, void* xhat_dev, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = df_unsupported(p, "pac_forward_unordered")) return rc;
    if (int rc = check_ptr(x_dev, "x_dev")) return rc;
    if (int rc = check_ptr(xhat_dev, "xhat_dev")) return rc;
    return run_forward(p, x_dev, xhat_dev, static_cast<cudaStream_t>(stream));
}

// Column blocks of the host-buffer call: the first pass (group 0, axis 0, a
// rows pass) reads and the last pass (its inverse) writes each column of
// the array independently, and column q of every row sits at q + g C, so a
// block of whole tiles' columns is one strided copy.  The copies of block
// k + 1 in (on one copy stream) and of block k - 1 out (on another) run while
// the passes work on block k.  Arrays under 64 MiB keep one copy each way:
// there the per-copy cost of 16 strided copies outweighed the overlap
// (128^3 FP32, 16 MiB: 228 -> 260 us per call).
constexpr int kHostBlocks = 8;
constexpr int64_t kHostBlockMinBytes = int64_t(64) << 20;

static bool host_pipelined(pac_plan p) {
    if (p->groups.size() < 2 || p->single_launch || p->bytes() < kHostBlockMinBytes) return false;
    const GroupPlan& g = p->groups[0];
    if (g.axis != 0 || g.C <= 1 || g.mix_nr > 0 || (p->plane && p->plane_g1 == 0)) return false;
    const int W = group_w(g, p->ces);
    return (g.Q + W - 1) / W >= 2 * kHostBlocks;
}

static int ensure_host_pipeline(pac_plan p) {
    cudaError_t e = cudaSuccess;
    if (!p->h2d) e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->d2h) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    while (e == cudaSuccess && p->chunk_ev.size() < 2 * kHostBlocks + 1) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) p->chunk_ev.push_back(ev);
    }
    return e == cudaSuccess ? PAC_OK : cuda_fail(e, "copy streams of the host-buffer call");
}

// One pass over tiles [t0, t0 + nt) of group g.
static int run_pass_tiles(pac_plan p, const GroupPlan& g, const Step& st, int64_t t0, int64_t nt, cudaStream_t s) {
    PassArgs a = make_pass(p, g, st.mode, st.src, st.dst, st.io);
    a.tile0 = t0;
    a.tiles = nt;
    cudaError_t e = launch_pass(p->esize, g.M, a, s);
    return e == cudaSuccess ? PAC_OK : cuda_fail(e, "pass kernel launch");
}

static int convolve_host_pipelined(pac_plan p, const void* x_host, void* y_host, cudaStream_t s) {
    if (int rc = ensure_host_pipeline(p)) return rc;
    const GroupPlan& g = p->groups[0];
    const int W = group_w(g, p->ces);
    const int64_t tiles = (g.Q + W - 1) / W, per = (tiles + kHostBlocks - 1) / kHostBlocks;
    const size_t S = (size_t)p->esize, pitch = (size_t)g.C * S;
    unsigned char* d = static_cast<unsigned char*>(p->d_stage);
    std::vector<Step> steps;
    convolve_steps(p, p->d_stage, p->d_stage, steps);
    cudaEvent_t* ev = p->chunk_ev.data();
    cudaError_t e = cudaEventRecord(ev[2 * kHostBlocks], s);  // the copies start after the caller's prior work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h2d, ev[2 * kHostBlocks], 0);
    if (e != cudaSuccess) return cuda_fail(e, "host-buffer call ordering");
    // blocks in: copy on h2d, then the first pass on those tiles on s
    for (int k = 0; k < kHostBlocks; ++k) {
        const int64_t t0 = k * per, t1 = std::min(tiles, t0 + per);
        if (t0 >= t1) break;
        const int64_t q0 = t0 * W, q1 = std::min<int64_t>(g.Q, t1 * W);
        e = cudaMemcpy2DAsync(d + q0 * S, pitch, static_cast<const unsigned char*>(x_host) + q0 * S, pitch,
                              (size_t)(q1 - q0) * S, (size_t)g.M, cudaMemcpyHostToDevice, p->h2d);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k], p->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "copy x to device");
        if (int rc = run_pass_tiles(p, g, steps.front(), t0, t1 - t0, s)) return rc;
    }
    // the middle passes on the whole array
    std::vector<Step> mid(steps.begin() + 1, steps.end() - 1);
    if (int rc = run_steps(p, mid, s, false)) return rc;
    // blocks out: the last pass on those tiles on s, then the copy on d2h
    for (int k = 0; k < kHostBlocks; ++k) {
        const int64_t t0 = k * per, t1 = std::min(tiles, t0 + per);
        if (t0 >= t1) break;
        const int64_t q0 = t0 * W, q1 = std::min<int64_t>(g.Q, t1 * W);
        if (int rc = run_pass_tiles(p, g, steps.back(), t0, t1 - t0, s)) return rc;
        e = cudaEventRecord(ev[kHostBlocks + k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, ev[kHostBlocks + k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(static_cast<unsigned char*>(y_host) + q0 * S, pitch, d + q0 * S, pitch,
                                  (size_t)(q1 - q0) * S, (size_t)g.M, cudaMemcpyDeviceToHost, p->d2h);
        if (e != cudaSuccess) return cuda_fail(e, "copy y to host");
    }
    e = cudaStreamSynchronize(p->d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAC_OK : cuda_fail(e, "pac_convolve_host");
}

extern "C" int pac_convolve_host(pac_plan p, const void* x_host, void* y_host, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (!x_host || !y_host) return fail(PAC_ERR_ARG, "null host pointer");
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_filter_spectrum was not called for this plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (!p->d_stage) {
            cudaError_t e = cudaMalloc(&p->d_stage, (size_t)p->bytes());
            if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "staging buffer: %s", cudaGetErrorString(e));
            p->device_bytes += (size_t)p->bytes();
        }
        if (host_pipelined(p)) return convolve_host_pipelined(p, x_host, y_host, s);
    }
    const size_t nb = (size_t)p->bytes();
    cudaError_t e = cudaMemcpyAsync(p->d_stage, x_host, nb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy x to device");
    int rc = run_convolve(p, p->d_stage, p->d_stage, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(y_host, p->d_stage, nb, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy y to host");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "pac_convolve_host");
    return PAC_OK;
}

// Per-axis [pos_to_freq | freq_to_pos] tables and an N-element scratch.
static int ensure_perm_tables(pac_plan p) {
    cudaError_t e;
    if (!p->d_perm) {
        int64_t tot = 0;
        for (int a = 0; a < p->ndim; ++a) tot += 2 * p->dims[a];
        std::vector<int64_t> h(tot);
        int64_t o = 0;
        for (int a = 0; a < p->ndim; ++a) {
            const int64_t n = p->dims[a];
            for (int64_t i = 0; i < n; ++i) {
                h[o + i] = p->pos_to_freq[a][i];
                h[o + n + p->pos_to_freq[a][i]] = i;
            }
            o += 2 * n;
        }
        e = cudaMalloc(&p->d_perm, tot * sizeof(int64_t));
        if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "permutation tables: %s", cudaGetErrorString(e));
        e = cudaMemcpy(p->d_perm, h.data(), tot * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "copy permutation tables");
        p->device_bytes += tot * sizeof(int64_t);
    }
    if (!p->d_scratch) {
        e = cudaMalloc(&p->d_scratch, (size_t)p->bytes());
        if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "scratch: %s", cudaGetErrorString(e));
        p->device_bytes += (size_t)p->bytes();
    }
    return PAC_OK;
}

// Comparator state: the tables and scratch above, and the natural-order
// spectrum (one permutation pass at filter time).
static int ensure_permuted_state(pac_plan p) {
    cudaError_t e;
    if (int rc = ensure_perm_tables(p)) return rc;
    if (!p->d_spec_nat) {
        e = cudaMalloc(&p->d_spec_nat, (size_t)p->bytes());
        if (e != cudaSuccess) return fail(PAC_ERR_NOMEM, "natural spectrum: %s", cudaGetErrorString(e));
        const int64_t* idx[3];
        int64_t o = 0;
        for (int a = 0; a < p->ndim; ++a) {
            idx[a] = p->d_perm + o + p->dims[a];  // natural k <- position of k
            o += 2 * p->dims[a];
        }
        const void* dif = p->d_spec;
        if (!p->groups.empty()) {  // back to the plain index-reversed order first
            e = launch_spec_order(p->esize, spec_order_of(p), p->N, p->d_spec, p->d_scratch, false, 0);
            if (e != cudaSuccess) return cuda_fail(e, "spectrum order kernel");
            dif = p->d_scratch;
        }
        e = launch_permute(p->esize, p->ndim, p->dims, idx, dif, p->d_spec_nat, nullptr, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "natural-order spectrum");
    }
    return PAC_OK;
}

extern "C" int pac_convolve_permuted(pac_plan p, const void* x_dev, void* y_dev, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = df_unsupported(p, "pac_convolve_permuted")) return rc;
    if (int rc = check_ptr(x_dev, "x_dev")) return rc;
    if (int rc = check_ptr(y_dev, "y_dev")) return rc;
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "pac_filter_spectrum was not called for this plan");
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (int rc = ensure_permuted_state(p)) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int G = (int)p->groups.size();
    // FFT2 = permute o uFFT2 (Algorithm 5): DIF passes, then reversed -> natural
    int rc = run_forward(p, x_dev, y_dev, s);
    if (rc) return rc;
    const int64_t* to_nat[3];
    const int64_t* to_rev[3];
    int64_t o = 0;
    for (int a = 0; a < p->ndim; ++a) {
        to_rev[a] = p->d_perm + o;                // position p <- frequency pos_to_freq[p]
        to_nat[a] = p->d_perm + o + p->dims[a];   // frequency k <- position of k
        o += 2 * p->dims[a];
    }
    // x := h o x in natural order, fused into the permutation
    cudaError_t e = timed_permute(p, to_nat, y_dev, p->d_scratch, p->d_spec_nat, s);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    // iFFT = uiFFT o permute (Algorithm 9)
    e = timed_permute(p, to_rev, p->d_scratch, y_dev, nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    std::vector<Step> steps;
    for (int i = G - 1; i >= 0; --i) steps.push_back({i, kInv, y_dev, y_dev});
    return run_steps(p, steps, s, true);
}

// Ordered transforms (Algorithm 5 FFT2 and Algorithm 9 iFFT): the DIF passes
// then the index-reversal permutation into natural frequency order, or the
// permutation (with 1/N) then the conjugate DIT passes.
static int ensure_perm_tables(pac_plan p);

extern "C" int pac_fft(pac_plan p, const void* in_dev, void* out_dev, int inverse, void* stream) {
    if (!p) return fail(PAC_ERR_ARG, "null plan");
    if (int rc = df_unsupported(p, "pac_fft")) return rc;
    if (int rc = check_ptr(in_dev, "in_dev")) return rc;
    if (int rc = check_ptr(out_dev, "out_dev")) return rc;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (int rc = ensure_perm_tables(p)) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t* to_nat[3];
    const int64_t* to_rev[3];
    int64_t o = 0;
    for (int a = 0; a < p->ndim; ++a) {
        to_rev[a] = p->d_perm + o;
        to_nat[a] = p->d_perm + o + p->dims[a];
        o += 2 * p->dims[a];
    }
    const int G = (int)p->groups.size();
    if (!inverse) {
        int rc = run_forward(p, in_dev, p->d_scratch, s);  // A^T x, index-reversed
        if (rc) return rc;
        cudaError_t e = timed_permute(p, to_nat, p->d_scratch, out_dev, nullptr, s);
        return e == cudaSuccess ? PAC_OK : cuda_fail(e, "permute kernel");
    }
    // x = conj(A) P X / N
    timer_mark(s, 3, true);
    cudaError_t e = launch_permute(p->esize, p->ndim, p->dims, to_rev, in_dev, p->d_scratch, nullptr, s,
                                   1.0 / (double)p->N);
    timer_mark(s, 3, false);
    if (e != cudaSuccess) return cuda_fail(e, "permute kernel");
    if (G == 0) {
        e = cudaMemcpyAsync(out_dev, p->d_scratch, (size_t)p->bytes(), cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? PAC_OK : cuda_fail(e, "copy");
    }
    std::vector<Step> steps;
    for (int i = G - 1; i >= 0; --i) steps.push_back({i, kInv, i == G - 1 ? (const void*)p->d_scratch : out_dev, out_dev});
    return run_steps(p, steps, s, false);
}

extern "C" int pac_convolve_timed(pac_plan p, int which, const void* x_dev, void* y_dev, void* stream,
                                  int max_launches, float* launch_ms, int* kernel_ids, int* n_launches) {
    if (!p || !launch_ms || !kernel_ids || !n_launches || max_launches < 1) return fail(PAC_ERR_ARG, "bad arguments");
    if (which < 0 || which > 3) return fail(PAC_ERR_ARG, "which must be 0, 1, 2 or 3");
    LaunchTimer timer;
    timer.max = max_launches;
    t_timer = &timer;
    int rc = which == 0   ? pac_convolve(p, x_dev, y_dev, stream)
             : which == 1 ? pac_convolve_permuted(p, x_dev, y_dev, stream)
                          : pac_fft(p, x_dev, y_dev, which == 3 ? 1 : 0, stream);
    t_timer = nullptr;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    const int n = (int)timer.ids.size();
    if (rc == PAC_OK && e == cudaSuccess && !timer.overflow && (int)timer.ev.size() == 2 * n) {
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, timer.ev[2 * i], timer.ev[2 * i + 1]);
            launch_ms[i] = ms;
            kernel_ids[i] = timer.ids[i];
        }
        *n_launches = n;
    }
    for (cudaEvent_t ev : timer.ev) cudaEventDestroy(ev);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "pac_convolve_timed");
    if (timer.overflow) return fail(PAC_ERR_ARG, "more than %d launches", max_launches);
    return PAC_OK;
}

extern "C" int pac_plan_stages(pac_plan p, int axis, int* radices, int* count) {
    if (!p || !count) return fail(PAC_ERR_ARG, "null argument");
    if (axis < 0 || axis >= p->ndim) return fail(PAC_ERR_ARG, "axis %d out of range", axis);
    const auto& st = p->stages[axis];
    if (radices) {
        if (*count < (int)st.size()) return fail(PAC_ERR_ARG, "radices array too small");
        std::copy(st.begin(), st.end(), radices);
    }
    *count = (int)st.size();
    return PAC_OK;
}

extern "C" int pac_plan_reverse_table(pac_plan p, int axis, int64_t* pos_to_freq) {
    if (!p || !pos_to_freq) return fail(PAC_ERR_ARG, "null argument");
    if (axis < 0 || axis >= p->ndim) return fail(PAC_ERR_ARG, "axis %d out of range", axis);
    std::copy(p->pos_to_freq[axis].begin(), p->pos_to_freq[axis].end(), pos_to_freq);
    return PAC_OK;
}

static bool single_ok(pac_plan p, int npasses) {
    return p->single_launch && npasses > 1 && npasses <= kMaxPasses && p->uniform_m > 0 && conv_grid(p->esize, p->uniform_m, p->device) > 0;
}

extern "C" int pac_plan_query(pac_plan p, int key, int64_t* value) {
    if (!p || !value) return fail(PAC_ERR_ARG, "null argument");
    const int64_t G = (int64_t)p->groups.size();
    switch (key) {
        case PAC_Q_NDIM: *value = p->ndim; break;
        case PAC_Q_N_TOTAL: *value = p->N; break;
        case PAC_Q_ELEM_BYTES: *value = p->esize; break;
        case PAC_Q_LAUNCHES_CONVOLVE: {
            std::vector<Step> st;
            convolve_steps(p, nullptr, nullptr, st);
            *value = G == 0 ? 1 : (!p->plane && single_ok(p, (int)st.size()) ? 1 : (int64_t)st.size());
            break;
        }
        case PAC_Q_LAUNCHES_PERMUTED:
            *value = (G == 0 ? 1 : (single_ok(p, G) ? 1 : G)) * 2 + 2;
            break;
        case PAC_Q_LAUNCHES_FORWARD: *value = G == 0 ? 1 : (single_ok(p, G) ? 1 : G); break;
        case PAC_Q_DEVICE_ERROR: {
            unsigned v = 0;
            if (int rc = take_device_error(p->device, &v)) return rc;
            *value = v;
            break;
        }
        case PAC_Q_DEVICE_BYTES: *value = (int64_t)p->device_bytes; break;
        case PAC_Q_HAS_SPECTRUM: *value = p->has_spec ? 1 : 0; break;
        case PAC_Q_GROUPS: *value = G; break;
        case PAC_Q_PLANE: *value = p->plane ? p->plane_k : 0; break;
        case PAC_Q_GROUP_CAP: *value = p->schedule.cap; break;
        case PAC_Q_NARROW: {
            int64_t k = 0;
            for (const GroupPlan& g : p->groups) k += g.nv;
            *value = k;
            break;
        }
        default: return fail(PAC_ERR_ARG, "unknown query key %d", key);
    }
    return PAC_OK;
}
