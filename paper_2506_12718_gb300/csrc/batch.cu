// Batched convolutions (pac_convolve_many).
//
// Every instance i runs the pass sequence of its plan (forward groups, the
// fused group, inverse groups: 2 G_i - 1 passes).  Passes are aligned by
// level: level l holds pass l of every instance that has one.  Within a
// level, the passes that share a kernel shape (element type, group size M,
// rows or lines; for plane passes both group sizes) run as ONE launch of
// pass_multi_kernel (plane_multi_kernel), which numbers the tiles (planes)
// of all its passes consecutively; launches of one level are
// independent and run as parallel branches, and each level waits for the one
// before.  A batch of any mix of shapes therefore costs a handful of
// launches.  The launch sequence of a distinct batch (same plans, same x and
// y pointers) is captured once into a CUDA graph and replayed on later calls;
// the graph's pass arguments live in one device buffer owned by the cache
// entry.  Destroying a plan drops every cached batch that uses it.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <tuple>

#include "pac_internal.h"
#include "persist.h"

namespace pac {
int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s);
int persist_grid(int dev, int smem);
cudaError_t launch_persist(const PersistArgs& A, int grid, int smem, cudaStream_t s);
}

using namespace pac;

namespace {

struct MultiLaunch {
    int esize, M;
    bool lines;
    int nv = 0;          // the narrow tile variant of the group
    int M2;              // > 0: a plane launch (groups M x M2), arguments are PlaneArgs
    int K;               // plane launch: CTAs per plane
    int n;               // passes in the launch
    size_t off_args;     // byte offset of its PassArgs[n] in the buffer
    size_t off_starts;   // byte offset of its uint32 tile starts [n + 1]
    int64_t tiles;       // total tiles
};

struct BatchEntry {
    std::vector<const void*> key;  // plans, x and y pointers
    int device = 0;
    bool persistent = false;       // the whole batch is one launch of the persistent kernel
    void* d_buf = nullptr;
    std::vector<std::vector<MultiLaunch>> levels;
    PersistArgs pargs = {};        // persistent form: arguments (in d_buf), grid, shared memory
    int pgrid = 0, psmem = 0;
    std::vector<int> pointwise;    // instances with N = 1 (no pass: a plain product)
    cudaGraphExec_t exec = nullptr;
};

// PAC_BATCH=graph in the environment keeps merged launches per level (a
// captured graph of several launches) even where the persistent kernel
// applies; PAC_BATCH=persistent (the default) uses the persistent kernel
// whenever every pass of the batch has a shape it carries.
bool persistent_wanted() {
    const char* v = std::getenv("PAC_BATCH");
    return !(v && std::strcmp(v, "graph") == 0);
}

// index in kPersistShapes of a step's shape (-1: the persistent kernel does not carry it)
int persist_shape_of(pac_plan p, const Step& st) {
    if (p->esize != 8) return -1;
    if (st.mode == kPlane) {
        if (p->plane_k != 1) return -1;
        const int m1 = p->groups[p->plane_g1].M, m2 = p->groups[p->plane_g1 + 1].M;
        for (int i = 0; i < kPersistShapeCount; ++i)
            if (kPersistShapes[i].m2 == m2 && kPersistShapes[i].m == m1) return i;
        return -1;
    }
    const GroupPlan& g = p->groups[st.group];
    if (g.mix_nr > 0) return -1;
    // a narrow tile of a forward or inverse pass is dropped (the kernel has its own tiles); the
    // fused pass' tile width fixes the layout of the stored spectrum, so a narrow one stays out
    if (g.nv && st.mode == kFused) return -1;
    const int lines = g.C == 1 ? 1 : 0;
    for (int i = 0; i < kPersistShapeCount; ++i)
        if (kPersistShapes[i].m2 == 0 && kPersistShapes[i].m == g.M && kPersistShapes[i].lines == lines) return i;
    return -1;
}

constexpr size_t kCacheEntries = 8;
std::mutex g_mu;
std::list<BatchEntry*> g_cache;  // most recently used first

void free_entry(BatchEntry* e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->d_buf) cudaFree(e->d_buf);
    delete e;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Kernel shape of a step: element size, group size, rows/lines (for a plane
// step: CTAs per plane; else bit 0 lines, bit 1 the narrow tile variant),
// and for a plane step the second group size.
using ShapeKey = std::tuple<int, int, int, int>;

ShapeKey shape_key(pac_plan p, const Step& st) {
    if (st.mode == kPlane)
        return ShapeKey(p->esize, p->groups[p->plane_g1].M, p->plane_k, p->groups[p->plane_g1 + 1].M);
    const GroupPlan& g = p->groups[st.group];
    return ShapeKey(p->esize, g.mix_nr > 0 ? -g.M : g.M, (g.C == 1 ? 1 : 0) | (g.nv ? 2 : 0), 0);  // -M: a mixed group
}

// Append one merged launch (arguments, then tile starts) to the host image.
int add_launch(std::vector<unsigned char>& blob, const ShapeKey& key, const void* args, size_t arg_size,
               const std::vector<int64_t>& tiles, std::vector<MultiLaunch>& out) {
    MultiLaunch m;
    int lines;
    std::tie(m.esize, m.M, lines, m.M2) = key;
    m.lines = m.M2 == 0 && (lines & 1) != 0;
    m.nv = m.M2 == 0 && (lines & 2) != 0 ? 1 : 0;
    m.K = m.M2 > 0 ? lines : 1;
    m.n = (int)tiles.size();
    m.off_args = align_up(blob.size(), 64);
    blob.resize(m.off_args + tiles.size() * arg_size);
    std::memcpy(blob.data() + m.off_args, args, tiles.size() * arg_size);
    m.off_starts = align_up(blob.size(), 16);
    blob.resize(m.off_starts + (tiles.size() + 1) * sizeof(uint32_t));
    uint32_t* st = reinterpret_cast<uint32_t*>(blob.data() + m.off_starts);
    int64_t acc = 0;
    for (size_t k = 0; k < tiles.size(); ++k) {
        st[k] = (uint32_t)acc;
        acc += tiles[k];
    }
    st[tiles.size()] = (uint32_t)acc;
    if (acc > 0x7fffffffLL) return fail(PAC_ERR_SIZE, "batch launch has too many tiles");
    m.tiles = acc;
    out.push_back(m);
    return PAC_OK;
}

// Build the merged launches of a batch and upload their arguments.
int build_entry(int count, const pac_plan* plans, const void* const* x, void* const* y, BatchEntry* e) {
    std::vector<std::vector<Step>> seq(count);
    size_t levels = 0;
    for (int i = 0; i < count; ++i) {
        if (plans[i]->groups.empty()) {
            e->pointwise.push_back(i);
            continue;
        }
        convolve_steps(plans[i], x[i], y[i], seq[i]);
        levels = std::max(levels, seq[i].size());
    }
    // level -> shape -> passes (plane steps keyed by both group sizes)
    std::vector<std::map<ShapeKey, std::vector<PassArgs>>> by_level(levels);
    std::vector<std::map<ShapeKey, std::vector<PlaneArgs>>> planes_by_level(levels);
    for (int i = 0; i < count; ++i) {
        for (size_t l = 0; l < seq[i].size(); ++l) {
            const Step& st = seq[i][l];
            const ShapeKey k = shape_key(plans[i], st);
            if (st.mode == kPlane)
                planes_by_level[l][k].push_back(make_plane(plans[i], st.src, st.dst));
            else
                by_level[l][k].push_back(make_pass(plans[i], plans[i]->groups[st.group], st.mode, st.src, st.dst));
        }
    }
    // one host image of every launch's arguments and tile starts
    std::vector<unsigned char> blob;
    e->levels.assign(levels, {});
    for (size_t l = 0; l < levels; ++l) {
        for (auto& kv : by_level[l]) {
            std::vector<int64_t> tiles;
            for (const PassArgs& a : kv.second) tiles.push_back(a.tiles);
            int rc = add_launch(blob, kv.first, kv.second.data(), sizeof(PassArgs), tiles, e->levels[l]);
            if (rc) return rc;
        }
        for (auto& kv : planes_by_level[l]) {
            std::vector<int64_t> tiles;
            for (const PlaneArgs& a : kv.second) tiles.push_back(a.planes);
            int rc = add_launch(blob, kv.first, kv.second.data(), sizeof(PlaneArgs), tiles, e->levels[l]);
            if (rc) return rc;
        }
    }
    if (!blob.empty()) {
        cudaError_t ce = cudaMalloc(&e->d_buf, blob.size());
        if (ce != cudaSuccess) return fail(PAC_ERR_NOMEM, "batch arguments: %s", cudaGetErrorString(ce));
        ce = cudaMemcpy(e->d_buf, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) return cuda_fail(ce, "copy batch arguments");
    }
    return PAC_OK;
}

// The persistent form of a batch: every pass of every instance as tiles of
// one launch of the persistent kernel.  Returns 1 when the batch does not
// qualify (an element type, group or plane the kernel does not carry, or an
// instance whose quarter-unit pass would precede a whole-CTA pass: the
// kernel runs all whole-CTA tiles before any quarter tile).
constexpr long long kPersistWaitCycles = 4000000000LL;  // about two seconds

int build_persistent(int count, const pac_plan* plans, const void* const* x, void* const* y, unsigned bias,
                     long long wait_cycles, BatchEntry* e) {
    struct Rec {
        PersistPass pp;
        int inst, level, tiles;
        bool quarter;
    };
    std::vector<Rec> recs;
    std::vector<std::vector<int>> of(count);  // per instance: its records in level order
    for (int i = 0; i < count; ++i) {
        if (plans[i]->groups.empty()) {  // N = 1: a plain product outside the launch
            e->pointwise.push_back(i);
            continue;
        }
        std::vector<Step> seq;
        convolve_steps(plans[i], x[i], y[i], seq);
        bool seen_quarter = false;
        for (size_t l = 0; l < seq.size(); ++l) {
            const Step& st = seq[l];
            const int sh = persist_shape_of(plans[i], st);
            if (sh < 0) return 1;
            Rec r = {};
            r.pp.shape = sh;
            r.inst = i;
            r.level = (int)l;
            r.quarter = persist_quarter(sh);
            if (!r.quarter && seen_quarter) return 1;
            seen_quarter = seen_quarter || r.quarter;
            if (st.mode == kPlane) {
                r.pp.pa = make_plane(plans[i], st.src, st.dst);
                r.tiles = (int)r.pp.pa.planes;
            } else {
                GroupPlan g = plans[i]->groups[st.group];
                g.nv = 0;  // the persistent kernel's tiles are the default ones
                r.pp.pa.a1 = make_pass(plans[i], g, st.mode, st.src, st.dst);
                r.tiles = (int)r.pp.pa.a1.tiles;
            }
            of[i].push_back((int)recs.size());
            recs.push_back(r);
        }
    }
    // order: whole-CTA passes by level, then quarter passes by level; within a level passes of one
    // shape together (units that take neighbouring tiles then run the same code), instances in order
    std::vector<int> order(recs.size());
    for (size_t k = 0; k < recs.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (recs[a].quarter != recs[b].quarter) return !recs[a].quarter;
        if (recs[a].level != recs[b].level) return recs[a].level < recs[b].level;
        return recs[a].pp.shape < recs[b].pp.shape;
    });
    std::vector<int> pos(recs.size());
    for (size_t k = 0; k < order.size(); ++k) pos[order[k]] = (int)k;
    const int npass = (int)order.size();
    int nfull = 0;
    int smem_full = 0;
    bool any_quarter = false;
    std::vector<PersistPass> passes(npass);
    std::vector<uint32_t> starts(npass + 1, 0);
    int64_t acc = 0;
    for (int k = 0; k < npass; ++k) {
        const Rec& r = recs[order[k]];
        PersistPass pp = r.pp;
        pp.dep = -1;
        pp.dep_tiles = 0;
        if (r.level > 0) {
            const int prev = of[r.inst][r.level - 1];
            pp.dep = pos[prev];
            pp.dep_tiles = (uint32_t)recs[prev].tiles;
        }
        passes[k] = pp;
        starts[k] = (uint32_t)acc;
        acc += r.tiles;
        if (acc > 0x7fffffffLL) return 1;
        if (!r.quarter) {
            nfull = k + 1;
            smem_full = std::max(smem_full, persist_smem(r.pp.shape));
        } else {
            any_quarter = true;
        }
    }
    starts[npass] = (uint32_t)acc;
    if (npass == 0) return 1;
    const int smem = std::max(smem_full, any_quarter ? kPersistUnits * kPersistQuarterSmem : 0);
    const int grid = persist_grid(e->device, smem);
    if (grid <= 0) return 1;
    // one device image: passes, tile starts, counters (zeroed; the kernel leaves them zeroed)
    const size_t off_starts = align_up((size_t)npass * sizeof(PersistPass), 64);
    const size_t off_pass_of = align_up(off_starts + (size_t)(npass + 1) * sizeof(uint32_t), 64);
    const size_t off_ctr = align_up(off_pass_of + (size_t)acc * sizeof(uint32_t), 128);
    const size_t bytes = off_ctr + (size_t)(3 + npass) * sizeof(unsigned);
    std::vector<unsigned char> blob(bytes, 0);
    std::memcpy(blob.data(), passes.data(), (size_t)npass * sizeof(PersistPass));
    std::memcpy(blob.data() + off_starts, starts.data(), (size_t)(npass + 1) * sizeof(uint32_t));
    uint32_t* po = reinterpret_cast<uint32_t*>(blob.data() + off_pass_of);  // tile -> pass, one load per tile
    for (int k = 0; k < npass; ++k)
        for (uint32_t g = starts[k]; g < starts[k + 1]; ++g) po[g] = (uint32_t)k;
    cudaError_t ce = cudaMalloc(&e->d_buf, bytes);
    if (ce != cudaSuccess) return fail(PAC_ERR_NOMEM, "batch arguments: %s", cudaGetErrorString(ce));
    ce = cudaMemcpy(e->d_buf, blob.data(), bytes, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "copy batch arguments");
    unsigned char* b = static_cast<unsigned char*>(e->d_buf);
    PersistArgs& A = e->pargs;
    A.passes = reinterpret_cast<const PersistPass*>(b);
    A.starts = reinterpret_cast<const uint32_t*>(b + off_starts);
    A.pass_of = reinterpret_cast<const uint32_t*>(b + off_pass_of);
    A.nfull = nfull;
    A.npass = npass;
    A.ctr = reinterpret_cast<unsigned*>(b + off_ctr);
    if (int rc = device_error_word(e->device, &A.error)) return rc;
    A.bias = bias;
    A.wait_cycles = wait_cycles;
    e->pgrid = grid;
    e->psmem = smem;
    e->persistent = true;
    return PAC_OK;
}

cudaError_t enqueue_launch(const BatchEntry* e, const MultiLaunch& m, cudaStream_t s) {
    const unsigned char* b = static_cast<const unsigned char*>(e->d_buf);
    const uint32_t* starts = reinterpret_cast<const uint32_t*>(b + m.off_starts);
    if (m.M2 > 0)
        return launch_plane_multi(m.esize, m.M, m.M2, m.K, reinterpret_cast<const PlaneArgs*>(b + m.off_args),
                                  starts, m.n, m.tiles, s);
    return launch_multi(m.esize, m.M, m.lines, m.nv, reinterpret_cast<const PassArgs*>(b + m.off_args), starts, m.n,
                        m.tiles, s);
}

// per-kernel set-up (shared-memory attribute, occupancy): a launch with no work
cudaError_t prepare_launch(const MultiLaunch& m, cudaStream_t s) {
    if (m.M2 > 0) return launch_plane_multi(m.esize, m.M, m.M2, m.K, nullptr, nullptr, 0, 0, s);
    return launch_multi(m.esize, m.M, m.lines, m.nv, nullptr, nullptr, 0, 0, s);
}

// Capture the batch's launches into a graph: the one persistent launch, or
// per level a fork over the level's launches (one stream each) and a join.
int capture(BatchEntry* e) {
    if (e->persistent) {
        cudaStream_t st = nullptr;
        cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        if (ce == cudaSuccess) ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            const cudaError_t le = launch_persist(e->pargs, e->pgrid, e->psmem, st);
            ce = cudaStreamEndCapture(st, &graph);
            if (le != cudaSuccess) ce = le;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st) cudaStreamDestroy(st);
        return ce == cudaSuccess ? PAC_OK : cuda_fail(ce, "batch graph capture");
    }
    size_t width = 1;
    for (const auto& lv : e->levels) width = std::max(width, lv.size());
    std::vector<cudaStream_t> st(width, nullptr);
    std::vector<cudaEvent_t> ev(width + 1, nullptr);
    int rc = PAC_OK;
    cudaError_t ce = cudaSuccess;
    for (size_t i = 0; i < width && ce == cudaSuccess; ++i) ce = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
    for (size_t i = 0; i <= width && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    // per-kernel set-up (shared-memory attribute, occupancy) happens outside the capture
    for (const auto& lv : e->levels)
        for (const MultiLaunch& m : lv)
            if (ce == cudaSuccess) ce = prepare_launch(m, st[0]);
    cudaGraph_t graph = nullptr;
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(st[0], cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (const auto& lv : e->levels) {
            if (le != cudaSuccess) break;
            if (lv.size() == 1) {
                le = enqueue_launch(e, lv[0], st[0]);
                continue;
            }
            le = cudaEventRecord(ev[width], st[0]);  // fork
            for (size_t k = 1; k < lv.size() && le == cudaSuccess; ++k) le = cudaStreamWaitEvent(st[k], ev[width], 0);
            for (size_t k = 0; k < lv.size() && le == cudaSuccess; ++k) le = enqueue_launch(e, lv[k], st[k]);
            for (size_t k = 1; k < lv.size() && le == cudaSuccess; ++k) {  // join
                le = cudaEventRecord(ev[k], st[k]);
                if (le == cudaSuccess) le = cudaStreamWaitEvent(st[0], ev[k], 0);
            }
        }
        ce = cudaStreamEndCapture(st[0], &graph);
        if (le != cudaSuccess) ce = le;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->exec, graph, 0);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "batch graph capture");
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    for (cudaStream_t x : st)
        if (x) cudaStreamDestroy(x);
    return rc;
}

}  // namespace

namespace pac {

void batch_forget_plan(pac_plan p) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        BatchEntry* e = *it;
        if (std::find(e->key.begin(), e->key.end(), static_cast<const void*>(p)) != e->key.end()) {
            free_entry(e);
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace pac

extern "C" int pac_convolve_many(int count, const pac_plan* plans, const void* const* x_dev, void* const* y_dev,
                                 void* stream) {
    if (count < 0 || (count > 0 && (!plans || !x_dev || !y_dev))) return fail(PAC_ERR_ARG, "bad arguments");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !x_dev[i] || !y_dev[i]) return fail(PAC_ERR_ARG, "null entry %d", i);
        if (reinterpret_cast<uintptr_t>(x_dev[i]) % 16 || reinterpret_cast<uintptr_t>(y_dev[i]) % 16)
            return fail(PAC_ERR_ARG, "instance %d: arrays must be 16-byte aligned", i);
        if (!plans[i]->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "instance %d: plan has no spectrum", i);
        if (plans[i]->device != dev) return fail(PAC_ERR_ARG, "instance %d: plan belongs to another device", i);
        if (int rc = df_unsupported(plans[i], "pac_convolve_many")) return rc;
    }
    if (count == 0) return PAC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<const void*> key;
    key.reserve(3 * (size_t)count + 1);
    for (int i = 0; i < count; ++i) {
        key.push_back(plans[i]);
        key.push_back(x_dev[i]);
        key.push_back(y_dev[i]);
    }
    key.push_back(reinterpret_cast<const void*>(uintptr_t(persistent_wanted() ? 1 : 2)));  // the batch form
    std::lock_guard<std::mutex> lk(g_mu);
    BatchEntry* e = nullptr;
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if ((*it)->device == dev && (*it)->key == key) {
            e = *it;
            g_cache.erase(it);
            break;
        }
    }
    if (!e) {
        e = new (std::nothrow) BatchEntry();
        if (!e) return fail(PAC_ERR_NOMEM, "host allocation failed");
        e->key = key;
        e->device = dev;
        int rc = 1;
        if (persistent_wanted()) {
            rc = build_persistent(count, plans, x_dev, y_dev, 0u, kPersistWaitCycles, e);
            if (rc == 1) e->pointwise.clear();  // not applicable: merged launches instead
        }
        if (rc == 1) rc = build_entry(count, plans, x_dev, y_dev, e);
        if (rc == PAC_OK) rc = capture(e);
        if (rc != PAC_OK) {
            free_entry(e);
            return rc;
        }
        while (g_cache.size() >= kCacheEntries) {
            free_entry(g_cache.back());
            g_cache.pop_back();
        }
    }
    g_cache.push_front(e);
    for (int i : e->pointwise) {  // N = 1 instances: a plain product, outside the graph
        int rc = run_convolve(plans[i], x_dev[i], y_dev[i], s);
        if (rc) return rc;
    }
    ce = cudaGraphLaunch(e->exec, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch graph launch");
    return PAC_OK;
}

// whether the persistent kernel carries every pass of the batch (host only; the
// same rules as build_persistent)
static bool persist_applies(int count, const pac_plan* plans) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
        if (plans[i]->groups.empty()) continue;
        std::vector<Step> seq;
        convolve_steps(plans[i], nullptr, nullptr, seq);
        bool seen_quarter = false;
        for (const Step& st : seq) {
            const int sh = persist_shape_of(plans[i], st);
            if (sh < 0) return false;
            if (!persist_quarter(sh) && seen_quarter) return false;
            seen_quarter = seen_quarter || persist_quarter(sh);
            any = true;
        }
    }
    return any;
}

extern "C" int pac_convolve_many_launches(int count, const pac_plan* plans, int* launches) {
    if (count < 0 || !launches || (count > 0 && !plans)) return fail(PAC_ERR_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(PAC_ERR_ARG, "null plan %d", i);
        if (int rc = df_unsupported(plans[i], "pac_convolve_many_launches")) return rc;
    }
    if (persistent_wanted() && persist_applies(count, plans)) {
        int n = 1;
        for (int i = 0; i < count; ++i) n += plans[i]->groups.empty() ? 1 : 0;
        *launches = n;
        return PAC_OK;
    }
    std::vector<std::map<ShapeKey, int>> by_level;
    int pointwise = 0;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(PAC_ERR_ARG, "null plan %d", i);
        if (plans[i]->groups.empty()) {
            ++pointwise;
            continue;
        }
        std::vector<Step> seq;
        convolve_steps(plans[i], nullptr, nullptr, seq);
        if (by_level.size() < seq.size()) by_level.resize(seq.size());
        for (size_t l = 0; l < seq.size(); ++l) by_level[l][shape_key(plans[i], seq[l])] += 1;
    }
    int n = pointwise;
    for (const auto& lv : by_level) n += (int)lv.size();
    *launches = n;
    return PAC_OK;
}


extern "C" int pac_test_batch_timeout(int count, const pac_plan* plans, const void* const* x_dev, void* const* y_dev,
                                      void* stream, int wait_us) {
    if (count < 1 || !plans || !x_dev || !y_dev) return fail(PAC_ERR_ARG, "bad arguments");
    if (wait_us < 1 || wait_us > 1000000) return fail(PAC_ERR_ARG, "wait_us %d not in [1, 10^6]", wait_us);
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !x_dev[i] || !y_dev[i]) return fail(PAC_ERR_ARG, "null entry %d", i);
        if (!plans[i]->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "instance %d: plan has no spectrum", i);
        if (int rc = df_unsupported(plans[i], "a batch")) return rc;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    BatchEntry e;
    e.device = dev;
    // every dependency target one tile beyond what its pass has: each dependent wait runs out
    int rc = build_persistent(count, plans, x_dev, y_dev, 1u, (long long)wait_us * 2070, &e);
    if (rc == 1) rc = fail(PAC_ERR_ARG, "the batch has no form of the persistent kernel");
    if (rc == PAC_OK) {
        bool dep = false;
        for (int i = 0; i < count; ++i) dep = dep || plans[i]->groups.size() > 1;
        if (!dep) rc = fail(PAC_ERR_ARG, "no instance of the batch has a pass that waits for another");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rc == PAC_OK) {
        ce = launch_persist(e.pargs, e.pgrid, e.psmem, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "persistent kernel");
    }
    if (e.d_buf) cudaFree(e.d_buf);
    return rc;
}
