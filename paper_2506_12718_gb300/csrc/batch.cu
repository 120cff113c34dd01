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
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <tuple>

#include "pac_internal.h"

namespace pac {
int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s);
}

using namespace pac;

namespace {

struct MultiLaunch {
    int esize, M;
    bool lines;
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
    void* d_buf = nullptr;
    std::vector<std::vector<MultiLaunch>> levels;
    std::vector<int> pointwise;    // instances with N = 1 (no pass: a plain product)
    cudaGraphExec_t exec = nullptr;
};

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
// step: CTAs per plane), and for a plane step the second group size.
using ShapeKey = std::tuple<int, int, int, int>;

ShapeKey shape_key(pac_plan p, const Step& st) {
    if (st.mode == kPlane)
        return ShapeKey(p->esize, p->groups[p->plane_g1].M, p->plane_k, p->groups[p->plane_g1 + 1].M);
    const GroupPlan& g = p->groups[st.group];
    return ShapeKey(p->esize, g.mix_nr > 0 ? -g.M : g.M, g.C == 1 ? 1 : 0, 0);  // -M: a mixed group
}

// Append one merged launch (arguments, then tile starts) to the host image.
int add_launch(std::vector<unsigned char>& blob, const ShapeKey& key, const void* args, size_t arg_size,
               const std::vector<int64_t>& tiles, std::vector<MultiLaunch>& out) {
    MultiLaunch m;
    int lines;
    std::tie(m.esize, m.M, lines, m.M2) = key;
    m.lines = m.M2 == 0 && lines != 0;
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
                by_level[l][k].push_back(make_pass(plans[i], plans[i]->groups[st.group], st.mode, st.src, st.dst,
                                                   st.scale));
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

cudaError_t enqueue_launch(const BatchEntry* e, const MultiLaunch& m, cudaStream_t s) {
    const unsigned char* b = static_cast<const unsigned char*>(e->d_buf);
    const uint32_t* starts = reinterpret_cast<const uint32_t*>(b + m.off_starts);
    if (m.M2 > 0)
        return launch_plane_multi(m.esize, m.M, m.M2, m.K, reinterpret_cast<const PlaneArgs*>(b + m.off_args),
                                  starts, m.n, m.tiles, s);
    return launch_multi(m.esize, m.M, m.lines, reinterpret_cast<const PassArgs*>(b + m.off_args), starts, m.n,
                        m.tiles, s);
}

// per-kernel set-up (shared-memory attribute, occupancy): a launch with no work
cudaError_t prepare_launch(const MultiLaunch& m, cudaStream_t s) {
    if (m.M2 > 0) return launch_plane_multi(m.esize, m.M, m.M2, m.K, nullptr, nullptr, 0, 0, s);
    return launch_multi(m.esize, m.M, m.lines, nullptr, nullptr, 0, 0, s);
}

// Capture the batch's launches into a graph: per level a fork over the
// level's launches (one stream each) and a join.
int capture(BatchEntry* e) {
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
    }
    if (count == 0) return PAC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<const void*> key;
    key.reserve(3 * (size_t)count);
    for (int i = 0; i < count; ++i) {
        key.push_back(plans[i]);
        key.push_back(x_dev[i]);
        key.push_back(y_dev[i]);
    }
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
        int rc = build_entry(count, plans, x_dev, y_dev, e);
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

extern "C" int pac_convolve_many_launches(int count, const pac_plan* plans, int* launches) {
    if (count < 0 || !launches || (count > 0 && !plans)) return fail(PAC_ERR_ARG, "bad arguments");
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

