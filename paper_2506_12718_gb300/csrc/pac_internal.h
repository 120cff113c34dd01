// Internal declarations of the pac library (host side).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pac.h"
#include "config.h"
#include "pass_args.h"

namespace pac {

// One group of consecutive DIF stages of one axis, executed by one pass.
struct GroupPlan {
    int axis = 0;
    int M = 1;              // product of the group's stage radices
    int first_stage = 0;    // index into the axis' stage list
    int nstages = 0;
    int64_t L = 1;          // block length (axis units) at the group's start
    int64_t Lp = 1;         // L / M
    int64_t C = 1;          // row stride in elements = Lp * I
    int64_t I = 1;          // product of the dims after the axis
    int64_t Q = 1;          // columns = N / M
    int tw_T = 1, tw_shift = 0;
    bool has_ext = false;
    int mix_nr = 0;         // > 0: a mixed group (several prime bases), rounds mix_r of the runtime-radix kernel
    int nv = 0;             // 1: the narrow tile variant (has_narrow in config.h)
    int mix_r[kMixMaxRounds] = {0};
    size_t off_twi = 0, off_lo = 0, off_hi = 0, off_rowmap = 0, off_freq = 0, off_r2g = 0, off_r2f = 0;  // in tables
};

// tile width of a group's pass
inline int group_w(const GroupPlan& g, int esize) {
    return g.mix_nr > 0 ? mix_w(g.M, esize) : tile_w(g.M, esize, g.nv);
}

// A pass schedule: the largest group exponent per pass (0: the largest a CTA
// takes) and whether the last two axes may run as a plane pass.
struct Schedule {
    int cap = 0;
    bool plane = true;
    // stage lists of several prime bases: 1 groups may span bases, 0 they may not,
    // -1 (the default) they do when every group spanning bases has a compiled kernel
    int mixed = -1;
    bool mix_runtime = false;  // groups spanning bases always in the runtime-radix kernel
    // the plane pass' tile: CTAs per plane (1: a whole plane per CTA, K > 1: split over a
    // K-CTA cluster); 0: the rule of plane_cluster
    int plane_k = 0;
    // 1: the passes' tiles take the narrow variant (half the columns) where the group has one
    int nv = 0;
};
int plan_build(int ndim, const int64_t* dims, int radix, pac_dtype dtype, const Schedule& sch, pac_plan* out);
// the same from explicit per-axis DIF stage lists (radix: the label the plan reports; -1 = explicit)
int plan_build_stages(int ndim, const int64_t* dims, const std::vector<std::vector<int>>& stages, int radix,
                      pac_dtype dtype, const Schedule& sch, pac_plan* out);
// the tuned schedule for a problem, if pac_tune (or the tuning file) has one (tune.cu)
bool tuned_schedule(int ndim, const int64_t* dims, int radix, pac_dtype dtype, Schedule* out);

void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// exp(-2 pi i e / L) in FP64 with the angle reduced exactly to an eighth turn
void root_fp64(int64_t e, int64_t L, double* re, double* im);

// kernel launchers (kern_dispatch.cu)
cudaError_t launch_pass(int esize, int M, const PassArgs& a, cudaStream_t s);
int conv_grid(int esize, int M, int dev);  // co-resident CTAs of the single-launch kernel (0: unavailable)
cudaError_t launch_conv(int esize, int M, ConvArgs& args, int grid, cudaStream_t s);
int pass_kernel_supported(int M, int esize);
// plane pass (kern_plane.cu): whole planes of the last two axes in one CTA
int plane_supported(int M1, int M2, int esize);
int plane_supported_k(int M1, int M2, int esize, int K);
int plane_cluster(int M1, int M2, int esize, int64_t planes, int device);  // CTAs per plane (0: none)
cudaError_t launch_plane(int esize, int M1, int M2, int K, const PlaneArgs& pa, cudaStream_t s);
cudaError_t launch_plane_multi(int esize, int M1, int M2, int K, const PlaneArgs* list, const uint32_t* starts, int n,
                               int64_t total, cudaStream_t s);
PlaneArgs make_plane(pac_plan p, const void* src, void* dst);

// n passes of one shape in one launch; list and starts in device memory (starts has n + 1 entries)
cudaError_t launch_multi(int esize, int M, bool lines, int nv, const PassArgs* list, const uint32_t* starts, int n,
                         int64_t total, cudaStream_t s);

// pass sequence of a convolution (plan.cu): group, mode, source, destination, scale
struct Step {
    int group, mode;
    const void* src;
    void* dst;
    int io = 0;  // double-float plans: kDfSrc64 / kDfDst64 (the caller's FP64 arrays)
};
void convolve_steps(pac_plan p, const void* x, void* y, std::vector<Step>& out);
PassArgs make_pass(pac_plan p, const GroupPlan& g, int mode, const void* src, void* dst, int io = 0);
int run_pass(pac_plan p, const GroupPlan& g, int mode, const void* src, void* dst, cudaStream_t s, int io = 0);
// PAC_ERR_ARG for an entry point that does not take double-float plans (PAC_OK otherwise)
int df_unsupported(pac_plan p, const char* what);
// forget every cached batch that uses plan p (batch.cu); called by pac_plan_destroy
void batch_forget_plan(pac_plan p);

// Barrier counters of single-launch convolutions: a device pool of slots,
// handed out round robin; *base receives the slot's counter value at launch.
int barrier_slot(int device, unsigned** counter, unsigned* base, unsigned arrivals, unsigned** error);
// The library's device error word (created with the barrier pool), for kernels that report a wait that gave up.
int device_error_word(int device, unsigned** error);
// Device error word of the library (barrier timeouts); returns and clears it.
int take_device_error(int device, unsigned* value);

// auxiliary kernels (aux.cu)
cudaError_t launch_permute(int esize, int ndim, const int64_t* dims, const int64_t* const* idx_dev,
                           const void* src, void* dst, const void* mul, cudaStream_t s, double scale = 1.0);
// to_kernel: dst[slot(e)] = src[e] * scale; else dst[e] = src[slot(e)] * scale
// double-float spectra (df): 16-byte elements of two double-float parts, the scale applied in double-float
cudaError_t launch_spec_order_df(const SpecOrder& o, int64_t n, const void* src, void* dst, cudaStream_t s,
                                 double scale);
cudaError_t launch_spec_order(int esize, const SpecOrder& o, int64_t n, const void* src, void* dst, bool to_kernel,
                              cudaStream_t s, double scale = 1.0);
cudaError_t launch_pointwise_mul(int esize, int64_t n, const void* a, const void* b, void* out, double scale,
                                 cudaStream_t s);

int device_sm_count(int device);

// storage order of a plan's filter spectrum (plan.cu); the plan needs a group
SpecOrder spec_order_of(pac_plan p);

}  // namespace pac

struct pac_plan_s {
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    int radix = 2;
    pac_dtype dtype = PAC_C64;
    int esize = 8;
    bool df = false;  // PAC_C128_DF: double-float passes (kDf* bits in PassArgs::df)
    int ces = 8;      // key of the tiling rules (config.h): esize, or kEsDf for double-float plans
    int64_t N = 1;
    int uniform_m = 0;  // group size shared by every pass (0: sizes differ)
    bool plane = false;  // the last two axes run as one plane pass (groups plane_g1, plane_g1 + 1)
    int plane_g1 = -1;
    int plane_k = 1;     // CTAs (a thread-block cluster) per plane
    pac::Schedule schedule;
    bool single_launch = false;  // run a pass sequence as one cooperative launch
    int device = 0;
    std::vector<std::vector<int>> stages;          // per axis, DIF order
    std::vector<std::vector<int64_t>> pos_to_freq; // per axis
    std::vector<pac::GroupPlan> groups;            // forward order
    void* d_tables = nullptr;
    size_t tables_bytes = 0;
    void* d_spec = nullptr;       // A^T h / N, in the fused pass' storage order (SpecOrder)
    int64_t spec_elems = 0;       // slots of d_spec (>= N: whole tiles of the fused pass)
    bool has_spec = false;
    // comparator (permuted form) state, created on first use
    void* d_spec_nat = nullptr;   // DFT(h) / N in natural order
    void* d_scratch = nullptr;    // N elements
    int64_t* d_perm = nullptr;    // per axis: [pos_to_freq | freq_to_pos], 2 * dims[a] each
    // host-buffer convolution staging, created on first use
    void* d_stage = nullptr;      // N elements
    cudaStream_t h2d = nullptr, d2h = nullptr;  // copy streams of the pipelined host-buffer call
    std::vector<cudaEvent_t> chunk_ev;          // its events (2 per column block)
    std::mutex mu;
    size_t device_bytes = 0;

    int64_t bytes() const { return N * esize; }
};
