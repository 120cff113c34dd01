// Arguments of one pass kernel launch (shared by host and device code).
#pragma once
#include <stdint.h>

namespace pac {

enum PassMode : int { kFwd = 0, kInv = 1, kFused = 2, kPlane = 3 };

// PassArgs::df bits of a double-float plan's passes: the pass runs the
// double-float kernels; its source / destination holds complex FP64 (the
// caller's arrays) instead of double-float pairs (the intermediate arrays).
enum : int { kDfKernel = 1, kDfSrc64 = 2, kDfDst64 = 4 };

// One pass over the array, viewed as [beta][m][c]: m in [0, M) is the group
// axis (row stride C elements); column q = beta * C + c, Q = N / M columns.
// Element (row g, column q) sits at (q - q mod C) * M + q mod C + g * C.
struct PassArgs {
    const void* src;
    void* dst;              // may equal src (in place)
    const void* spec;       // filter spectrum (kFused), same layout as the DIF output
    const void* tw_int;     // w_M^u, u in [0, M): round twiddles
    const void* tw_lo;      // w_L^u, u in [0, T)       (external factor, two-level)
    const void* tw_hi;      // w_L^{T v}, v in [0, ceil(L/T))
    const int* rowmap;      // [M] shared-memory row that holds global row g after the rounds
    const int* freq;        // [M] group frequency k' held by global row g
    const int* r2g;         // [M] global row of shared-memory row r (inverse of rowmap)
    const int* r2f;         // [M] group frequency k' of shared-memory row r
    int64_t Q;              // columns
    int64_t C;              // row stride in elements
    int64_t I;              // inner stride of the axis: column j = (q mod C) / I
    int64_t tiles;          // tiles of this launch: ceil(Q / W) for a whole pass
    int64_t tile0;          // first tile of this launch (0; > 0 when a pass runs in column blocks)
    int tw_T;               // two-level split of the external exponent e = hi * T + lo
    int tw_shift;           // log2(tw_T) when tw_T is a power of two, else -1
    int mode;               // PassMode
    int has_ext;            // apply w_L^{j k'} (L' > 1)
    int nv;                 // 1: the narrow tile variant of the group (has_narrow), 0: the default tile
    int df;                 // double-float plans: kDf* bits; 0 otherwise
    // mixed group (stages of several prime bases, the runtime-radix kernel):
    // mix_nr rounds of radices mix_r (0: a one-base group), group size mix_m,
    // tile width mix_w
    int mix_nr;
    int mix_m;
    int mix_w;
    int mix_r[8];
};

// A plane pass (the last two axes, one group each, whole planes in one CTA):
// a1 = the group of axis d-2 (rows of the plane), a2 = the group of axis d-1
// (lines of the plane); planes = N / (n1 n2).  a2.src / a2.dst are the
// pass' input and output, a1.spec the spectrum.
struct PlaneArgs {
    PassArgs a1, a2;
    int64_t planes;
};

// Storage order of a filter spectrum (see spec_slot in fft_device.cuh).
struct SpecOrder {
    uint32_t M;       // group size of the fused pass (plane: n1)
    uint32_t W;       // its tile width (plane: n2)
    uint32_t C;       // its row stride
    uint32_t R;       // radix of its last round (plane: of axis d-2's last round)
    uint32_t tasks;   // W * M / R
    const int* rowmap;  // [M] in-CTA row of global row g (plane: of axis d-2)
    uint32_t M2;        // plane order when > 0: n2
    const int* rowmap2; // plane: [n2] in-CTA row of axis d-1
    uint32_t K;         // plane: CTAs per plane (columns of axis d-1 split K ways)
};

// One step of a convolution as pac_test_host_steps lists it for the CPU
// emulation of the kernels: a pass (kind 0, the pass kernel of group size M,
// lines layout when lines != 0, the arguments a), the spectrum reorder
// (kind 1: dst[slot(e)] = src[e] * scale for e < n, the order o), or a plane
// pass with one CTA per plane (kind 2: planes of M x lines points, the
// arguments pa).
struct HostStep {
    int kind;
    int M;
    int lines;
    int64_t n;
    double scale;
    const void* src;
    void* dst;
    PassArgs a;
    SpecOrder o;
    PlaneArgs pa;
};

constexpr int kMaxPasses = 12;

// A whole convolution (or forward transform) as one cooperative launch:
// passes run as phases separated by grid-wide barriers.
struct ConvArgs {
    PassArgs pass[kMaxPasses];
    int npasses;
    unsigned* barrier;  // arrival counter (monotonic; never reset)
    unsigned base;      // its value when this launch starts
    unsigned* error;    // set to 1 if a barrier wait gave up
    unsigned target_bias;  // added to every barrier's target (0; > 0 only from the timeout test hook)
    unsigned spin_limit;   // polls before a wait gives up (0: kBarrierSpinLimit)
};

}  // namespace pac
