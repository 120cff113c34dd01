// Shapes and arguments of the persistent batched kernel (kern_persist.cu),
// shared by the host code that builds a batch (batch.cu) and the kernel.
#pragma once
#include <stdint.h>

#include "config.h"
#include "pass_args.h"

namespace pac {

// A CTA of the persistent kernel has kPersistThreads threads.  Items whose
// tile or plane fits a unit's share of the shared memory run in units
// (kPersistUnits independent units of kPersistUnit threads per CTA, each on
// its own item; "quarter" below for short); larger ones run on the whole
// CTA.
constexpr int kPersistThreads = 1024;
constexpr int kPersistUnit = 256;
constexpr int kPersistUnits = kPersistThreads / kPersistUnit;
// shared memory of one unit: an equal share of what one CTA may take (less 4 KB for the
// kernel's own variables), in whole 128-byte lines
constexpr int kPersistQuarterSmem = ((227 * 1024 - 4096) / kPersistUnits) / 128 * 128;
// units of 256 threads match the pass kernels' own CTAs; smaller units load several tasks at once
constexpr bool kPersistPrefetch = kPersistUnit < 256;

// One shape the kernel carries: a one-base group pass of size m (rows or
// lines) or, with m2 > 0, a plane pass of m x m2 (K = 1).  Complex FP32.
struct PersistShape {
    int m, lines, m2;
};
constexpr PersistShape kPersistShapes[] = {
    {2, 0, 0},    {2, 1, 0},    {4, 0, 0},    {4, 1, 0},     {8, 0, 0},     {8, 1, 0},     {16, 0, 0},
    {16, 1, 0},   {32, 0, 0},   {32, 1, 0},   {64, 0, 0},    {64, 1, 0},    {128, 0, 0},   {128, 1, 0},
    {256, 0, 0},  {256, 1, 0},  {512, 0, 0},  {512, 1, 0},   {1024, 0, 0},  {1024, 1, 0},  {2048, 0, 0},
    {2048, 1, 0}, {4096, 0, 0}, {4096, 1, 0}, {3, 0, 0},     {3, 1, 0},     {9, 0, 0},     {9, 1, 0},
    {27, 0, 0},   {27, 1, 0},   {81, 0, 0},   {81, 1, 0},    {243, 0, 0},   {243, 1, 0},   {729, 0, 0},
    {729, 1, 0},  {2187, 0, 0}, {2187, 1, 0}, {5, 0, 0},     {5, 1, 0},     {25, 0, 0},    {25, 1, 0},
    {125, 0, 0},  {125, 1, 0},  {625, 0, 0},  {625, 1, 0},   {3125, 0, 0},  {3125, 1, 0},  {16, 0, 16},
    {32, 0, 32},  {64, 0, 64},  {128, 0, 128}, {27, 0, 27},  {81, 0, 81},   {25, 0, 25},   {125, 0, 125}};
constexpr int kPersistShapeCount = (int)(sizeof(kPersistShapes) / sizeof(kPersistShapes[0]));

// shared-memory bytes of one item of shape i (complex FP32)
constexpr int persist_smem(int i) {
    return kPersistShapes[i].m2 > 0 ? plane_smem_bytes(kPersistShapes[i].m, kPersistShapes[i].m2, 8)
                                    : tile_elems(kPersistShapes[i].m, 8, kPersistShapes[i].lines != 0) * 8;
}
// true: the shape runs in quarter units, false: on the whole CTA
constexpr bool persist_quarter(int i) { return persist_smem(i) <= kPersistQuarterSmem; }

// One pass of one instance.
struct alignas(16) PersistPass {
    PlaneArgs pa;        // a plane pass uses all of it; a group pass uses pa.a1
    int shape;           // index into kPersistShapes
    int dep;             // the pass whose tiles must all be done first (-1: none)
    uint32_t dep_tiles;  // its tile count
};

// Kernel arguments.  Passes [0, nfull) run on whole CTAs, passes
// [nfull, npass) in quarter units; within each class the passes are in
// level order, so every pass' dependency has a smaller index.
struct PersistArgs {
    const PersistPass* passes;
    const uint32_t* starts;  // [npass + 1]: first global tile of each pass (full tiles, then quarter tiles)
    const uint32_t* pass_of; // [starts[npass]]: the pass of each global tile
    int nfull, npass;
    unsigned* ctr;           // [0] next full tile, [1] next quarter tile, [2] CTAs done, [3 + p] tiles done of pass p
    unsigned* error;         // device error word: 1 when a dependency wait gave up
    unsigned bias;           // added to every dependency target (0; > 0 only from the timeout test hook)
    long long wait_cycles;   // cycles before a dependency wait gives up
};

}  // namespace pac
