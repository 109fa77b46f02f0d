// Data layout of the batched query engine (device side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mhr_internal.cuh"
#include "mhr_mlp.cuh"

namespace mhr {

constexpr int kMidThreads = 1024;               // middle-join block (one per SM)
constexpr int kMidWarps = kMidThreads / 32;
constexpr int kMaxChunk = 32768;                // edges per work item, upper limit (<= 32 x threads)
constexpr int kDefaultChunk = 16384;
static_assert(kMaxChunk / 32 <= kMidThreads, "one 32-edge group per thread in the group map");
constexpr int kCandCap = 4096;                  // per-CTA fp32 candidate buffer
constexpr int kDenseLimit = kCandCap / 2;       // band denser than this -> exact path
constexpr int kMaxBmWords = 32768;              // shared-memory bitmap: 2^20 vertices
constexpr int kRankWords = 8;                   // one rank entry per 256 bitmap bits
constexpr int kMaxRank = kMaxBmWords / kRankWords;
constexpr int kDefaultTile = 4;                 // 32-edge groups in flight per warp (also 8)

// fp32 candidate: one path, identified by its hop-1 entry (index into the CSR
// row of s), its hop-3 entry (index into the reverse CSR row of t) and r2.
struct Cand {
    float s32;
    uint32_t a_idx;
    uint32_t c_idx;
    uint16_t r2;
    uint16_t pad;
};
static_assert(sizeof(Cand) == 16, "Cand is 16 bytes");

// middle edge joining a near-side entry to a far-side entry
struct Hit {
    uint32_t near_k;
    uint32_t far_k;
    uint32_t r2;  // relation id of the middle edge
};

// one distinct frontier vertex of a query
struct ListEnt {
    uint32_t vertex;
    uint32_t run_start;  // first entry in the hop-1 row of s (or hop-3 row of t)
    uint32_t run_len;    // number of parallel edges (relations) to this vertex
    float maxw;          // max fp32 weight over the run
    uint32_t deg;        // scan degree: out-degree (hop-1 side) / in-degree (hop-3 side)
    uint32_t rowstart;   // first CSR (or reverse CSR) position of that scan row
    float midw;          // bound of any middle-edge weight at this vertex: the largest fp32
                         // weight of its out-edges (hop-1 side) / in-edges (hop-3 side)
    uint32_t pad;
};
static_assert(sizeof(ListEnt) == 32, "ListEnt is 32 bytes");

enum {
    kCntItem = 0,
    kCntScanned = 1,
    kCntHits = 2,
    kCntCands = 3,
    kCntRescored = 4,
    kCntDense = 5,
    kCntPruned = 6,
    kCntPaths = 7,
    kCntSeed = 8,
    kCntSkippedItems = 9,
    kCntLabels = 10,
    kCntTcTimeouts = 11,  // ordering-MLP tiles whose tensor-core MMA gave up waiting
    kCntCount = 16
};

// Everything a batch needs, in device memory; kernels take a pointer to it so
// a captured CUDA graph keeps working when buffers are regrown between calls.
struct PlanDev {
    int32_t nq, K, chunk, sigma;
    int32_t nbw, pq, band_cap, score_width;  // score_width: lanes per edge in the expansion
    int32_t hit_width;                        // lanes per middle edge in the join's hit scorer
    int32_t grid, prune;  // persistent CTAs of the join; bound pruning on/off
    int32_t order, label;  // near-row order: 0 natural, 1 by bound, 2 by learned score; label dump on/off
    int32_t precision;     // 0 fp32 CUDA-core middle-edge screen, 1 bf16 tensor-core screen (DistMult)
    float prune_slack;     // added to every pruning bound when the middle edge comes from the tensor cores
    const uint16_t* wsplit;  // [2][R][d] bf16 hi / lo relation table
    // constrained query: flags [rel1: R][rel2: R][rel3: R][types of u: 256][types of v: 256]
    // (nonzero = allowed), or NULL when the call has no constraint
    const uint8_t* cons;
    int32_t part_count, part_index;  // vertex partition: hop-1 vertices u with u % count == index
    MlpDev mlp;            // order 2 weights
    int64_t nhist;        // nq * 256 order buckets
    int64_t item_cap;     // capacity of item_ub
    int64_t X;     // slots = totA + totC
    int64_t totA;  // slots of the hop-1 side
    double err_path;
    // per-call inputs
    const uint32_t* S;
    const uint32_t* T;
    const int64_t* a_off;  // [nq+1] hop-1 slot offsets (entries of row s)
    const int64_t* c_off;  // [nq+1] hop-3 slot offsets (entries of reverse row t)
    // slot arrays [X] (+1 for scans)
    float* w32;
    uint32_t* flag;
    int64_t* scan1;
    ListEnt* list;
    uint2* nearP;  // (prefix of scan degree within the query, row start)
    ListEnt* nearL;  // near entries in ordered position
    float* nearB;  // upper bound of the fp32 score of any path through a near entry
    // near-row ordering (slot arrays [X], scans [X+1])
    uint32_t* okey;     // order key of a near entry (natural position)
    uint32_t* orank;    // rank inside its bucket
    float* bnat;        // row bound in natural position
    uint32_t* nperm;    // ordered position -> dense index of the near entry
    uint32_t* degv3;    // scan degree in ordered position
    int64_t* scan4;     // prefix of degv3
    float* mlp_pred;    // order 2: predicted slack (<= 0) of each near entry's row bound
    uint32_t* ubest;    // label dump: key of the best fp32 path through a near entry (ordered position)
    double* w64s;       // fp64 weight of a hop-1 / hop-3 slot used by the band
    int32_t* w64own;    // 1 once a band entry has claimed the slot's fp64 sum
    uint32_t* qkey;     // [2 nq] min / max order key per query
    uint32_t* hist;     // [nq * 256] bucket counts
    int64_t* hscan;     // [nq * 256 + 1]
    uint32_t* item_ub;  // [item_cap] key of the largest row bound in a work item
    uint4* item_desc;   // [item_cap] (query | seeded << 31, near entry holding the item's first
                        //  edge, near entry holding its last edge, index of the item in its query)
    uint2* seed_k;      // [nq] near entries holding edge kSeedEdges - 1 and edge kSeedEdges
    float* mlp_qbias;   // [nq x 256] learned order: b1 + W1[:, 128:] e_end[0:128] per query
    // per query [nq] (+1 for item_off)
    int32_t* status;
    int32_t* dir;       // 1 = forward (scan out-rows of hop-1 vertices), 0 = backward
    int32_t* near_cnt;
    int32_t* far_cnt;
    int64_t* s_near;
    int64_t* item_off;
    int64_t* near_off;  // [nq+1] prefix of near_cnt (rows of the learned-order MLP)
    uint32_t* thr_g;    // order-preserving key of the best known K-th fp32 score
    uint32_t* qmax;     // [2 nq] keys: max hop-1 weight, max hop-3 weight
    unsigned long long* sdeg_q;  // [2 nq] S_f and S_b: scan degrees of the distinct frontier vertices
    int32_t* dense;
    int32_t* pool_cnt;
    int32_t* band_cnt;
    // buffers
    Hit* hits;          // [grid x kMaxChunk]
    Cand* pool;         // [nq x pq]
    Cand* band_cand;    // [nq x band_cap]
    double* band_w2;    // [nq x band_cap] fp64 weight of each band entry's middle edge
    uint32_t* chains;   // [nq x 3 band_cap] fp64 sums to run: kind << 30 | index
    int32_t* chain_cnt; // [nq]
    mhr_path* out;      // [nq x K]
    int32_t* n_out;     // [nq]
    unsigned long long* counters;  // kCntCount
    unsigned long long* cursors;   // [grid] next item of each CTA's own range
    uint32_t* drained;             // [(grid + 31) / 32] bit v: range v has no item left
    uint4* far_start;              // [grid x far_cap] coarse bitmap, indexed by the bit: its run in the far
                                   // list (first entry, its vertex, last vertex, its entry); set bits only
    int64_t far_cap;               // entries per CTA: the coarse bitmap's bits (coarse bitmaps only)
    int64_t* partials;             // scan scratch
};

}  // namespace mhr
