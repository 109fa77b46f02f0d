// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/mhr.h"

namespace mhr {

// ---------------------------------------------------------------------------
// error plumbing: every failure becomes a status plus a thread-local message
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
mhr_status fail(mhr_status st, const std::string& msg);
mhr_status cuda_fail(cudaError_t e, const char* what);

#define MHR_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t e__ = (expr);                                 \
        if (e__ != cudaSuccess) return ::mhr::cuda_fail(e__, #expr); \
    } while (0)

#define MHR_TRY(expr)                      \
    do {                                   \
        mhr_status s__ = (expr);           \
        if (s__ != MHR_OK) return s__;     \
    } while (0)

// ---------------------------------------------------------------------------
// device view of a loaded graph (POD, passed by value to kernels)
// ---------------------------------------------------------------------------
struct DevGraph {
    int64_t n, E;
    int32_t R, d, dtype, fn;
    double gamma;
    float gamma32;
    float pad0;
    const int64_t* off;    // CSR by source: row starts [n+1]
    const uint32_t* col;   // destinations [E]
    const uint16_t* rel;   // relation ids [E]
    const int64_t* roff;   // CSR by destination: row starts [n+1]
    const uint32_t* rcol;  // sources, rows sorted by (source, relation) [E]
    const uint16_t* rrel;  // relation ids [E]
    const uint8_t* vtypes;
    const void* vemb;      // [n x d] f32 or bf16
    const void* remb;      // [R x d]
    // upper bounds (fp32, rounded up, any summation order) of the fp32 edge
    // weight over the out-edges / in-edges of each vertex; -inf if none
    const float* maxw_out;
    const float* maxw_in;
    // the same per (vertex, relation): [n x R], entry v * R + r; NULL when
    // n x R exceeds kMaxRelBoundEntries
    const float* maxw_out_r;
    const float* maxw_in_r;
};

constexpr int64_t kMaxRelBoundEntries = int64_t(1) << 29;  // 2 GiB per table

// device allocation owned by the graph
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct PlanCache;  // batched-query plans, defined in mhr_query.cu
struct TailCache;  // tail-prediction candidate lists and scratch, defined in mhr_tail.cu

}  // namespace mhr

// the opaque handle
struct mhr_graph {
    mhr::DevGraph dg;
    int device = 0;
    mhr_score_fn fn = MHR_SCORE_TRANSE_L1;
    // device storage
    std::vector<void*> allocations;
    size_t alloc_bytes = 0;  // device bytes held in `allocations`
    size_t memory_cap = 0;   // MHR_GRAPH_MEMORY_CAP_BYTES at load (0 = none)
    // host copies of the row starts (query sizing)
    std::vector<int64_t> h_off, h_roff;
    int64_t max_out_deg = 0, max_in_deg = 0;
    // fp32 screening error bounds (see mhr_graph.cu)
    double eps32_edge = 0, eps64_edge = 0, err_path = 0;
    // tensor-core screen of the middle edge (DistMult, bf16 hi/lo split):
    // per-edge bound and the path bound when w2 comes from it
    double epstc_edge = 0, err_path_tc = 0;
    uint16_t* wsplit = nullptr;  // [2][R][d] bf16 hi / lo parts of the relation table
    double max_l1 = 0, max_rel_l1 = 0, max_rel_inf = 0, max_l2sq = 0;
    int num_sms = 0;
    mhr::PlanCache* plans = nullptr;
    mhr::TailCache* tail = nullptr;
};

namespace mhr {

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_to_f32(uint16_t b) {
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

__device__ __forceinline__ float emb_f32(const void* tab, int dtype, int64_t row, int d, int j) {
    if (dtype == MHR_F32) return static_cast<const float*>(tab)[row * d + j];
    return bf16_to_f32(static_cast<const uint16_t*>(tab)[row * d + j]);
}

// order-preserving map float -> uint32 (larger float -> larger key)
__device__ __forceinline__ uint32_t f2key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// Edge weight in fp32: the screening arithmetic.  `lane`/`width` split the
// embedding dimension over a group of `width` lanes (a power of two <= 32,
// aligned inside the warp); every lane of the group returns the full value.
// Summation order is unspecified; the error bound in mhr_graph.cu holds for
// any order and with or without fused multiply-add.
__device__ __forceinline__ float edge_w32_group(const DevGraph& g, uint32_t u, uint32_t r,
                                                uint32_t v, int lane, int width) {
    float acc = 0.f;
    const int d = g.d;
    if (g.dtype == MHR_F32) {
        const float* eu = static_cast<const float*>(g.vemb) + static_cast<int64_t>(u) * d;
        const float* wr = static_cast<const float*>(g.remb) + static_cast<int64_t>(r) * d;
        const float* ev = static_cast<const float*>(g.vemb) + static_cast<int64_t>(v) * d;
        if ((d & 3) == 0) {
            const float4* eu4 = reinterpret_cast<const float4*>(eu);
            const float4* wr4 = reinterpret_cast<const float4*>(wr);
            const float4* ev4 = reinterpret_cast<const float4*>(ev);
            for (int j = lane; j < (d >> 2); j += width) {
                float4 a = __ldg(eu4 + j), b = __ldg(wr4 + j), c = __ldg(ev4 + j);
                if (g.fn == MHR_SCORE_TRANSE_L1) {
                    acc += fabsf(__fsub_rn(__fadd_rn(a.x, b.x), c.x));
                    acc += fabsf(__fsub_rn(__fadd_rn(a.y, b.y), c.y));
                    acc += fabsf(__fsub_rn(__fadd_rn(a.z, b.z), c.z));
                    acc += fabsf(__fsub_rn(__fadd_rn(a.w, b.w), c.w));
                } else {
                    acc += (a.x * b.x) * c.x;
                    acc += (a.y * b.y) * c.y;
                    acc += (a.z * b.z) * c.z;
                    acc += (a.w * b.w) * c.w;
                }
            }
        } else {
            for (int j = lane; j < d; j += width) {
                float a = __ldg(eu + j), b = __ldg(wr + j), c = __ldg(ev + j);
                if (g.fn == MHR_SCORE_TRANSE_L1) acc += fabsf(__fsub_rn(__fadd_rn(a, b), c));
                else acc += (a * b) * c;
            }
        }
    } else {
        const uint16_t* eu = static_cast<const uint16_t*>(g.vemb) + static_cast<int64_t>(u) * d;
        const uint16_t* wr = static_cast<const uint16_t*>(g.remb) + static_cast<int64_t>(r) * d;
        const uint16_t* ev = static_cast<const uint16_t*>(g.vemb) + static_cast<int64_t>(v) * d;
        if ((d & 7) == 0) {
            const uint4* eu8 = reinterpret_cast<const uint4*>(eu);
            const uint4* wr8 = reinterpret_cast<const uint4*>(wr);
            const uint4* ev8 = reinterpret_cast<const uint4*>(ev);
            for (int j = lane; j < (d >> 3); j += width) {
                uint4 A = __ldg(eu8 + j), B = __ldg(wr8 + j), C = __ldg(ev8 + j);
                const uint32_t aw[4] = {A.x, A.y, A.z, A.w};
                const uint32_t bw[4] = {B.x, B.y, B.z, B.w};
                const uint32_t cw[4] = {C.x, C.y, C.z, C.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float a0 = __uint_as_float(aw[k] << 16), a1 = __uint_as_float(aw[k] & 0xffff0000u);
                    float b0 = __uint_as_float(bw[k] << 16), b1 = __uint_as_float(bw[k] & 0xffff0000u);
                    float c0 = __uint_as_float(cw[k] << 16), c1 = __uint_as_float(cw[k] & 0xffff0000u);
                    if (g.fn == MHR_SCORE_TRANSE_L1) {
                        acc += fabsf(__fsub_rn(__fadd_rn(a0, b0), c0));
                        acc += fabsf(__fsub_rn(__fadd_rn(a1, b1), c1));
                    } else {
                        acc += (a0 * b0) * c0;
                        acc += (a1 * b1) * c1;
                    }
                }
            }
        } else {
            for (int j = lane; j < d; j += width) {
                float a = bf16_to_f32(eu[j]), b = bf16_to_f32(wr[j]), c = bf16_to_f32(ev[j]);
                if (g.fn == MHR_SCORE_TRANSE_L1) acc += fabsf(__fsub_rn(__fadd_rn(a, b), c));
                else acc += (a * b) * c;
            }
        }
    }
    for (int o = width >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, width);
    if (g.fn == MHR_SCORE_TRANSE_L1) return __fsub_rn(g.gamma32, acc);
    return acc;
}

// bf16 halves of a 32-bit word widened to fp32, and one TransE-L1 / DistMult term
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ float term_tr(float a, float b, float c, bool transe) {
    return transe ? fabsf(__fsub_rn(__fadd_rn(a, b), c)) : (a * b) * c;
}

// Edge weight in fp64, canonical order: j = 0..d-1 sequentially, explicit
// round-to-nearest adds and multiplies (never fused).  This is the exact
// arithmetic of the CPU reference definition, so results are bit-identical.
__device__ __forceinline__ double emb_f64(const void* tab, int dtype, int64_t row, int d, int j) {
    return static_cast<double>(emb_f32(tab, dtype, row, d, j));
}

static __device__ __noinline__ double edge_w64(const DevGraph& g, uint32_t u, uint32_t r, uint32_t v) {
    double acc = 0.0;
    const int d = g.d;
    if (g.fn == MHR_SCORE_TRANSE_L1) {
        for (int j = 0; j < d; ++j) {
            double a = emb_f64(g.vemb, g.dtype, u, d, j);
            double b = emb_f64(g.remb, g.dtype, r, d, j);
            double c = emb_f64(g.vemb, g.dtype, v, d, j);
            acc = __dadd_rn(acc, fabs(__dsub_rn(__dadd_rn(a, b), c)));
        }
        return __dsub_rn(g.gamma, acc);
    }
    for (int j = 0; j < d; ++j) {
        double a = emb_f64(g.vemb, g.dtype, u, d, j);
        double b = emb_f64(g.remb, g.dtype, r, d, j);
        double c = emb_f64(g.vemb, g.dtype, v, d, j);
        acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(a, b), c));
    }
    return acc;
}

// smallest group width (power of two <= 32) that covers one vector step of d
__host__ __device__ inline int score_group_width(int d, int dtype) {
    int vec = (dtype == MHR_F32) ? ((d & 3) == 0 ? d / 4 : d) : ((d & 7) == 0 ? d / 8 : d);
    int w = 1;
    while (w < vec && w < 32) w <<= 1;
    return w;
}

// host helpers
int device_sm_count();
mhr_status check_graph(const mhr_graph* g);

}  // namespace mhr
