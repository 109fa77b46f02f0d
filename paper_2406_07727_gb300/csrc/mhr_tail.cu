// Tail prediction (Alg. 3, Alg. 4): for a head h and a relation r, score every
// candidate vertex c of one type with the edge weight w(h, r, c) and keep the
// K best (score descending, then c ascending).
//
// Alg. 3 and Alg. 4 loop over every person / university with one thread-private
// heap per OpenMP thread and merge the heaps with a tree (Alg. 2).  The GB300
// form streams the candidates' embedding rows once per batch of queries:
//
//   1. candidate list of the type (built once per type, ordered compaction);
//   2. sampling pass: the fp32 scores of an evenly strided sample of M
//      candidates; per query, the K-th best sampled score minus twice the
//      per-edge error bound is a threshold that can drop no candidate of the
//      exact top K (the K-th best of a subset is at most the K-th best of all);
//   3. full pass (k_tail_scan): every candidate row is read once with 16-byte
//      loads, a group of G lanes holding two rows in registers, and scored
//      against every query of the batch (query vectors e_h + w_r or
//      e_h * w_r in shared memory, each load feeding both rows); scores at or
//      above the threshold are appended to the query's survivor list
//      (warp-aggregated atomics);
//   4. per query (k_tail_final): the exact K-th best fp32 survivor score by a
//      radix select, the band of survivors within twice the error bound of it
//      rescored in fp64 in the canonical operation order (one member per
//      thread, e_h + w_r formed once in fp64 in shared memory), and the K best
//      of the band sorted in shared memory.
//
// Exactness: |S32 - w64| <= E = eps32 + eps64 for every candidate (the bound of
// mhr_graph.cu holds for any (u, r, v) triple and any summation order).  If c
// is in the exact top K then S32(c) >= w64_K - E >= S32_K - 2E, so the band
// holds every result, and sorting the band by (w64, c) gives them in order.
// A survivor list that overflows its sized buffer is detected on the host and
// that query is rescanned alone with room for every candidate.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "mhr_internal.cuh"
#include "mhr_util.cuh"

namespace mhr {

struct TailCache {
    uint32_t* cands[256] = {};  // candidate ids per vertex type (device; nullptr = not built)
    int64_t ncand[256] = {};
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    void* big = nullptr;  // survivors + band of one query rescanned alone
    size_t big_bytes = 0;
    cudaEvent_t ev[4] = {};

    ~TailCache() {
        for (uint32_t* p : cands)
            if (p) cudaFree(p);
        if (scratch) cudaFree(scratch);
        if (big) cudaFree(big);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

void destroy_tail(mhr_graph* g) {
    delete g->tail;
    g->tail = nullptr;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kFinalThreads = 1024;
constexpr int kSortMax = MHR_TAIL_K_MAX;       // power of two
constexpr size_t kQueryBytes = 64 * 1024;      // query vectors + thresholds per scan launch
constexpr int kMaxBatch = 256;                 // queries per scan launch
constexpr size_t kScratchBudget = size_t(1) << 30;
constexpr int kCompactBlocks = 512;

static_assert((kSortMax & (kSortMax - 1)) == 0, "sort size must be a power of two");

struct SurvRec {
    float s;     // fp32 screening score
    uint32_t v;  // candidate
};

struct BandRec {
    double w;  // fp64 score, canonical order
    uint32_t v;
    uint32_t pad;
};

struct ScanArgs {
    DevGraph g;
    const uint32_t* h;     // [nq] heads
    const uint16_t* r;     // [nq] relations
    int nq;
    int G;                 // lanes per candidate row (power of two, vector kernels)
    const uint32_t* cand;  // candidate ids; nullptr: candidate i is vertex i
    int64_t n_visit;       // candidates visited: positions i * stride for i < n_visit
    int64_t stride;
    const float* thr;      // [nq] keep scores >= thr[q]; nullptr keeps every score
    SurvRec* surv;         // query q's survivors at surv[q * cap]
    int64_t cap;
    unsigned int* cnt;     // [nq] survivors found (may exceed cap)
};

// ---------------------------------------------------------------------------
// candidate lists: ids of the vertices of one type, increasing
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_type_count(const uint8_t* __restrict__ vt, int64_t n, int type,
                                                     int64_t per_block, int64_t* __restrict__ counts) {
    const int64_t lo = blockIdx.x * per_block, hi = min(n, lo + per_block);
    int64_t c = 0;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        c += __syncthreads_count(i < hi && vt[i] == type);
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) k_type_offsets(int64_t* __restrict__ counts, int nb) {
    // exclusive scan of nb <= 1024 block counts in place; counts[nb] = total
    __shared__ int64_t sm[33];
    const int64_t x = threadIdx.x < nb ? counts[threadIdx.x] : 0;
    int64_t total;
    const int64_t ex = block_excl_scan<int64_t>(x, sm, &total);
    if (threadIdx.x < nb) counts[threadIdx.x] = ex;
    if (threadIdx.x == 0) counts[nb] = total;
}

__global__ void __launch_bounds__(1024) k_type_write(const uint8_t* __restrict__ vt, int64_t n, int type,
                                                     int64_t per_block, const int64_t* __restrict__ offsets,
                                                     uint32_t* __restrict__ out) {
    __shared__ int64_t sm[33];
    const int64_t lo = blockIdx.x * per_block, hi = min(n, lo + per_block);
    int64_t pos = offsets[blockIdx.x];
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t f = (i < hi && vt[i] == type) ? 1 : 0;
        int64_t tile;
        const int64_t ex = block_excl_scan<int64_t>(f, sm, &tile);
        if (f) out[pos + ex] = static_cast<uint32_t>(i);
        pos += tile;
    }
}

// ---------------------------------------------------------------------------
// query vectors: q = fl32(e_h + w_r) (TransE) or fl32(e_h * w_r) (DistMult),
// the first rounding of the screening arithmetic of every edge weight
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_queries(const ScanArgs& a, float* sq, float* sthr) {
    const int d = a.g.d;
    const int64_t total = static_cast<int64_t>(a.nq) * d;
    const bool transe = a.g.fn == MHR_SCORE_TRANSE_L1;
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int qi = static_cast<int>(idx / d), j = static_cast<int>(idx - static_cast<int64_t>(qi) * d);
        const float e = emb_f32(a.g.vemb, a.g.dtype, a.h[qi], d, j);
        const float w = emb_f32(a.g.remb, a.g.dtype, a.r[qi], d, j);
        sq[idx] = transe ? __fadd_rn(e, w) : __fmul_rn(e, w);
    }
    for (int qi = threadIdx.x; qi < a.nq; qi += blockDim.x) sthr[qi] = a.thr ? a.thr[qi] : -INFINITY;
    __syncthreads();
}

// one survivor per qualifying lane; warp-uniform call
__device__ __forceinline__ void append(const ScanArgs& a, int qi, bool keep, float s32, uint32_t v, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(a.cnt + qi, static_cast<unsigned>(__popc(m)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
        const unsigned pos = base + static_cast<unsigned>(__popc(m & ((1u << lane) - 1u)));
        if (pos < static_cast<unsigned long long>(a.cap)) a.surv[static_cast<int64_t>(qi) * a.cap + pos] = SurvRec{s32, v};
    }
}

// ---------------------------------------------------------------------------
// scan, 16-byte rows: a group of G lanes holds two adjacent candidate rows in
// registers (lane s of the group: 16-byte vectors s, s + G, ..., NV of them per
// row), so the group's loads of one step are G consecutive vectors of a row,
// and every query vector load from shared memory feeds both rows.  EV elements
// per vector (4 fp32 or 8 bf16).
// ---------------------------------------------------------------------------
template <bool BF16>
__device__ __forceinline__ void unpack_row(const uint4& w, float* x) {
    if constexpr (BF16) {
        x[0] = bf_lo(w.x);
        x[1] = bf_hi(w.x);
        x[2] = bf_lo(w.y);
        x[3] = bf_hi(w.y);
        x[4] = bf_lo(w.z);
        x[5] = bf_hi(w.z);
        x[6] = bf_lo(w.w);
        x[7] = bf_hi(w.w);
    } else {
        x[0] = __uint_as_float(w.x);
        x[1] = __uint_as_float(w.y);
        x[2] = __uint_as_float(w.z);
        x[3] = __uint_as_float(w.w);
    }
}

template <bool TRANSE>
__device__ __forceinline__ float term32(float q, float c) {
    if constexpr (TRANSE) return fabsf(__fsub_rn(q, c));
    else return q * c;
}

// keep-every-score mode (no threshold): candidate i of the visit order owns
// slot i, no counter needed; otherwise a warp-aggregated append
__device__ __forceinline__ void emit(const ScanArgs& a, int qi, bool valid, bool leader, float s32, uint32_t v,
                                     int64_t i, int lane, float thr) {
    if (a.thr == nullptr) {
        if (valid && leader) a.surv[static_cast<int64_t>(qi) * a.cap + i] = SurvRec{s32, v};
    } else {
        append(a, qi, valid && leader && s32 >= thr, s32, v, lane);
    }
}

__device__ __forceinline__ void keep_all_counts(const ScanArgs& a) {
    if (a.thr == nullptr && blockIdx.x == 0)
        for (int qi = threadIdx.x; qi < a.nq; qi += blockDim.x) a.cnt[qi] = static_cast<unsigned>(a.n_visit);
}

template <int NV, bool BF16, bool TRANSE>
__global__ void __launch_bounds__(kScanThreads) k_tail_scan(ScanArgs a) {
    extern __shared__ float4 smem4[];
    float* sq = reinterpret_cast<float*>(smem4);
    const int d = a.g.d, nq = a.nq;
    float* sthr = sq + static_cast<int64_t>(nq) * d;
    load_queries(a, sq, sthr);
    keep_all_counts(a);

    constexpr int EV = BF16 ? 8 : 4;
    const int dv = d / EV;
    const int G = a.G;
    const int lane = threadIdx.x & 31;
    const int s = lane & (G - 1);
    const int grp = lane / G;
    const int cpw = 2 * (32 / G);
    const int64_t ntiles = (a.n_visit + cpw - 1) / cpw;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kScanWarps;
    const size_t row_bytes = static_cast<size_t>(d) * (BF16 ? 2 : 4);
    const float gamma32 = a.g.gamma32;

    for (int64_t t = static_cast<int64_t>(blockIdx.x) * kScanWarps + (threadIdx.x >> 5); t < ntiles; t += nwarps) {
        const int64_t i0 = t * cpw + 2 * grp, i1 = i0 + 1;
        const bool valid0 = i0 < a.n_visit, valid1 = i1 < a.n_visit;
        uint32_t v0 = 0, v1 = 0;
        if (valid0) v0 = a.cand ? __ldg(a.cand + i0 * a.stride) : static_cast<uint32_t>(i0 * a.stride);
        if (valid1) v1 = a.cand ? __ldg(a.cand + i1 * a.stride) : static_cast<uint32_t>(i1 * a.stride);
        const uint4* row0 = reinterpret_cast<const uint4*>(static_cast<const char*>(a.g.vemb) + v0 * row_bytes);
        const uint4* row1 = reinterpret_cast<const uint4*>(static_cast<const char*>(a.g.vemb) + v1 * row_bytes);
        float x0[NV * EV], x1[NV * EV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int vi = s + G * k;
            uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
            if (valid0 && vi < dv) w0 = __ldg(row0 + vi);
            if (valid1 && vi < dv) w1 = __ldg(row1 + vi);
            unpack_row<BF16>(w0, x0 + k * EV);
            unpack_row<BF16>(w1, x1 + k * EV);
        }
        for (int qi = 0; qi < nq; ++qi) {
            const float4* q4 = reinterpret_cast<const float4*>(sq + static_cast<int64_t>(qi) * d);
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int vi = s + G * k;
                if (vi < dv) {
#pragma unroll
                    for (int e4 = 0; e4 < EV / 4; ++e4) {
                        const float4 qq = q4[vi * (EV / 4) + e4];
                        const float* y0 = x0 + k * EV + e4 * 4;
                        const float* y1 = x1 + k * EV + e4 * 4;
                        acc0 += term32<TRANSE>(qq.x, y0[0]);
                        acc1 += term32<TRANSE>(qq.x, y1[0]);
                        acc0 += term32<TRANSE>(qq.y, y0[1]);
                        acc1 += term32<TRANSE>(qq.y, y1[1]);
                        acc0 += term32<TRANSE>(qq.z, y0[2]);
                        acc1 += term32<TRANSE>(qq.z, y1[2]);
                        acc0 += term32<TRANSE>(qq.w, y0[3]);
                        acc1 += term32<TRANSE>(qq.w, y1[3]);
                    }
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) {
                acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
                acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            }
            const float s0 = TRANSE ? __fsub_rn(gamma32, acc0) : acc0;
            const float s1 = TRANSE ? __fsub_rn(gamma32, acc1) : acc1;
            const float thr = sthr[qi];
            emit(a, qi, valid0, s == 0, s0, v0, i0, lane, thr);
            emit(a, qi, valid1, s == 0, s1, v1, i1, lane, thr);
        }
    }
}

// scan, any row length: one warp per candidate, lanes stride over the row
template <bool TRANSE>
__global__ void __launch_bounds__(kScanThreads) k_tail_scan_any(ScanArgs a) {
    extern __shared__ float4 smem4[];
    float* sq = reinterpret_cast<float*>(smem4);
    const int d = a.g.d, nq = a.nq;
    float* sthr = sq + static_cast<int64_t>(nq) * d;
    load_queries(a, sq, sthr);
    keep_all_counts(a);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kScanWarps;
    const float gamma32 = a.g.gamma32;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kScanWarps + (threadIdx.x >> 5); i < a.n_visit; i += nwarps) {
        const int64_t pos = i * a.stride;
        const uint32_t v = a.cand ? __ldg(a.cand + pos) : static_cast<uint32_t>(pos);
        for (int qi = 0; qi < nq; ++qi) {
            const float* q = sq + static_cast<int64_t>(qi) * d;
            float acc = 0.f;
            for (int j = lane; j < d; j += 32) {
                const float c = emb_f32(a.g.vemb, a.g.dtype, v, d, j);
                if (TRANSE) acc += fabsf(__fsub_rn(q[j], c));
                else acc += q[j] * c;
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const float s32 = TRANSE ? __fsub_rn(gamma32, acc) : acc;
            emit(a, qi, true, lane == 0, s32, v, i, lane, sthr[qi]);
        }
    }
}

// ---------------------------------------------------------------------------
// CTA-wide radix select: the k-th largest key (1-based), 8 bits per pass
// ---------------------------------------------------------------------------
struct SelectSmem {
    unsigned hist[256];
    int digit;
    unsigned krem;
    unsigned count;
};

// warp 0: the digit whose bin holds the krem-th largest remaining key, and the
// rank inside that bin (bins scanned from 255 down)
__device__ __forceinline__ void pick_digit(SelectSmem& sm, unsigned krem) {
    if (threadIdx.x < 32) {
        const int L = threadIdx.x;
        unsigned c[8], local = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            c[m] = sm.hist[255 - 8 * L - m];
            local += c[m];
        }
        const unsigned incl = warp_incl_scan<unsigned>(local);
        const unsigned excl = incl - local;
        if (excl < krem && krem <= incl) {
            unsigned acc = excl;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (acc + c[m] >= krem) {
                    sm.digit = 255 - 8 * L - m;
                    sm.krem = krem - acc;
                    break;
                }
                acc += c[m];
            }
        }
    }
}

// the order-preserving key of an fp64 score, +0 and -0 mapped together (the
// result order compares scores numerically)
__device__ __forceinline__ uint64_t score_key(double w) {
    if (w == 0.0) w = 0.0;
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(w));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// k-th largest fp32 survivor score (1 <= k <= n)
__device__ float select_kth_score(const SurvRec* a, int64_t n, int64_t k, SelectSmem& sm) {
    uint32_t prefix = 0, mask = 0;
    unsigned krem = static_cast<unsigned>(k);
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sm.hist[b] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t key = f2key(a[i].s);
            if ((key & mask) == prefix) atomicAdd(&sm.hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        pick_digit(sm, krem);
        __syncthreads();
        prefix |= static_cast<uint32_t>(sm.digit) << shift;
        mask |= 255u << shift;
        krem = sm.krem;
        __syncthreads();
    }
    return key2f(prefix);
}

// composite key of a band record: (score key, ~v), larger = earlier in the result
__device__ __forceinline__ unsigned band_digit(uint64_t hi, uint32_t lo, int p) {
    return p < 8 ? static_cast<unsigned>((hi >> (56 - 8 * p)) & 255u)
                 : static_cast<unsigned>((lo >> (24 - 8 * (p - 8))) & 255u);
}

// k-th largest composite key of n band records (1 <= k <= n); keys are distinct
__device__ void select_kth_band(const BandRec* a, int64_t n, int64_t k, SelectSmem& sm, uint64_t* khi,
                                uint32_t* klo) {
    uint64_t phi = 0, mhi = 0;
    uint32_t plo = 0, mlo = 0;
    unsigned krem = static_cast<unsigned>(k);
    for (int p = 0; p < 12; ++p) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sm.hist[b] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t hi = score_key(a[i].w);
            const uint32_t lo = ~a[i].v;
            if ((hi & mhi) == phi && (lo & mlo) == plo) atomicAdd(&sm.hist[band_digit(hi, lo, p)], 1u);
        }
        __syncthreads();
        pick_digit(sm, krem);
        __syncthreads();
        const uint64_t dg = static_cast<uint64_t>(sm.digit);
        if (p < 8) {
            phi |= dg << (56 - 8 * p);
            mhi |= 255ull << (56 - 8 * p);
        } else {
            plo |= static_cast<uint32_t>(dg) << (24 - 8 * (p - 8));
            mlo |= 255u << (24 - 8 * (p - 8));
        }
        krem = sm.krem;
        __syncthreads();
    }
    *khi = phi;
    *klo = plo;
}

// ---------------------------------------------------------------------------
// sampling threshold: thr[q] = (K-th best sampled fp32 score) - 2E, rounded
// down; -inf when the sample holds fewer than K candidates
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFinalThreads) k_tail_thr(const SurvRec* __restrict__ surv, int64_t cap,
                                                           const unsigned* __restrict__ cnt, int K, double E2,
                                                           float* __restrict__ thr) {
    __shared__ SelectSmem sm;
    const int q = blockIdx.x;
    const int64_t n = min(static_cast<int64_t>(cnt[q]), cap);
    if (n < K) {
        if (threadIdx.x == 0) thr[q] = -INFINITY;
        return;
    }
    const float kth = select_kth_score(surv + static_cast<int64_t>(q) * cap, n, K, sm);
    if (threadIdx.x == 0) thr[q] = __double2float_rd(__dsub_rd(static_cast<double>(kth), E2));
}

// ---------------------------------------------------------------------------
// per query: band, fp64 rescoring, the K best in order
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ranks_before(const BandRec& x, const BandRec& y) {
    return x.w > y.w || (x.w == y.w && x.v < y.v);
}

constexpr int kQ64Max = 2048;  // rows up to this length use the shared fp64 query vector

template <bool TRANSE>
__device__ __forceinline__ double term64(double q, float c) {
    if constexpr (TRANSE) return fabs(__dsub_rn(q, static_cast<double>(c)));
    else return __dmul_rn(q, static_cast<double>(c));
}

// w(h, r, v) in the canonical order, with q64[j] = e_h[j] + w_r[j] (TransE)
// or e_h[j] * w_r[j] (DistMult) already formed in fp64: the same operations
// on the same values as the reference definition, j = 0..d-1 in order
template <bool TRANSE>
__device__ double rescore_row(const DevGraph& g, const double* q64, uint32_t v) {
    const int d = g.d;
    double acc = 0.0;
    if (g.dtype == MHR_F32 && (d & 3) == 0) {
        const float4* c4 = reinterpret_cast<const float4*>(static_cast<const float*>(g.vemb) + static_cast<int64_t>(v) * d);
#pragma unroll 4
        for (int j4 = 0; j4 < (d >> 2); ++j4) {
            const float4 c = __ldg(c4 + j4);
            const double* q = q64 + 4 * j4;
            acc = __dadd_rn(acc, term64<TRANSE>(q[0], c.x));
            acc = __dadd_rn(acc, term64<TRANSE>(q[1], c.y));
            acc = __dadd_rn(acc, term64<TRANSE>(q[2], c.z));
            acc = __dadd_rn(acc, term64<TRANSE>(q[3], c.w));
        }
    } else if (g.dtype == MHR_BF16 && (d & 7) == 0) {
        const uint4* c8 = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(g.vemb) + static_cast<int64_t>(v) * d);
#pragma unroll 2
        for (int j8 = 0; j8 < (d >> 3); ++j8) {
            const uint4 w = __ldg(c8 + j8);
            const double* q = q64 + 8 * j8;
            acc = __dadd_rn(acc, term64<TRANSE>(q[0], bf_lo(w.x)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[1], bf_hi(w.x)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[2], bf_lo(w.y)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[3], bf_hi(w.y)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[4], bf_lo(w.z)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[5], bf_hi(w.z)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[6], bf_lo(w.w)));
            acc = __dadd_rn(acc, term64<TRANSE>(q[7], bf_hi(w.w)));
        }
    } else {
        for (int j = 0; j < d; ++j) acc = __dadd_rn(acc, term64<TRANSE>(q64[j], emb_f32(g.vemb, g.dtype, v, d, j)));
    }
    return TRANSE ? __dsub_rn(g.gamma, acc) : acc;
}

__global__ void __launch_bounds__(kFinalThreads)
    k_tail_final(DevGraph g, const uint32_t* __restrict__ h, const uint16_t* __restrict__ r,
                 const SurvRec* __restrict__ surv, int64_t cap, const unsigned* __restrict__ cnt,
                 BandRec* __restrict__ band, int K, double E2, mhr_tail* __restrict__ out,
                 int32_t* __restrict__ n_out, unsigned* __restrict__ band_cnt) {
    __shared__ SelectSmem sm;
    extern __shared__ BandRec sbuf[];  // kSortMax records, then the fp64 query vector
    double* q64 = reinterpret_cast<double*>(sbuf + kSortMax);
    const int q = blockIdx.x;
    if (static_cast<int64_t>(cnt[q]) > cap) return;  // overflowed: rescanned alone by the host
    const int64_t n = cnt[q];
    const SurvRec* a = surv + static_cast<int64_t>(q) * cap;
    BandRec* b = band + static_cast<int64_t>(q) * cap;
    const uint32_t hq = h[q], rq = r[q];
    const bool transe = g.fn == MHR_SCORE_TRANSE_L1;
    const bool shared_q = g.d <= kQ64Max;

    // 1. the band: survivors within 2E of the K-th best fp32 score
    double lo = -INFINITY;
    if (n > K) lo = __dsub_rd(static_cast<double>(select_kth_score(a, n, K, sm)), E2);
    if (threadIdx.x == 0) sm.count = 0u;
    if (shared_q) {
        for (int j = threadIdx.x; j < g.d; j += blockDim.x) {
            const double e = static_cast<double>(emb_f32(g.vemb, g.dtype, hq, g.d, j));
            const double w = static_cast<double>(emb_f32(g.remb, g.dtype, rq, g.d, j));
            q64[j] = transe ? __dadd_rn(e, w) : __dmul_rn(e, w);
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const SurvRec x = a[i];
        if (static_cast<double>(x.s) >= lo) {
            const unsigned p = atomicAdd(&sm.count, 1u);
            b[p].v = x.v;
        }
    }
    __syncthreads();
    const unsigned nb = sm.count;
    // fp64 rescoring, one band member per thread over dense warps
    for (unsigned p = threadIdx.x; p < nb; p += blockDim.x) {
        const uint32_t v = b[p].v;
        double w;
        if (!shared_q) w = edge_w64(g, hq, rq, v);
        else if (transe) w = rescore_row<true>(g, q64, v);
        else w = rescore_row<false>(g, q64, v);
        b[p] = BandRec{w, v, 0u};
    }
    __syncthreads();

    // 2. the records to sort: the whole band, or exactly its K best
    unsigned m;
    if (nb <= static_cast<unsigned>(kSortMax)) {
        for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) sbuf[i] = b[i];
        m = nb;
    } else {
        uint64_t khi;
        uint32_t klo;
        select_kth_band(b, nb, K, sm, &khi, &klo);
        if (threadIdx.x == 0) sm.count = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const uint64_t hi = score_key(b[i].w);
            const uint32_t lw = ~b[i].v;
            if (hi > khi || (hi == khi && lw >= klo)) {
                const unsigned p = atomicAdd(&sm.count, 1u);
                if (p < static_cast<unsigned>(kSortMax)) sbuf[p] = b[i];
            }
        }
        __syncthreads();
        m = min(sm.count, static_cast<unsigned>(kSortMax));
    }
    unsigned P = 1;
    while (P < m) P <<= 1;
    for (unsigned i = m + threadIdx.x; i < P; i += blockDim.x) sbuf[i] = BandRec{-INFINITY, 0xffffffffu, 0u};
    __syncthreads();

    // 3. bitonic sort of P records, best first
    for (unsigned size = 2; size <= P; size <<= 1) {
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
                const unsigned j = i ^ stride;
                if (j > i) {
                    const BandRec x = sbuf[i], y = sbuf[j];
                    const bool best_first = (i & size) == 0;
                    if (best_first ? ranks_before(y, x) : ranks_before(x, y)) {
                        sbuf[i] = y;
                        sbuf[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }

    // 4. output
    const unsigned nout = min(m, static_cast<unsigned>(K));
    mhr_tail* o = out + static_cast<int64_t>(q) * K;
    for (unsigned i = threadIdx.x; i < nout; i += blockDim.x) {
        mhr_tail t;
        t.score = sbuf[i].w;
        t.v = sbuf[i].v;
        t.pad = 0u;
        o[i] = t;
    }
    if (threadIdx.x == 0) {
        n_out[q] = static_cast<int32_t>(nout);
        band_cnt[q] = nb;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

cudaError_t grow(void** p, size_t* have, size_t want) {
    if (*have >= want && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, want ? want : 16);
    if (e == cudaSuccess) *have = want;
    return e;
}

// scan kernel and launch shape for the graph's row format
struct ScanKernel {
    void (*fn)(ScanArgs) = nullptr;
    int G = 1;
    int rows_per_group = 1;
};

ScanKernel pick_scan(const DevGraph& dg) {
    const bool transe = dg.fn == MHR_SCORE_TRANSE_L1;
    const int d = dg.d;
    const bool bf = dg.dtype == MHR_BF16;
    // two rows per lane group: at most 16 elements of each row per lane
    const int ev = bf ? 8 : 4, nvmax = bf ? 2 : 4;
    ScanKernel k;
    if (d % ev == 0 && d / ev <= 32 * nvmax) {
        const int dv = d / ev;
        int G = 1;
        while ((dv + G - 1) / G > nvmax) G <<= 1;
        const int need = (dv + G - 1) / G;
        int NV = 1;
        while (NV < need) NV <<= 1;
        k.G = G;
        k.rows_per_group = 2;
        if (bf) {
            if (NV == 1) k.fn = transe ? k_tail_scan<1, true, true> : k_tail_scan<1, true, false>;
            else k.fn = transe ? k_tail_scan<2, true, true> : k_tail_scan<2, true, false>;
        } else {
            if (NV == 1) k.fn = transe ? k_tail_scan<1, false, true> : k_tail_scan<1, false, false>;
            else if (NV == 2) k.fn = transe ? k_tail_scan<2, false, true> : k_tail_scan<2, false, false>;
            else k.fn = transe ? k_tail_scan<4, false, true> : k_tail_scan<4, false, false>;
        }
        return k;
    }
    k.G = 32;
    k.rows_per_group = 1;
    k.fn = transe ? k_tail_scan_any<true> : k_tail_scan_any<false>;
    return k;
}

// Host-side set-up of the scan kernel for launches of up to nq_max queries:
// the shared-memory attribute and the resident blocks per SM.  Done once per
// call, before any event is recorded, so event times cover device work only.
mhr_status scan_setup(const mhr_graph* g, const ScanKernel& sk, int nq_max, int* per_sm) {
    const size_t smem = static_cast<size_t>(nq_max) * g->dg.d * 4 + static_cast<size_t>(nq_max) * 4;
    MHR_CUDA_TRY(cudaFuncSetAttribute(sk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int n = 0;
    MHR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sk.fn, kScanThreads, smem));
    *per_sm = std::max(1, n);
    return MHR_OK;
}

// a.nq <= the nq_max given to scan_setup, whose per_sm this takes
mhr_status launch_scan(const mhr_graph* g, const ScanKernel& sk, const ScanArgs& a, int per_sm, cudaStream_t st) {
    if (a.nq <= 0 || a.n_visit <= 0) return MHR_OK;
    const size_t smem = static_cast<size_t>(a.nq) * g->dg.d * 4 + static_cast<size_t>(a.nq) * 4;
    const int cpw = sk.rows_per_group * (32 / sk.G);
    const int64_t ntiles = (a.n_visit + cpw - 1) / cpw;
    const int64_t need = (ntiles + kScanWarps - 1) / kScanWarps;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(std::max(1, g->num_sms)) * per_sm)));
    ScanArgs b = a;
    b.G = sk.G;
    sk.fn<<<grid, kScanThreads, smem, st>>>(b);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}

mhr_status ensure_cands(mhr_graph* g, int type, cudaStream_t st) {
    TailCache* tc = g->tail;
    if (tc->cands[type]) return MHR_OK;
    const int64_t n = g->dg.n;
    const int nb = kCompactBlocks;
    const int64_t per_block = (n + nb - 1) / nb;
    int64_t* counts = nullptr;
    MHR_CUDA_TRY(cudaMalloc(&counts, sizeof(int64_t) * (nb + 1)));
    auto bail = [&](mhr_status s) {
        cudaFree(counts);
        return s;
    };
    k_type_count<<<nb, 1024, 0, st>>>(g->dg.vtypes, n, type, per_block, counts);
    k_type_offsets<<<1, 1024, 0, st>>>(counts, nb);
    int64_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, counts + nb, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "candidate count"));
    uint32_t* ids = nullptr;
    e = cudaMalloc(&ids, sizeof(uint32_t) * std::max<int64_t>(1, total));
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc (candidate list)"));
    k_type_write<<<nb, 1024, 0, st>>>(g->dg.vtypes, n, type, per_block, counts, ids);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(ids);
        return bail(cuda_fail(e, "candidate list"));
    }
    tc->cands[type] = ids;
    tc->ncand[type] = total;
    return bail(MHR_OK);
}

}  // namespace
}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_tail_topk(const mhr_graph* gc, int32_t nq, const uint32_t* h, const uint16_t* r,
                                    int32_t cand_type, int32_t K, mhr_tail* out, int32_t* n_out, mhr_mem mem,
                                    mhr_stats* stats, void* cuda_stream) {
    const auto t_start = std::chrono::steady_clock::now();
    MHR_TRY(check_graph(gc));
    mhr_graph* g = const_cast<mhr_graph*>(gc);
    if (nq < 0) return fail(MHR_EINVAL, "nq must be >= 0");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_TAIL_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_TAIL_K_MAX");
    if (cand_type < -1 || cand_type > 255) return fail(MHR_EINVAL, "cand_type must be in [-1, 255]");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    const int d = g->dg.d;
    if (static_cast<size_t>(d) * 4 + 4 > kQueryBytes) return fail(MHR_ERANGE, "dim exceeds 16383 for tail prediction");
    if (stats) *stats = mhr_stats{};
    if (nq == 0) return MHR_OK;
    if (!h || !r || !out || !n_out) return fail(MHR_EINVAL, "NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // validate the queries on the host (a short copy when they live on the device)
    std::vector<uint32_t> hh(nq);
    std::vector<uint16_t> hr(nq);
    if (mem == MHR_MEM_HOST) {
        std::copy(h, h + nq, hh.begin());
        std::copy(r, r + nq, hr.begin());
    } else {
        MHR_CUDA_TRY(cudaMemcpyAsync(hh.data(), h, 4ull * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(hr.data(), r, 2ull * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < nq; ++i) {
        if (static_cast<int64_t>(hh[i]) >= g->dg.n) return fail(MHR_EINVAL, "head out of range");
        if (static_cast<int32_t>(hr[i]) >= g->dg.R) return fail(MHR_EINVAL, "relation out of range");
    }

    if (!g->tail) g->tail = new TailCache();
    TailCache* tc = g->tail;
    for (cudaEvent_t& e : tc->ev)
        if (!e) MHR_CUDA_TRY(cudaEventCreate(&e));

    const uint32_t* cand = nullptr;
    int64_t Nc = g->dg.n;
    if (cand_type >= 0) {
        MHR_TRY(ensure_cands(g, cand_type, st));
        cand = tc->cands[cand_type];
        Nc = tc->ncand[cand_type];
    }

    // sizes: sample M, survivor capacity per query, queries per launch
    const int64_t M = std::min<int64_t>(Nc, std::max<int64_t>({int64_t(8192), int64_t(32) * K, Nc / 256}));
    const bool one_pass = M >= Nc;
    const int64_t ratio = one_pass ? 1 : (Nc + M - 1) / M;
    const int64_t capB = one_pass ? Nc : std::min<int64_t>(Nc, int64_t(8) * K * ratio + 8192);
    const int64_t capA = one_pass ? 0 : M;
    const size_t per_query = static_cast<size_t>(capA) * sizeof(SurvRec) +
                             static_cast<size_t>(capB) * (sizeof(SurvRec) + sizeof(BandRec)) + 64;
    int QB = static_cast<int>(std::min<int64_t>({static_cast<int64_t>(nq), int64_t(kMaxBatch),
                                                 static_cast<int64_t>(kQueryBytes / (static_cast<size_t>(d) * 4 + 4))}));
    QB = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(QB, static_cast<int64_t>(kScratchBudget / per_query))));

    // scratch layout
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_h = carve(4ull * nq), o_r = carve(2ull * nq), o_out = carve(sizeof(mhr_tail) * nq * K),
                 o_nout = carve(4ull * nq), o_thr = carve(4ull * QB), o_cnt = carve(4ull * QB * 2),
                 o_bc = carve(4ull * QB), o_sa = carve(sizeof(SurvRec) * QB * capA),
                 o_sb = carve(sizeof(SurvRec) * QB * capB), o_band = carve(sizeof(BandRec) * QB * capB);
    MHR_CUDA_TRY(grow(&tc->scratch, &tc->scratch_bytes, off));
    char* base = static_cast<char*>(tc->scratch);
    uint32_t* d_h = reinterpret_cast<uint32_t*>(base + o_h);
    uint16_t* d_r = reinterpret_cast<uint16_t*>(base + o_r);
    mhr_tail* d_out = reinterpret_cast<mhr_tail*>(base + o_out);
    int32_t* d_nout = reinterpret_cast<int32_t*>(base + o_nout);
    float* d_thr = reinterpret_cast<float*>(base + o_thr);
    unsigned* d_cnt = reinterpret_cast<unsigned*>(base + o_cnt);  // [QB] sample, [QB] full pass
    unsigned* d_bc = reinterpret_cast<unsigned*>(base + o_bc);
    SurvRec* d_sa = reinterpret_cast<SurvRec*>(base + o_sa);
    SurvRec* d_sb = reinterpret_cast<SurvRec*>(base + o_sb);
    BandRec* d_band = reinterpret_cast<BandRec*>(base + o_band);
    if (mem == MHR_MEM_HOST) {
        MHR_CUDA_TRY(cudaMemcpyAsync(d_h, hh.data(), 4ull * nq, cudaMemcpyHostToDevice, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(d_r, hr.data(), 2ull * nq, cudaMemcpyHostToDevice, st));
    } else {
        d_h = const_cast<uint32_t*>(h);
        d_r = const_cast<uint16_t*>(r);
        d_out = out;
        d_nout = n_out;
    }

    const double E2 = 2.0 * (g->eps32_edge + g->eps64_edge) * (1.0 + 1e-6);
    const ScanKernel sk = pick_scan(g->dg);
    const size_t final_smem = sizeof(BandRec) * kSortMax + (d <= kQ64Max ? sizeof(double) * d : 0);
    MHR_CUDA_TRY(cudaFuncSetAttribute(k_tail_final, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(final_smem)));
    int per_sm = 1;
    MHR_TRY(scan_setup(g, sk, std::min(QB, nq), &per_sm));

    int64_t n_pairs = 0, n_surv = 0, n_band = 0, n_rescan = 0;
    double ms_scan = 0.0;
    MHR_CUDA_TRY(cudaEventRecord(tc->ev[0], st));
    std::vector<unsigned> hc(2 * QB), hb(QB);
    for (int c0 = 0; c0 < nq && Nc > 0; c0 += QB) {
        const int qb = std::min(QB, nq - c0);
        MHR_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 4ull * QB * 2, st));
        ScanArgs a{};
        a.g = g->dg;
        a.h = d_h + c0;
        a.r = d_r + c0;
        a.nq = qb;
        a.cand = cand;
        unsigned* cntB = d_cnt + QB;
        if (!one_pass) {
            a.n_visit = M;
            a.stride = Nc / M;
            a.thr = nullptr;
            a.surv = d_sa;
            a.cap = capA;
            a.cnt = d_cnt;
            MHR_TRY(launch_scan(g, sk, a, per_sm, st));
            k_tail_thr<<<qb, kFinalThreads, 0, st>>>(d_sa, capA, d_cnt, K, E2, d_thr);
            MHR_CUDA_TRY(cudaGetLastError());
            n_pairs += static_cast<int64_t>(qb) * M;
        }
        a.n_visit = Nc;
        a.stride = 1;
        a.thr = one_pass ? nullptr : d_thr;
        a.surv = d_sb;
        a.cap = capB;
        a.cnt = cntB;
        MHR_CUDA_TRY(cudaEventRecord(tc->ev[2], st));
        MHR_TRY(launch_scan(g, sk, a, per_sm, st));
        MHR_CUDA_TRY(cudaEventRecord(tc->ev[3], st));
        n_pairs += static_cast<int64_t>(qb) * Nc;
        k_tail_final<<<qb, kFinalThreads, final_smem, st>>>(g->dg, d_h + c0, d_r + c0, d_sb, capB, cntB, d_band, K, E2,
                                                            d_out + static_cast<int64_t>(c0) * K, d_nout + c0, d_bc);
        MHR_CUDA_TRY(cudaGetLastError());
        MHR_CUDA_TRY(cudaMemcpyAsync(hc.data(), cntB, 4ull * qb, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(hb.data(), d_bc, 4ull * qb, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
        float ms = 0.f;
        MHR_CUDA_TRY(cudaEventElapsedTime(&ms, tc->ev[2], tc->ev[3]));
        ms_scan += ms;
        for (int i = 0; i < qb; ++i) {
            if (static_cast<int64_t>(hc[i]) <= capB) {
                n_surv += hc[i];
                n_band += hb[i];
                continue;
            }
            // survivors overflowed the sized buffer: rescan this query alone with
            // room for every candidate
            const size_t o_bs = align_up(sizeof(SurvRec) * Nc, 256);
            const size_t need = o_bs + sizeof(BandRec) * Nc + 256;
            MHR_CUDA_TRY(grow(&tc->big, &tc->big_bytes, need));
            SurvRec* bs = static_cast<SurvRec*>(tc->big);
            BandRec* bb = reinterpret_cast<BandRec*>(static_cast<char*>(tc->big) + o_bs);
            unsigned* bcnt = d_cnt;  // the sample counts are no longer needed
            MHR_CUDA_TRY(cudaMemsetAsync(bcnt, 0, 4, st));
            ScanArgs b = a;
            b.h = d_h + c0 + i;
            b.r = d_r + c0 + i;
            b.nq = 1;
            b.thr = one_pass ? nullptr : d_thr + i;
            b.surv = bs;
            b.cap = Nc;
            b.cnt = bcnt;
            MHR_TRY(launch_scan(g, sk, b, per_sm, st));
            k_tail_final<<<1, kFinalThreads, final_smem, st>>>(g->dg, d_h + c0 + i, d_r + c0 + i, bs, Nc, bcnt, bb, K, E2,
                                                               d_out + static_cast<int64_t>(c0 + i) * K, d_nout + c0 + i,
                                                               d_bc + i);
            MHR_CUDA_TRY(cudaGetLastError());
            unsigned c1 = 0, b1 = 0;
            MHR_CUDA_TRY(cudaMemcpyAsync(&c1, bcnt, 4, cudaMemcpyDeviceToHost, st));
            MHR_CUDA_TRY(cudaMemcpyAsync(&b1, d_bc + i, 4, cudaMemcpyDeviceToHost, st));
            MHR_CUDA_TRY(cudaStreamSynchronize(st));
            n_pairs += Nc;
            n_surv += c1;
            n_band += b1;
            ++n_rescan;
        }
    }
    if (Nc == 0) MHR_CUDA_TRY(cudaMemsetAsync(d_nout, 0, 4ull * nq, st));
    MHR_CUDA_TRY(cudaEventRecord(tc->ev[1], st));
    if (mem == MHR_MEM_HOST) {
        MHR_CUDA_TRY(cudaMemcpyAsync(out, d_out, sizeof(mhr_tail) * nq * K, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(n_out, d_nout, 4ull * nq, cudaMemcpyDeviceToHost, st));
    }
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats) {
        float ms_dev = 0.f;
        MHR_CUDA_TRY(cudaEventElapsedTime(&ms_dev, tc->ev[0], tc->ev[1]));
        stats->edges_scanned = n_pairs;
        stats->candidates = n_surv;
        stats->rescored = n_band;
        stats->dense_queries = n_rescan;
        stats->ms_device = ms_dev;
        stats->ms_join = ms_scan;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    return MHR_OK;
}
