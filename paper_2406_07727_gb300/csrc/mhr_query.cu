// Batched exact three-hop top-K path search (the hot path).
//
// For each query (s, t) every simple path s -r1-> u -r2-> v -r3-> t is scored
// as w(s,r1,u) + w(u,r2,v) + w(v,r3,t) and the K best are returned in the
// order score descending, (u, r1, v, r2, r3) ascending.  The paper's CPU
// design (Sec. 3.3, Alg. 2-4; Sec. 5, Alg. 6-7) keeps thread-private k-heaps
// and merges them with a barrier tree; here the same exact result comes from
// a meet-in-the-middle join sized for one GB300:
//
//   expand   hop-1 row of s and hop-3 (reverse) row of t, fp32 weights,
//            distinct frontier vertices with their best weight; S_f = sum of
//            out-degrees over N_out(s), S_b = sum of in-degrees over N_in(t)  (k_expand, k_lists)
//   plan     per query: scan the smaller side; split the scan into work
//            items of `chunk` CSR entries; order the near rows (natural, by
//            their score bound, or by bound + learned slack) and describe
//            every item                                               (k_plan, k_order_*, k_mlp_*, k_near)
//   join     a seed launch does the first rows of every multi-item query, then
//            one persistent 1024-thread CTA per SM takes items from its own
//            range and steals from the others; the far frontier sits in a
//            shared-memory bitmap (with a popcount rank for an exact bitmap,
//            a run table indexed by the bit for a coarse one, so the join needs
//            no hash probe), the near rows are streamed warp-cooperatively, every
//            hit whose bound can reach the kept band is scored in fp32 and
//            every path whose fp32 score can still reach the top K (within the
//            proven fp32 error bound of the running K-th score) is kept in a
//            shared-memory buffer; radix select + compaction bound the buffer,
//            and the CTA's K-th score is published with atomicMax      (k_middle)
//   merge    per query: exact K-th fp32 score over the kept candidates, the
//            band within twice the error bound, fp64 rescoring in the
//            canonical order (each distinct edge once), bitonic sort by the
//            total order                                             (k_merge1, k_rescore, k_merge2)
//   exact    queries whose band overflows every buffer (ties) are
//            recomputed with fp64 keys throughout                      (k_exact)
//
// Every kernel reads sizes and pointers from a device-resident PlanDev, so the
// whole sequence is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "mhr_internal.cuh"
#include "mhr_query.cuh"
#include "mhr_mlp_tc.cuh"
#include "mhr_util.cuh"

namespace mhr {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* __restrict__ a, int64_t n, int64_t x) {
    // first index i in [0, n) with a[i] > x (n if none)
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// thr - 2E rounded toward -inf, as float (conservative keep threshold)
__device__ __forceinline__ float keep_threshold(uint32_t key, double two_err) {
    if (key == 0u) return neg_inf();
    return __double2float_rd(__dsub_rd(static_cast<double>(key2f(key)), two_err));
}

// path order: 1 if a ranks strictly before b
__device__ __forceinline__ bool ranks_before(const mhr_path& a, const mhr_path& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.u != b.u) return a.u < b.u;
    if (a.r1 != b.r1) return a.r1 < b.r1;
    if (a.v != b.v) return a.v < b.v;
    if (a.r2 != b.r2) return a.r2 < b.r2;
    return a.r3 < b.r3;
}

__device__ __forceinline__ mhr_path worst_path() {
    mhr_path p;
    p.score = __longlong_as_double(0xfff0000000000000ll);  // -inf
    p.u = p.v = 0xffffffffu;
    p.r1 = p.r2 = p.r3 = p.pad = 0xffff;
    return p;
}

// in-place bitonic sort of m (power of two) paths, best first; all threads call
__device__ void block_sort_paths(mhr_path* a, int m) {
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                bool asc = (i & k) == 0;
                mhr_path x = a[i], y = a[i + j];
                bool swap = asc ? ranks_before(y, x) : ranks_before(x, y);
                if (swap) {
                    a[i] = y;
                    a[i + j] = x;
                }
            }
            __syncthreads();
        }
    }
}

// K-th largest order key among n keys (1 <= K <= n) by 4-pass radix select.
// key_at(i) gives key i; all threads call; hist has 256 slots.
template <typename KeyAt>
__device__ uint32_t block_select_kth(KeyAt key_at, int64_t n, int K, uint32_t* hist, uint32_t* bcast) {
    uint32_t prefix = 0, mask = 0;
    uint32_t remaining = static_cast<uint32_t>(K);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            uint32_t k = key_at(i);
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (wid == 0) {
            // lane l owns bins 255-8l .. 248-8l (descending)
            uint32_t c = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) c += hist[255 - 8 * lane - j];
            uint32_t cum = warp_incl_scan(c);
            unsigned b = __ballot_sync(FULL, cum >= remaining);
            int L = __ffs(b) - 1;
            if (lane == L) {
                uint32_t before = cum - c;
                for (int j = 0; j < 8; ++j) {
                    uint32_t bin = 255 - 8 * lane - j;
                    uint32_t h = hist[bin];
                    if (before + h >= remaining) {
                        bcast[0] = prefix | (bin << shift);
                        bcast[1] = remaining - before;
                        break;
                    }
                    before += h;
                }
            }
        }
        __syncthreads();
        prefix = bcast[0];
        remaining = bcast[1];
        mask |= 255u << shift;
        __syncthreads();
    }
    return prefix;
}

// ===========================================================================
// frontier expansion
// ===========================================================================
__global__ void k_init(const PlanDev* __restrict__ P, DevGraph g) {
    const int nq = P->nq;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = tid; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t s = P->S[q], t = P->T[q];
        P->status[q] = (s < g.n && t < g.n && s != t) ? 0 : 1;
        P->thr_g[q] = 0u;
        P->qmax[2 * q] = 0u;
        P->qmax[2 * q + 1] = 0u;
        P->sdeg_q[2 * q] = 0ull;
        P->sdeg_q[2 * q + 1] = 0ull;
        P->dense[q] = 0;
        P->pool_cnt[q] = 0;
        P->band_cnt[q] = 0;
        P->chain_cnt[q] = 0;
        P->n_out[q] = 0;
    }
    if (tid < kCntCount) P->counters[tid] = 0ull;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int c = tid; c < P->grid; c += gridDim.x * blockDim.x) P->cursors[c] = 0ull;
    for (int c = tid; c < (P->grid + 31) / 32; c += gridDim.x * blockDim.x) P->drained[c] = 0u;
    for (int64_t i = tid; i < 2 * static_cast<int64_t>(nq); i += stride) P->qkey[i] = (i & 1) ? 0u : 0xffffffffu;
    for (int64_t i = tid; i < P->nhist; i += stride) P->hist[i] = 0u;
    for (int64_t i = tid; i < P->item_cap; i += stride) P->item_ub[i] = 0u;
}

// One expansion slot: its query, position in the row of s (hop-1 side) or the
// reverse row of t (hop-3 side), the edge's far endpoint vtx and relation, the
// previous entry's vertex (run heads) and vtx's scan degree.
struct SlotInfo {
    uint32_t s, t, vtx, r, prev, sdeg;
    int64_t k;
    int q;
    bool sideA;
};

__device__ __forceinline__ SlotInfo slot_info(const PlanDev* __restrict__ P, const DevGraph& g, int64_t x, bool live) {
    SlotInfo o;
    o.s = o.t = o.vtx = o.r = o.sdeg = 0;
    o.prev = 0xffffffffu;
    o.k = 0;
    o.q = 0;
    o.sideA = true;
    if (!live) return o;
    const int64_t totA = P->totA;
    o.sideA = x < totA;
    const int64_t lx = o.sideA ? x : x - totA;
    const int64_t* offs = o.sideA ? P->a_off : P->c_off;
    o.q = static_cast<int>(upper_bound_i64(offs, P->nq + 1, lx) - 1);
    o.k = lx - offs[o.q];
    o.s = P->S[o.q];
    o.t = P->T[o.q];
    if (o.sideA) {
        const int64_t p = g.off[o.s] + o.k;
        o.vtx = g.col[p];
        o.r = g.rel[p];
        if (o.k > 0) o.prev = g.col[p - 1];
        o.sdeg = static_cast<uint32_t>(g.off[o.vtx + 1] - g.off[o.vtx]);
    } else {
        const int64_t p = g.roff[o.t] + o.k;
        o.vtx = g.rcol[p];
        o.r = g.rrel[p];
        if (o.k > 0) o.prev = g.rcol[p - 1];
        o.sdeg = static_cast<uint32_t>(g.roff[o.vtx + 1] - g.roff[o.vtx]);
    }
    return o;
}

// Writes a slot's fp32 weight, exclusion and run-head flag and adds the
// distinct frontier vertices' scan degrees to S_f / S_b.  All lanes call.
__device__ __forceinline__ void slot_commit(const PlanDev* __restrict__ P, const DevGraph& g, int64_t x, bool live,
                                            const SlotInfo& o, float wmine, int lane) {
    uint32_t key = 0xffffffffu;
    unsigned long long dsum = 0ull;
    if (live) {
        const uint32_t s = o.s, t = o.t, vtx = o.vtx, r = o.r;
        const bool sideA = o.sideA;
        const bool excl = (vtx == s) || (vtx == t);
        // A vertex with no scan edges can neither be scanned nor be hit, so it
        // never lies on a path: it is dropped from the distinct list.
        bool head = !excl && o.sdeg > 0 && (o.k == 0 || o.prev != vtx);
        // vertex partition: this call owns the paths whose hop-1 vertex u it owns
        if (sideA && P->part_count > 1 && vtx % static_cast<uint32_t>(P->part_count) !=
                                              static_cast<uint32_t>(P->part_index))
            head = false;
        bool allowed = true;
        const uint8_t* cons = P->cons;
        if (cons) {
            // constrained query: a slot of a disallowed hop-1 / hop-3 relation
            // weighs -inf; a vertex heads its run only when its type is allowed
            // and at least one edge of the run has an allowed relation
            const int R = g.R;
            const uint8_t* rf = cons + (sideA ? 0 : 2 * R);
            allowed = rf[r] != 0;
            if (head) {
                head = cons[3 * R + (sideA ? 0 : 256) + g.vtypes[vtx]] != 0;
                if (head && !allowed) {
                    const int64_t p0 = sideA ? g.off[s] : g.roff[t];
                    const int64_t rlen = (sideA ? g.off[s + 1] : g.roff[t + 1]) - p0;
                    const uint32_t* cc = sideA ? g.col : g.rcol;
                    const uint16_t* rr = sideA ? g.rel : g.rrel;
                    bool any = false;
                    for (int64_t j = o.k + 1; j < rlen && cc[p0 + j] == vtx && !any; ++j) any = rf[rr[p0 + j]] != 0;
                    head = any;
                }
            }
        }
        P->w32[x] = (excl || !allowed) ? neg_inf() : wmine;
        P->flag[x] = head ? 1u : 0u;
        P->w64own[x] = 0;
        key = 2u * static_cast<uint32_t>(o.q) + (sideA ? 0u : 1u);
        dsum = head ? o.sdeg : 0u;
    }
    // S_f / S_b: scan degrees of the distinct frontier vertices, summed per
    // (query, side) with one atomic per run of lanes sharing the key
    // (the 32-bit degrees summed as two 16-bit halves, so the warp sums cannot overflow)
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const uint32_t dd = static_cast<uint32_t>(dsum);
    const unsigned long long tot = (static_cast<unsigned long long>(__reduce_add_sync(peers, dd >> 16)) << 16) +
                                   __reduce_add_sync(peers, dd & 0xffffu);
    if (key != 0xffffffffu && lane == __ffs(peers) - 1 && tot) atomicAdd(&P->sdeg_q[key], tot);
}

// fp32 weight, exclusion and run-head flag of every slot.  Each lane resolves
// one slot of its warp's 32 (query, CSR position, endpoint degree) in
// parallel; then groups of G lanes score the 32 edges, H = 32 / G at a time.
__global__ void __launch_bounds__(256) k_expand(const PlanDev* __restrict__ P, DevGraph g) {
    const int lane = threadIdx.x & 31;
    const int G = P->score_width, H = 32 / G;
    const int sub = lane & (G - 1);
    const int64_t X = P->X;
    const int64_t warp_id = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t base = warp_id * 32; base < X; base += nwarps * 32) {  // warp-uniform
        const int64_t x = base + lane;
        const bool live = x < X;
        const SlotInfo o = slot_info(P, g, x, live);
        const uint32_t hu = o.sideA ? o.s : o.vtx, tv = o.sideA ? o.vtx : o.t;
        float wmine = 0.f;
        for (int rd = 0; rd < G; ++rd) {
            const int src = rd * H + lane / G;
            const uint32_t a = __shfl_sync(0xffffffffu, hu, src);
            const uint32_t rr = __shfl_sync(0xffffffffu, o.r, src);
            const uint32_t b = __shfl_sync(0xffffffffu, tv, src);
            // dead lanes score vertex 0's rows
            const float w = edge_w32_group(g, a, rr, b, sub, G);
            const float tw = __shfl_sync(0xffffffffu, w, ((lane - rd * H) & (H - 1)) * G);
            if (lane / H == rd) wmine = tw;
        }
        slot_commit(P, g, x, live, o, wmine, lane);
    }
}

// Query of a slot at position lx of one side: the last q with offs[q] <= lx.
// The warp's live slots are consecutive and on one side, so the warp finds
// the query q0 of its first slot (position lx0) with a 32-ary search (three
// rounds of one load per lane for 4,096 queries instead of twelve dependent
// loads per lane), then each lane counts the query starts after q0 that are
// <= lx among the next 32 (five shuffle steps).  A lane with more than 31
// query starts between lx0 and lx (empty queries) searches on its own.
__device__ __forceinline__ int warp_query_of(const int64_t* __restrict__ offs, int nq, int64_t lx0, int64_t lx,
                                             int lane) {
    int64_t lo = 0, span = static_cast<int64_t>(nq) + 1;  // offs[lo] <= lx0 < offs[lo + span] (or the end)
    while (span > 32) {
        const int64_t step = (span + 31) >> 5;
        const int64_t j = lane * step;
        const bool le = j < span && offs[lo + j] <= lx0;
        const int64_t c = __popc(__ballot_sync(0xffffffffu, le));  // >= 1: offs[lo] <= lx0
        const int64_t nlo = (c - 1) * step;
        span = min(step, span - nlo);
        lo += nlo;
    }
    {
        const bool le = lane < span && offs[lo + lane] <= lx0;
        lo += __popc(__ballot_sync(0xffffffffu, le)) - 1;
    }
    const int64_t j = lo + 1 + lane;
    const int64_t b = j <= nq ? offs[j] : INT64_MAX;
    int own = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int64_t pv = __shfl_sync(0xffffffffu, b, own + step - 1);
        if (pv <= lx) own += step;
    }
    const int64_t b31 = __shfl_sync(0xffffffffu, b, 31);
    if (b31 <= lx) return static_cast<int>(upper_bound_i64(offs, nq + 1, lx) - 1);
    return static_cast<int>(lo) + own;
}

// slot_info without the scan degree, the query found warp-cooperatively.
// All lanes call (the search uses the whole warp); lane 0 is live.
__device__ __forceinline__ SlotInfo slot_locate_warp(const PlanDev* __restrict__ P, const DevGraph& g, int64_t x,
                                                     bool live, int lane) {
    SlotInfo o;
    o.s = o.t = o.vtx = o.r = o.sdeg = 0;
    o.prev = 0xffffffffu;
    o.k = 0;
    o.q = 0;
    o.sideA = true;
    const int64_t totA = P->totA;
    const bool sA = x < totA;
    const unsigned mC = __ballot_sync(0xffffffffu, live && !sA);
    const unsigned mA = __ballot_sync(0xffffffffu, live && sA);
    const bool uniform = mA == 0u || mC == 0u;  // warp-uniform
    const int64_t lx = live ? (sA ? x : x - totA) : 0;
    int q = 0;
    if (uniform) {
        const int64_t* offs = mC == 0u ? P->a_off : P->c_off;
        const int64_t lx0 = __shfl_sync(0xffffffffu, lx, 0);
        q = warp_query_of(offs, P->nq, lx0, live ? lx : lx0, lane);
    } else if (live) {
        q = static_cast<int>(upper_bound_i64(sA ? P->a_off : P->c_off, P->nq + 1, lx) - 1);
    }
    if (!live) return o;
    const int64_t* offs = sA ? P->a_off : P->c_off;
    o.sideA = sA;
    o.q = q;
    o.k = lx - offs[q];
    o.s = P->S[q];
    o.t = P->T[q];
    if (sA) {
        const int64_t p = g.off[o.s] + o.k;
        o.vtx = g.col[p];
        o.r = g.rel[p];
        if (o.k > 0) o.prev = g.col[p - 1];
    } else {
        const int64_t p = g.roff[o.t] + o.k;
        o.vtx = g.rcol[p];
        o.r = g.rrel[p];
        if (o.k > 0) o.prev = g.rcol[p - 1];
    }
    return o;
}

// k_expand for rows of at most two 16-byte vectors per lane of a G-lane group
// (bf16 with d % 8 == 0 and d / 8 <= 2G, fp32 with d % 4 == 0 and d / 4 <=
// 2G).  The rows of the random side (the slot's far endpoint) of up to four
// rounds are loaded before any arithmetic, with the endpoint's scan-degree
// loads beside them, so a warp keeps up to four rows per group in flight
// instead of one; the fixed side (the query's s or t) and the relation row
// are the same few rows for many slots and come from L1.  The group sums of
// RB rounds are reduced together: plain xor steps down to RB lanes, then a
// butterfly in which each step halves the rounds a lane carries, so lane
// `sub` ends with round (sub mod RB): RB - 1 shuffles for the last log2(RB)
// steps of RB rounds instead of RB log2(RB).  Every lane still adds its own partial to
// its partner's at each step of the same xor tree, and fp32 addition is
// commutative, so with the same per-element expression and the same order
// within a lane the weights are those edge_w32_group computes.
// Four rounds at a time and three 256-thread blocks per SM (80 registers)
// measured fastest on the batching workload (3.31 ms per launch; eight rounds
// at two blocks per SM 3.88 ms; two rounds at four blocks 3.32 ms).
constexpr int kExpandRounds = 4;
template <int G>
__global__ void __launch_bounds__(256, 3) k_expand_v(const PlanDev* __restrict__ P, DevGraph g) {
    constexpr int H = 32 / G;
    constexpr int RB = G < kExpandRounds ? G : kExpandRounds;  // rounds loaded and reduced together
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);
    const int64_t X = P->X;
    const int64_t warp_id = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const bool f32 = g.dtype == MHR_F32;
    const bool transe = g.fn == MHR_SCORE_TRANSE_L1;
    const int nvec = f32 ? (g.d >> 2) : (g.d >> 3);  // 16-byte vectors per row
    const bool h0 = sub < nvec, h1 = sub + G < nvec;
    const uint4* E = static_cast<const uint4*>(g.vemb);
    const uint4* Rw = static_cast<const uint4*>(g.remb);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t base = warp_id * 32; base < X; base += nwarps * 32) {  // warp-uniform
        const int64_t x = base + lane;
        const bool live = x < X;
        SlotInfo o = slot_locate_warp(P, g, x, live, lane);
        const uint32_t fixv = o.sideA ? o.s : o.t;               // dead lanes: vertex 0
        const uint32_t rsa = (o.r << 1) | (o.sideA ? 1u : 0u);   // relation and side, one shuffle
        const int64_t* so = o.sideA ? g.off : g.roff;
        int64_t d0 = 0, d1 = 0;
        if (live) {
            d0 = so[o.vtx];
            d1 = so[o.vtx + 1];
        }
        float wmine = 0.f;
#pragma unroll
        for (int rb = 0; rb < G; rb += RB) {
            uint4 C0[RB], C1[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int src = (rb + i) * H + lane / G;
                const int64_t v = __shfl_sync(FULL, o.vtx, src);
                C0[i] = h0 ? __ldg(E + v * nvec + sub) : z;
                C1[i] = h1 ? __ldg(E + v * nvec + sub + G) : z;
            }
            float acc[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int src = (rb + i) * H + lane / G;
                const uint32_t q2 = __shfl_sync(FULL, rsa, src);
                const int64_t rr = q2 >> 1;
                const bool sa = (q2 & 1u) != 0u;
                const int64_t fv = __shfl_sync(FULL, fixv, src);
                const uint4 F0 = h0 ? __ldg(E + fv * nvec + sub) : z, B0 = h0 ? __ldg(Rw + rr * nvec + sub) : z;
                const uint4 F1 = h1 ? __ldg(E + fv * nvec + sub + G) : z,
                            B1 = h1 ? __ldg(Rw + rr * nvec + sub + G) : z;
                // side A: the edge (s, r, vtx), head fixed; side C: (vtx, r, t), tail fixed
                const uint4 As[2] = {sa ? F0 : C0[i], sa ? F1 : C1[i]};
                const uint4 Cs[2] = {sa ? C0[i] : F0, sa ? C1[i] : F1};
                const uint4 Bs[2] = {B0, B1};
                float a_ = 0.f;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 0 && !h0) break;
                    if (k == 1 && !h1) break;
                    const uint32_t a[4] = {As[k].x, As[k].y, As[k].z, As[k].w};
                    const uint32_t b[4] = {Bs[k].x, Bs[k].y, Bs[k].z, Bs[k].w};
                    const uint32_t c[4] = {Cs[k].x, Cs[k].y, Cs[k].z, Cs[k].w};
                    if (f32) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            a_ += term_tr(__uint_as_float(a[e]), __uint_as_float(b[e]), __uint_as_float(c[e]), transe);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            a_ += term_tr(bf_lo(a[e]), bf_lo(b[e]), bf_lo(c[e]), transe);
                            a_ += term_tr(bf_hi(a[e]), bf_hi(b[e]), bf_hi(c[e]), transe);
                        }
                    }
                }
                acc[i] = a_;
            }
            // xor steps G/2 .. RB: every round's sum over lanes that differ in those bits
#pragma unroll
            for (int off = G >> 1; off >= RB; off >>= 1)
#pragma unroll
                for (int i = 0; i < RB; ++i) acc[i] += __shfl_xor_sync(FULL, acc[i], off, G);
            // butterfly over the low log2(RB) bits: keep the half of the rounds
            // selected by this lane's bit, send the other half to the partner
#pragma unroll
            for (int off = RB >> 1; off > 0; off >>= 1) {
                const bool hi = (sub & off) != 0;
#pragma unroll
                for (int j = 0; j < off; ++j) {
                    const float send = hi ? acc[j] : acc[j + off];
                    const float keep = hi ? acc[j + off] : acc[j];
                    acc[j] = keep + __shfl_xor_sync(FULL, send, off, G);
                }
            }
            // lane sub of group gi now holds round rb + (sub mod RB) of slot (round) * H + gi
            const float w = transe ? __fsub_rn(g.gamma32, acc[0]) : acc[0];
            const int rd = lane / H;
            const float tw = __shfl_sync(FULL, w, (lane & (H - 1)) * G + (rd & (RB - 1)));
            if (rd >= rb && rd < rb + RB) wmine = tw;
        }
        o.sdeg = static_cast<uint32_t>(d1 - d0);
        slot_commit(P, g, x, live, o, wmine, lane);
    }
}

using ExpandKernel = void (*)(const PlanDev*, DevGraph);

// the expansion kernel for a graph's rows and group width
static ExpandKernel expand_kernel(const DevGraph& g, int G) {
    const bool vec2 = g.dtype == MHR_F32 ? ((g.d & 3) == 0 && (g.d >> 2) <= 2 * G)
                                         : ((g.d & 7) == 0 && (g.d >> 3) <= 2 * G);
    if (!vec2) return k_expand;
    switch (G) {
        case 1: return k_expand_v<1>;
        case 2: return k_expand_v<2>;
        case 4: return k_expand_v<4>;
        case 8: return k_expand_v<8>;
        case 16: return k_expand_v<16>;
        case 32: return k_expand_v<32>;
        default: return k_expand;
    }
}

// one thread per run head: the distinct frontier entry
__global__ void k_lists(const PlanDev* __restrict__ P, DevGraph g) {
    const int64_t X = P->X, totA = P->totA;
    const int nq = P->nq;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    // uniform trip count so whole warps reach the per-query max reduction
    const int64_t first = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t iters = (X + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t x = first + it * stride;
        uint32_t qkey = 0xffffffffu, mkey = 0u;
        if (x < X && P->flag[x]) {
            const bool sideA = x < totA;
            const int64_t lx = sideA ? x : x - totA;
            const int64_t* offs = sideA ? P->a_off : P->c_off;
            const int q = static_cast<int>(upper_bound_i64(offs, nq + 1, lx) - 1);
            const int64_t k = lx - offs[q];
            const int64_t rlen = offs[q + 1] - offs[q];
            const int64_t base = sideA ? offs[q] : totA + offs[q];
            const int64_t j = P->scan1[x] - P->scan1[base];
            const uint32_t s = P->S[q], t = P->T[q];
            const uint32_t* cc = sideA ? g.col + g.off[s] : g.rcol + g.roff[t];
            const uint32_t vtx = cc[k];
            float mw = P->w32[x];
            int64_t len = 1;
            while (k + len < rlen && cc[k + len] == vtx) {
                mw = fmaxf(mw, P->w32[x + len]);
                ++len;
            }
            ListEnt e;
            e.vertex = vtx;
            e.run_start = static_cast<uint32_t>(k);
            e.run_len = static_cast<uint32_t>(len);
            e.maxw = mw;
            if (sideA) {
                e.deg = static_cast<uint32_t>(g.off[vtx + 1] - g.off[vtx]);
                e.rowstart = static_cast<uint32_t>(g.off[vtx]);
                e.midw = g.maxw_out[vtx];
            } else {
                e.deg = static_cast<uint32_t>(g.roff[vtx + 1] - g.roff[vtx]);
                e.rowstart = static_cast<uint32_t>(g.roff[vtx]);
                e.midw = g.maxw_in[vtx];
            }
            e.pad = 0u;
            P->list[base + j] = e;
            qkey = 2u * static_cast<uint32_t>(q) + (sideA ? 0u : 1u);
            mkey = f2key(mw);
        }
        // per-(query, side) maximum: one atomic per group of lanes with the same key
        const unsigned peers = __match_any_sync(0xffffffffu, qkey);
        const uint32_t m = __reduce_max_sync(peers, mkey);
        if (qkey != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&P->qmax[qkey], m);
    }
}

// single block: direction choice and the work-item queue layout
__global__ void __launch_bounds__(1024) k_plan(const PlanDev* __restrict__ P) {
    __shared__ int64_t sm[33];
    __shared__ int64_t sm2[33];
    const int nq = P->nq;
    const int64_t totA = P->totA;
    const int64_t chunk = P->chunk;
    int64_t carry = 0, carry2 = 0;
    for (int base = 0; base < nq; base += blockDim.x) {
        const int q = base + threadIdx.x;
        int64_t items = 0, nn = 0;
        if (q < nq) {
            const int64_t a0 = P->a_off[q], a1 = P->a_off[q + 1];
            const int64_t c0 = totA + P->c_off[q], c1 = totA + P->c_off[q + 1];
            const int64_t du = P->scan1[a1] - P->scan1[a0];
            const int64_t dv = P->scan1[c1] - P->scan1[c0];
            const int64_t sf = static_cast<int64_t>(P->sdeg_q[2 * q]);
            const int64_t sb = static_cast<int64_t>(P->sdeg_q[2 * q + 1]);
            const bool fwd = sf <= sb;
            const int64_t near_cnt = fwd ? du : dv, far_cnt = fwd ? dv : du;
            const int64_t s_near = (P->status[q] == 0 && far_cnt > 0) ? (fwd ? sf : sb) : 0;
            P->dir[q] = fwd ? 1 : 0;
            P->near_cnt[q] = static_cast<int32_t>(near_cnt);
            P->far_cnt[q] = static_cast<int32_t>(far_cnt);
            P->s_near[q] = s_near;
            items = (s_near + chunk - 1) / chunk;
            nn = near_cnt;
        }
        int64_t tot, tot2;
        const int64_t ex = block_excl_scan(items, sm, &tot);
        const int64_t ex2 = block_excl_scan(nn, sm2, &tot2);
        if (q < nq) {
            P->item_off[q] = carry + ex;
            P->near_off[q] = carry2 + ex2;
        }
        carry += tot;
        carry2 += tot2;
    }
    if (threadIdx.x == 0) {
        P->item_off[nq] = carry;
        P->near_off[nq] = carry2;
    }
}

// Position of slot x: side, query, region base.  Returns false for slots
// that are not near-side entries of a valid near list.
__device__ __forceinline__ bool near_slot(const PlanDev* __restrict__ P, int64_t x, int& q, int64_t& base,
                                          bool& sideA) {
    const int64_t totA = P->totA;
    sideA = x < totA;
    const int64_t lx = sideA ? x : x - totA;
    const int64_t* offs = sideA ? P->a_off : P->c_off;
    q = static_cast<int>(upper_bound_i64(offs, P->nq + 1, lx) - 1);
    base = sideA ? offs[q] : totA + offs[q];
    if ((P->dir[q] == 1) != sideA) return false;
    return x - base < P->near_cnt[q];
}

// Learned order, per query: the endpoint half of the first layer, c_q = b1 +
// W1[:, 128:256] e_end[0:128] (bf16 inputs, fp32 sum), shared by all of the
// query's near entries.  One block per query, one thread per hidden unit.
__global__ void __launch_bounds__(kMlpHid) k_mlp_qbias(const PlanDev* __restrict__ P, DevGraph g) {
    if (P->order != 2) return;
    const int n = threadIdx.x;
    const uint32_t* W = reinterpret_cast<const uint32_t*>(P->mlp.W1);
    for (int q = blockIdx.x; q < P->nq; q += gridDim.x) {
        const uint32_t vb = P->dir[q] == 1 ? P->T[q] : P->S[q];
        float acc = __ldg(P->mlp.b1 + n);
        for (int k = 128; k < kMlpIn; k += 2) {
            const uint32_t a = feature_pair(g, 0u, vb, k);  // columns k, k+1 of [e_x; e_end]
            const uint32_t w = __ldg(W + (n * kMlpIn + k) / 2);
            acc += __uint_as_float(a << 16) * __uint_as_float(w << 16) +
                   __uint_as_float(a & 0xffff0000u) * __uint_as_float(w & 0xffff0000u);
        }
        P->mlp_qbias[static_cast<int64_t>(q) * kMlpHid + n] = acc;
    }
}

// Learned order (order 2): for every near entry the MLP predicts, from
// [e_entry; e_far endpoint], the slack of its row bound (best path score
// through the entry minus the bound); near_bucket orders the rows inside each
// bound level by it.  The endpoint half of the first layer is the per-query
// bias (k_mlp_qbias), so the tensor cores multiply 128-row tiles of the
// entries' first 128 features by W1[:, 0:128] (tcgen05, accumulator in TMEM).
// An MMA that does not complete within a second leaves its tile's predictions
// at 0 (the order only changes which rows go first, never the result) and
// counts in kCntTcTimeouts.
__device__ __forceinline__ uint4 feature_chunk(const DevGraph& g, uint32_t v, int c) {
    const int k = c * 8;
    if (g.dtype == MHR_BF16 && (g.d & 7) == 0 && k + 8 <= g.d)
        return __ldg(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(g.vemb) + static_cast<int64_t>(v) * g.d) + c);
    return make_uint4(feature_pair(g, v, 0u, k), feature_pair(g, v, 0u, k + 2), feature_pair(g, v, 0u, k + 4),
                      feature_pair(g, v, 0u, k + 6));
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_keys(const PlanDev* __restrict__ P, DevGraph g) {
    if (P->order != 2) return;
    const int nq = P->nq;
    const int64_t rows = P->near_off[nq];
    const int64_t ntiles = (rows + kTcRows - 1) / kTcRows;
    if (static_cast<int64_t>(blockIdx.x) >= ntiles) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTcSmem<128>& sm = *reinterpret_cast<MlpTcSmem<128>*>(smem_raw);
    __shared__ int64_t slot[kTcRows];
    __shared__ uint32_t va[kTcRows];
    __shared__ int qrow[kTcRows];
    tc_setup(sm);
    tc_stage_w1(sm, P->mlp.W1);
    uint32_t phase = 0;
    const float b2 = __ldg(P->mlp.b2);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * kTcRows;
        if (threadIdx.x < kTcRows) {
            const int64_t r = t0 + threadIdx.x;
            slot[threadIdx.x] = -1;
            va[threadIdx.x] = 0u;
            qrow[threadIdx.x] = 0;
            if (r < rows) {
                const int q = static_cast<int>(upper_bound_i64(P->near_off, nq + 1, r) - 1);
                const bool fwd = P->dir[q] == 1;
                const int64_t base = fwd ? P->a_off[q] : P->totA + P->c_off[q];
                const int64_t x = base + (r - P->near_off[q]);
                slot[threadIdx.x] = x;
                va[threadIdx.x] = P->list[x].vertex;
                qrow[threadIdx.x] = q;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTcRows * 16; i += blockDim.x) {
            const int r = i >> 4, c = i & 15;
            const uint4 v = slot[r] >= 0 ? feature_chunk(g, va[r], c) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(sm.A + tc::core_offset(r, c * 8, 128)) = v;
        }
        const bool ok = tc_mma_tile(sm, phase);
        if (!ok) {
            if (threadIdx.x < kTcRows && slot[threadIdx.x] >= 0) P->mlp_pred[slot[threadIdx.x]] = 0.f;
            if (threadIdx.x == 0) atomicAdd(&P->counters[kCntTcTimeouts], 1ull);
            break;
        }
        const int r = ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
        const int h = threadIdx.x >> 7;
        const float* qb = P->mlp_qbias + static_cast<int64_t>(qrow[r]) * kMlpHid;
        const float p = tc_row_half(
            sm.tmem, P->mlp.w2, [&](int c) { return qb[c]; }, [&](int, const float(&)[32]) {});
        sm.part[r][h] = p;
        __syncthreads();
        if (threadIdx.x < kTcRows && slot[threadIdx.x] >= 0) {
            // the predicted slack of the row bound (a path can only score below it)
            const float y = (sm.part[threadIdx.x][0] + sm.part[threadIdx.x][1]) + b2;
            P->mlp_pred[slot[threadIdx.x]] = fminf(y, 0.f);
        }
    }
    tc_teardown(sm);
}

// row bound of every near entry, its order key and the per-query key range
// (one atomic per run of lanes with the same query)
__global__ void k_order_key(const PlanDev* __restrict__ P, DevGraph g) {
    const int64_t X = P->X;
    const int order = P->order;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t iters = (X + stride - 1) / stride;  // uniform per warp
    const int64_t first = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t x = first + it * stride;
        uint32_t qid = 0xffffffffu, key = 0u;
        if (x < X) {
            P->degv3[x] = 0u;
            P->ubest[x] = 0u;
            int q;
            int64_t base;
            bool sideA;
            if (near_slot(P, x, q, base, sideA)) {
                const ListEnt e = P->list[x];
                // any path through this near entry scores (in fp32) at most:
                //   forward  (near = u): maxw1(u) + maxw_out(u) + max_v maxw3(v)
                //   backward (near = v): max_u maxw1(u) + maxw_in(v) + maxw3(v)
                float b;
                if (sideA) b = __fadd_rn(__fadd_rn(e.maxw, e.midw), key2f(P->qmax[2 * q + 1]));
                else b = __fadd_rn(__fadd_rn(key2f(P->qmax[2 * q]), e.midw), e.maxw);
                P->bnat[x] = b;
                if (order != 0) {  // both orders sort by the bound first
                    key = f2key(b);
                    P->okey[x] = key;
                    qid = static_cast<uint32_t>(q);
                }
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, qid);
        const uint32_t kmin = __reduce_min_sync(peers, key), kmax = __reduce_max_sync(peers, key);
        if (qid != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicMin(&P->qkey[2 * qid], kmin);
            atomicMax(&P->qkey[2 * qid + 1], kmax);
        }
    }
}

// `levels` buckets of the query's key range, highest keys first
__device__ __forceinline__ uint32_t order_bucket(uint32_t key, uint32_t kmin, uint32_t kmax, uint32_t levels) {
    const uint64_t range = static_cast<uint64_t>(kmax - kmin) + 1;
    return static_cast<uint32_t>((static_cast<uint64_t>(kmax - key) * levels) / range);
}

// Bucket (0..255) of near entry x of query q.  Order 1: 256 levels of the row
// bound.  Order 2: 64 levels of the row bound, each split in four by the
// learned slack prediction counted in level widths (0, 1, 2, 3 or more), so
// that within a bound level the rows predicted closest to their bound come
// first while the items keep falling bounds, which lets whole items be skipped.
__device__ __forceinline__ uint32_t near_bucket(const PlanDev* __restrict__ P, int64_t x, int q) {
    const uint32_t kmin = P->qkey[2 * q], kmax = P->qkey[2 * q + 1];
    if (P->order != 2) return order_bucket(P->okey[x], kmin, kmax, 256u);
    const uint32_t lvl = order_bucket(P->okey[x], kmin, kmax, 64u);
    const float width = (key2f(kmax) - key2f(kmin)) * (1.f / 64.f);
    const float slack = -P->mlp_pred[x];  // >= 0, or NaN
    uint32_t sub = 0u;
    if (width > 0.f && slack > 0.f) sub = static_cast<uint32_t>(fminf(3.f, floorf(slack / width)));
    return lvl * 4u + sub;
}

__global__ void k_order_hist(const PlanDev* __restrict__ P) {
    if (P->order == 0) return;
    const int64_t X = P->X;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < X; x += stride) {
        int q;
        int64_t base;
        bool sideA;
        if (!near_slot(P, x, q, base, sideA)) continue;
        const uint32_t b = near_bucket(P, x, q);
        P->orank[x] = atomicAdd(&P->hist[static_cast<int64_t>(q) * 256 + b], 1u);
    }
}

// ordered position of every near entry
__global__ void k_order_perm(const PlanDev* __restrict__ P) {
    const int64_t X = P->X;
    const int order = P->order;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < X; x += stride) {
        int q;
        int64_t base;
        bool sideA;
        if (!near_slot(P, x, q, base, sideA)) continue;
        int64_t pos = x - base;
        if (order != 0) {
            const uint32_t b = near_bucket(P, x, q);
            const int64_t h = static_cast<int64_t>(q) * 256;
            pos = P->hscan[h + b] - P->hscan[h] + P->orank[x];
        }
        P->nperm[base + pos] = static_cast<uint32_t>(x - base);
        P->degv3[base + pos] = P->list[x].deg;
    }
}

constexpr uint32_t kGposMulti = 0xffffffffu;   // group spans several near rows
constexpr uint32_t kGposPruned = 0xfffffffeu;  // group inside one row whose bound misses the band
constexpr int kSeedEdges = 32768;   // edges of each query's highest-bound rows done by the seed launch
constexpr int kSeedMinItems = 2;    // queries with fewer work items are not seeded

// near entries in ordered position: (prefix of scan degree, row start), row
// bound; per work item its descriptor and its largest row bound
__global__ void k_near(const PlanDev* __restrict__ P, DevGraph g) {
    const int64_t X = P->X;
    const int64_t chunk = P->chunk;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < X; x += stride) {
        int q;
        int64_t base;
        bool sideA;
        if (!near_slot(P, x, q, base, sideA)) continue;
        const int64_t old = base + P->nperm[x];
        const ListEnt e = P->list[old];
        const int64_t pre = P->scan4[x] - P->scan4[base];
        P->nearP[x] = make_uint2(static_cast<uint32_t>(pre), e.rowstart);
        P->nearL[x] = e;
        const float b = P->bnat[old];
        P->nearB[x] = b;
        if (e.deg == 0) continue;
        // Every near entry scans at least one edge, so each edge of the query's
        // near-edge space lies in exactly one entry: the entry holding an item's
        // first (last) edge writes that field of the item's descriptor.
        const int64_t s_near = P->s_near[q];
        const int64_t pend = pre + e.deg;
        const uint32_t xi = static_cast<uint32_t>(x - base);
        const int64_t i0 = P->item_off[q] + pre / chunk;
        const int64_t i1 = P->item_off[q] + (pend - 1) / chunk;
        const uint32_t key = f2key(b);
        // seeded: the seed launch does the query's first kSeedEdges edges
        const bool seeded = P->prune && P->item_off[q + 1] - P->item_off[q] >= kSeedMinItems;
        for (int64_t i = i0; i <= i1; ++i) {
            const int64_t ie0 = (i - P->item_off[q]) * chunk;
            const int64_t ie1 = min(ie0 + chunk, s_near) - 1;
            if (ie0 >= pre) {
                P->item_desc[i].x = static_cast<uint32_t>(q) | (seeded ? 0x80000000u : 0u);
                P->item_desc[i].y = xi;
                P->item_desc[i].w = static_cast<uint32_t>(i - P->item_off[q]);
            }
            if (ie1 < pend) P->item_desc[i].z = xi;
            if (P->prune) atomicMax(&P->item_ub[i], key);
        }
        if (pre <= kSeedEdges - 1 && kSeedEdges - 1 < pend) P->seed_k[q].x = xi;
        if (pre <= kSeedEdges && kSeedEdges < pend) P->seed_k[q].y = xi;
    }
}

// ===========================================================================
// the middle join (persistent)
// ===========================================================================
constexpr int kRelCacheVecs = 512;  // 8 KB of fp32 relation embeddings
// a work item taken from the queue, ready to run
struct ItemSel {
    int64_t item;  // == total items: none left
    int32_t q;
    uint32_t e0, e1, k0, k1;  // edge range; near entries holding its first and last edge
    uint32_t gk;              // the query's shared K-th score key when it was taken
    uint32_t ub;              // key of the item's largest row bound
};

struct MidSmem {
    uint32_t bm[kMaxBmWords];
    uint32_t rank[kMaxRank + 8];
    Cand cand[kCandCap];
    uint32_t gmap[kMaxChunk / 32 + 32];
    uint32_t gpos[kMaxChunk / 32];  // CSR position of a single-row group's first edge, or a marker
    uint32_t hist[256];
    uint32_t bc[4];
    int64_t red[33];
    uint32_t redu[33];
    float4 relc[kRelCacheVecs];  // relation embeddings (fp32) when R*d fits
    uint8_t compact[kMidWarps][32];  // per-warp lane map of surviving hits
    // per-query state
    int q, dir, near_cnt, far_cnt, local_dense, skip;
    uint32_t s, t;
    int64_t near_base, far_base, a_base, c_base, s_near;
    // per-item state
    int64_t item;
    int item_q;  // the item's query
    uint32_t e0, e1, k0, k1;
    int cand_cnt, hit_cnt;
    int batch_next;  // next batch of 32 hits to score
    int nx_claim;    // set by the warp that takes the next item
    int round_cnt;  // cand_cnt snapshot taken before the barrier that opens a round
    int pool_off;
    uint32_t lt_key;
    float thr_keep;
    // launch-wide constants and thread-0 counters (kept here to spare registers)
    double two_err;
    int64_t total_items;
    uint32_t f_gk;  // the query's shared K-th score key as read when the item was taken
    ItemSel nx;     // next item, taken during the current item's score phase
    int nx_ready;
    int victim;     // offset of the range the CTA currently drains
    unsigned long long c_scanned, c_hits, c_cands, c_skipped;
};

// block-wide in-place compaction of the candidate buffer to s32 >= thr
__device__ void compact_cands(MidSmem& sm, float thr) {
    const int n = sm.cand_cnt;
    int w = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        Cand c;
        bool keep = false;
        if (i < n) {
            c = sm.cand[i];
            keep = c.s32 >= thr;
        }
        int tot;
        const int pos = block_excl_scan(keep ? 1 : 0, reinterpret_cast<int*>(sm.redu), &tot);
        if (keep) sm.cand[w + pos] = c;
        w += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sm.cand_cnt = w;
    __syncthreads();
}

// raise the local threshold from the buffer and the global one, then compact
__device__ void flush_cands(MidSmem& sm, const PlanDev* __restrict__ P, int K) {
    const int n = sm.cand_cnt;
    if (n >= K) {
        const uint32_t key = block_select_kth([&](int64_t i) { return f2key(sm.cand[i].s32); }, n, K,
                                              sm.hist, sm.bc);
        if (threadIdx.x == 0) {
            if (key > sm.lt_key) sm.lt_key = key;
            atomicMax(&P->thr_g[sm.q], key);
        }
    }
    if (threadIdx.x == 0) {
        const uint32_t gk = atomicOr(&P->thr_g[sm.q], 0u);
        if (gk > sm.lt_key) sm.lt_key = gk;
        sm.thr_keep = keep_threshold(sm.lt_key, sm.two_err);
    }
    __syncthreads();
    compact_cands(sm, sm.thr_keep);
    // A band still denser than kDenseLimit goes to the query's pool now, which
    // frees the buffer; only a full pool sends the query to the exact path.
    if (threadIdx.x == 0) {
        sm.pool_off = -1;
        if (sm.cand_cnt > kDenseLimit && !sm.local_dense) {
            const int n = sm.cand_cnt;
            const int off = atomicAdd(&P->pool_cnt[sm.q], n);
            if (off + n > P->pq) {
                sm.local_dense = 1;
                atomicExch(&P->dense[sm.q], 1);
#ifdef MHR_PHASE_TIMING
                printf("MHR_DENSE spill q %d blk %d off %d n %d lt %.6f keep %.6f two_err %.6g\n", sm.q, blockIdx.x,
                       off, n, key2f(sm.lt_key), sm.thr_keep, sm.two_err);
#endif
            } else {
                sm.pool_off = off;
                sm.c_cands += static_cast<unsigned long long>(n);
            }
        }
        sm.round_cnt = sm.pool_off >= 0 ? 0 : sm.cand_cnt;
    }
    __syncthreads();
    if (sm.pool_off >= 0) {
        Cand* dst = P->pool + static_cast<int64_t>(sm.q) * P->pq + sm.pool_off;
        for (int i = threadIdx.x; i < sm.cand_cnt; i += blockDim.x) dst[i] = sm.cand[i];
        __syncthreads();
        if (threadIdx.x == 0) sm.cand_cnt = 0;
        __syncthreads();
    }
}

// final flush of the current query into its candidate pool
__device__ void finish_query(MidSmem& sm, const PlanDev* __restrict__ P, int K) {
    if (!sm.local_dense) flush_cands(sm, P, K);
    if (threadIdx.x == 0) {
        sm.pool_off = -1;
        if (!sm.local_dense && sm.cand_cnt > 0) {
            const int n = sm.cand_cnt;
            const int off = atomicAdd(&P->pool_cnt[sm.q], n);
            if (off + n > P->pq) {
                atomicExch(&P->dense[sm.q], 1);
#ifdef MHR_PHASE_TIMING
                printf("MHR_DENSE pool q %d blk %d off %d n %d lt %.6f\n", sm.q, blockIdx.x, off, n, key2f(sm.lt_key));
#endif
            }
            else sm.pool_off = off;
            sm.c_cands += static_cast<unsigned long long>(n);
        }
    }
    __syncthreads();
    if (sm.pool_off >= 0) {
        Cand* dst = P->pool + static_cast<int64_t>(sm.q) * P->pq + sm.pool_off;
        for (int i = threadIdx.x; i < sm.cand_cnt; i += blockDim.x) dst[i] = sm.cand[i];
    }
    __syncthreads();
}

// number of set bits of the far bitmap before bit b: the 256-bit block's rank,
// whole 64-bit words of the block below b, the low half of b's 64-bit word when
// b lies in its high half, then b's own word
__device__ __forceinline__ uint32_t bm_rank(const MidSmem& sm, uint32_t b) {
    const uint64_t* bm64 = reinterpret_cast<const uint64_t*>(sm.bm);
    uint32_t r = sm.rank[b >> 8];
    for (uint32_t w = (b >> 8) << 2; w < (b >> 6); ++w) r += __popcll(bm64[w]);
    if (b & 32u) r += __popc(sm.bm[(b >> 5) - 1u]);
    return r + __popc(sm.bm[b >> 5] & ((1u << (b & 31u)) - 1u));
}

__device__ void setup_query(MidSmem& sm, const PlanDev* __restrict__ P, int q) {
    if (threadIdx.x == 0) {
        sm.q = q;
        sm.s = P->S[q];
        sm.t = P->T[q];
        sm.dir = P->dir[q];
        sm.near_cnt = P->near_cnt[q];
        sm.far_cnt = P->far_cnt[q];
        sm.s_near = P->s_near[q];
        sm.a_base = P->a_off[q];
        sm.c_base = P->totA + P->c_off[q];
        sm.near_base = sm.dir ? sm.a_base : sm.c_base;
        sm.far_base = sm.dir ? sm.c_base : sm.a_base;
        sm.cand_cnt = 0;
        sm.lt_key = 0u;
        sm.thr_keep = neg_inf();
        sm.local_dense = 0;
    }
    const int nbw = P->nbw;
    for (int i = threadIdx.x; i < nbw; i += blockDim.x) sm.bm[i] = 0u;
    __syncthreads();
    const int sigma = P->sigma;
    const ListEnt* far = P->list + sm.far_base;
    for (int k = threadIdx.x; k < sm.far_cnt; k += blockDim.x) {
        const uint32_t bv = far[k].vertex >> sigma;
        atomicOr(&sm.bm[bv >> 5], 1u << (bv & 31u));
    }
    __syncthreads();
    if (sigma == 0) {
        // exact bitmap: rank[b] = set bits in words [0, 8b), so a far vertex's
        // rank is its far-list index
        const int nblk = (nbw + kRankWords - 1) / kRankWords;
        const int per = (nblk + blockDim.x - 1) / blockDim.x;  // <= 4
        int mine[4] = {0, 0, 0, 0};
        int sum = 0;
        for (int j = 0; j < per; ++j) {
            const int b = threadIdx.x * per + j;
            int c = 0;
            if (b < nblk)
                for (int w = b * kRankWords; w < min(nbw, (b + 1) * kRankWords); ++w) c += __popc(sm.bm[w]);
            mine[j] = c;
            sum += c;
        }
        int tot;
        int ex = block_excl_scan(sum, reinterpret_cast<int*>(sm.redu), &tot);
        for (int j = 0; j < per; ++j) {
            const int b = threadIdx.x * per + j;
            if (b < nblk) sm.rank[b] = static_cast<uint32_t>(ex);
            ex += mine[j];
        }
    }
    __syncthreads();
    if (sigma > 0) {
        // coarse bitmap (2^sigma vertices per bit): the far list is sorted by
        // vertex, so the vertices of a set bit are contiguous in it; record,
        // indexed by the bit itself, the run's first entry and vertex (written
        // by the thread at the run's start) and its last vertex and entry
        // (written by the thread at its end: the other 8-byte half).  Entries
        // of clear bits are stale but never read: the scan reads an entry only
        // after finding its bit set.
        uint2* fs = reinterpret_cast<uint2*>(P->far_start + static_cast<int64_t>(blockIdx.x) * P->far_cap);
        const int fc = sm.far_cnt;
        for (int k = threadIdx.x; k < fc; k += blockDim.x) {
            const uint32_t fv = far[k].vertex, bv = fv >> sigma;
            const bool first = k == 0 || (far[k - 1].vertex >> sigma) != bv;
            const bool last = k == fc - 1 || (far[k + 1].vertex >> sigma) != bv;
            if (first) fs[2 * static_cast<int64_t>(bv)] = make_uint2(static_cast<uint32_t>(k), fv);
            if (last) fs[2 * static_cast<int64_t>(bv) + 1] = make_uint2(fv, static_cast<uint32_t>(k));
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float4 ld4(const float* base, int64_t row, int d, int j) {
    return __ldg(reinterpret_cast<const float4*>(base + row * d) + j);
}

__device__ __forceinline__ float term4(const float4& h, const float4& r, const float4& t, bool transe) {
    if (transe)
        return fabsf(__fsub_rn(__fadd_rn(h.x, r.x), t.x)) + fabsf(__fsub_rn(__fadd_rn(h.y, r.y), t.y)) +
               fabsf(__fsub_rn(__fadd_rn(h.z, r.z), t.z)) + fabsf(__fsub_rn(__fadd_rn(h.w, r.w), t.w));
    return (h.x * r.x) * t.x + (h.y * r.y) * t.y + (h.z * r.z) * t.z + (h.w * r.w) * t.w;
}

// fp32 weight of the middle edge (u, r, v) for the f32 rows with d = 4*vec,
// vec <= kHitVecs*G: lane `sub` of a group of G owns vectors sub + k*G.  The
// near-side row (the scanned vertex) stays in registers across the group's
// consecutive hits, the relation row comes from shared memory when cached,
// and only the far-side row is fetched per hit (its kHitVecs loads issued
// together).
#ifndef MHR_HIT_VECS
#define MHR_HIT_VECS 2
#endif
constexpr int kHitVecs = MHR_HIT_VECS;  // 16-byte vectors per lane and row in the hit scorer

struct NearRow {
    float4 v[kHitVecs];
    uint32_t id;
};

__device__ __forceinline__ float hit_w32_f32(const DevGraph& g, NearRow& nr, uint32_t near_v, uint32_t far_v,
                                             uint32_t r, bool fwd, int sub, int G, int vec,
                                             const float4* relc) {
    const float* E = static_cast<const float*>(g.vemb);
    const float* Rw = static_cast<const float*>(g.remb);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    bool has[kHitVecs];
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) has[k] = sub + k * G < vec;
    if (near_v != nr.id) {
#pragma unroll
        for (int k = 0; k < kHitVecs; ++k) nr.v[k] = has[k] ? ld4(E, near_v, g.d, sub + k * G) : z;
        nr.id = near_v;
    }
    float4 f[kHitVecs], rv[kHitVecs];
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) f[k] = has[k] ? ld4(E, far_v, g.d, sub + k * G) : z;
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) {
        if (relc) rv[k] = has[k] ? relc[r * vec + sub + k * G] : z;
        else rv[k] = has[k] ? ld4(Rw, r, g.d, sub + k * G) : z;
    }
    const bool transe = g.fn == MHR_SCORE_TRANSE_L1;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k)
        acc += has[k] ? (fwd ? term4(nr.v[k], rv[k], f[k], transe) : term4(f[k], rv[k], nr.v[k], transe)) : 0.f;
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    return transe ? __fsub_rn(g.gamma32, acc) : acc;
}

// The same for bf16 rows with d = 8*vec, vec <= kHitVecs*G: 16-byte vectors of
// eight bf16 values, widened exactly to fp32 before the fp32 arithmetic (so
// the screening error bound is unchanged).  The near row's raw bits stay in
// the float4 registers of nr; relc holds the bf16 relation table when it fits.
__device__ __forceinline__ uint4 f4_bits(const float4& f) {
    return make_uint4(__float_as_uint(f.x), __float_as_uint(f.y), __float_as_uint(f.z), __float_as_uint(f.w));
}
__device__ __forceinline__ float4 bits_f4(const uint4& u) {
    return make_float4(__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z), __uint_as_float(u.w));
}
__device__ __forceinline__ float term8(const uint4& h, const uint4& r, const uint4& t, bool transe) {
    const uint32_t a[4] = {h.x, h.y, h.z, h.w}, b[4] = {r.x, r.y, r.z, r.w}, c[4] = {t.x, t.y, t.z, t.w};
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        acc += term_tr(bf_lo(a[i]), bf_lo(b[i]), bf_lo(c[i]), transe);
        acc += term_tr(bf_hi(a[i]), bf_hi(b[i]), bf_hi(c[i]), transe);
    }
    return acc;
}

__device__ __forceinline__ float hit_w32_bf16(const DevGraph& g, NearRow& nr, uint32_t near_v, uint32_t far_v,
                                              uint32_t r, bool fwd, int sub, int G, int vec, const float4* relc) {
    const uint4* E = static_cast<const uint4*>(g.vemb);
    const uint4* Rw = static_cast<const uint4*>(g.remb);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    bool has[kHitVecs];
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) has[k] = sub + k * G < vec;
    if (near_v != nr.id) {
#pragma unroll
        for (int k = 0; k < kHitVecs; ++k)
            nr.v[k] = bits_f4(has[k] ? __ldg(E + static_cast<int64_t>(near_v) * vec + sub + k * G) : z);
        nr.id = near_v;
    }
    uint4 f[kHitVecs], rv[kHitVecs];
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) f[k] = has[k] ? __ldg(E + static_cast<int64_t>(far_v) * vec + sub + k * G) : z;
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) {
        if (relc) rv[k] = has[k] ? f4_bits(relc[r * vec + sub + k * G]) : z;
        else rv[k] = has[k] ? __ldg(Rw + static_cast<int64_t>(r) * vec + sub + k * G) : z;
    }
    const bool transe = g.fn == MHR_SCORE_TRANSE_L1;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kHitVecs; ++k) {
        const uint4 nv = f4_bits(nr.v[k]);
        acc += has[k] ? (fwd ? term8(nv, rv[k], f[k], transe) : term8(f[k], rv[k], nv, transe)) : 0.f;
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    return transe ? __fsub_rn(g.gamma32, acc) : acc;
}

// A query is seeded (its first kSeedEdges edges done by the seed launch) when
// pruning is on and it has at least kSeedMinItems work items.
__device__ __forceinline__ bool seeded_query(const PlanDev* __restrict__ P, int q, bool prune) {
    return prune && P->item_off[q + 1] - P->item_off[q] >= kSeedMinItems;
}

// ---------------------------------------------------------------------------
// Tensor-core screen of the middle edges of a warp batch (DistMult, R <= 16).
// For hit h (lane h) the weight of every relation is (e_u (*) e_v) . W^T: the
// products p = fl32(e_u[j] e_v[j]) form a 32 x d bf16 hi/lo matrix, the
// relation table a d x R one, and three m16n8k16 products (hi.hi, hi.lo,
// lo.hi) accumulate in fp32.  Lane h returns the weight of its own relation.
__device__ __forceinline__ float2 emb_pair(const DevGraph& g, uint32_t v, int k) {
    float2 r = make_float2(0.f, 0.f);
    if (k < g.d) r.x = emb_f32(g.vemb, g.dtype, v, g.d, k);
    if (k + 1 < g.d) r.y = emb_f32(g.vemb, g.dtype, v, g.d, k + 1);
    return r;
}

__device__ __forceinline__ void split_pair(float2 p, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 hx = __float2bfloat16_rn(p.x), hy = __float2bfloat16_rn(p.y);
    const float rx = p.x - __bfloat162float(hx), ry = p.y - __bfloat162float(hy);
    hi = static_cast<uint32_t>(__bfloat16_as_ushort(hx)) | (static_cast<uint32_t>(__bfloat16_as_ushort(hy)) << 16);
    lo = pack_bf16x2(rx, ry);
}

__device__ float tc_batch_w2(const DevGraph& g, const uint16_t* __restrict__ wsplit, uint32_t hu, uint32_t hv,
                             uint32_t hr2, int lane) {
    const int gq = lane >> 2, tq = lane & 3;
    const int R = g.R, d = g.d;
    const int64_t rd = static_cast<int64_t>(R) * d;
    float acc[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = acc[a][b][2] = acc[a][b][3] = 0.f;
    uint32_t ru[2][2], rv[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            ru[mt][hlf] = __shfl_sync(0xffffffffu, hu, mt * 16 + gq + 8 * hlf);
            rv[mt][hlf] = __shfl_sync(0xffffffffu, hv, mt * 16 + gq + 8 * hlf);
        }
    for (int kt = 0; kt < (d + 15) / 16; ++kt) {
        const int k = kt * 16 + tq * 2;
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = nt * 8 + gq;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const int kc = k + 8 * kk;
                uint32_t h = 0u, l = 0u;
                if (n < R) {
                    const int64_t i = static_cast<int64_t>(n) * d + kc;
                    const uint32_t h0 = kc < d ? wsplit[i] : 0u, h1 = kc + 1 < d ? wsplit[i + 1] : 0u;
                    const uint32_t l0 = kc < d ? wsplit[rd + i] : 0u, l1 = kc + 1 < d ? wsplit[rd + i + 1] : 0u;
                    h = h0 | (h1 << 16);
                    l = l0 | (l1 << 16);
                }
                bh[nt][kk] = h;
                bl[nt][kk] = l;
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            uint32_t ah[4], al[4];
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                // q4: 0 -> (row g, k), 1 -> (row g+8, k), 2 -> (row g, k+8), 3 -> (row g+8, k+8)
                const int hlf = q4 & 1, kc = k + 8 * (q4 >> 1);
                const float2 a = emb_pair(g, ru[mt][hlf], kc), b = emb_pair(g, rv[mt][hlf], kc);
                split_pair(make_float2(a.x * b.x, a.y * b.y), ah[q4], al[q4]);
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma_bf16_16816(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bh[nt][0], bh[nt][1]);
                mma_bf16_16816(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bl[nt][0], bl[nt][1]);
                mma_bf16_16816(acc[mt][nt], al[0], al[1], al[2], al[3], bh[nt][0], bh[nt][1]);
            }
        }
    }
    // lane h wants row h, column r2: held by lane ((h % 16) % 8) * 4 + (r2 % 8) / 2,
    // register [h / 16][r2 / 8][((h % 16) / 8) * 2 + r2 % 2]
    const int h = lane;
    const int src = ((h & 15) & 7) * 4 + (static_cast<int>(hr2 & 7) >> 1);
    const int want = (h >> 4) * 8 + (static_cast<int>(hr2 >> 3) & 1) * 4 + ((h & 15) >> 3) * 2 + static_cast<int>(hr2 & 1);
    float w = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float v = __shfl_sync(0xffffffffu, acc[mt][nt][j], src);
                if (want == mt * 8 + nt * 4 + j) w = v;
            }
    return w;
}

// Thread 0 of a join CTA: the next work item of its own contiguous range, else
// of the following ranges (stealing).  A bit map marks ranges found drained so
// that a thief skips up to 32 of them with one read.
__device__ __forceinline__ int64_t take_item(const PlanDev* __restrict__ P, int64_t total_items, int& victim,
                                             unsigned long long& probes) {
    const int grid = static_cast<int>(gridDim.x);
    while (victim < grid) {
        const int v = (static_cast<int>(blockIdx.x) + victim) % grid;
        if (victim > 0) {
            const uint32_t w = __ldcg(P->drained + (v >> 5)) >> (v & 31);
            if (w & 1u) {
                // bits at and above `grid` are never set, so the run stays inside [v, grid)
                const uint32_t nw = ~w;
                victim += nw ? __ffs(nw) - 1 : 32 - (v & 31);
                continue;
            }
        }
        ++probes;
        const int64_t lo = total_items * v / grid;
        const int64_t hi = total_items * (v + 1) / grid;
        if (lo < hi) {
            const int64_t idx = static_cast<int64_t>(atomicAdd(&P->cursors[v], 1ull));
            if (lo + idx < hi) return lo + idx;
        }
        atomicOr(&P->drained[v >> 5], 1u << (v & 31));
        ++victim;
    }
    return total_items;
}

// Takes the next work item that cannot be skipped and prepares it.  An item is
// skipped without touching the CTA's query state when its query is being
// recomputed exactly, when the seed launch did all of it, or when no row of it
// can reach the query's kept band.  Run by one thread at a time.
template <bool SEED>
__device__ void select_item(MidSmem& sm, const PlanDev* __restrict__ P, int nq, bool prune, ItemSel& out,
                            unsigned long long& iters, unsigned long long& probes) {
    const int64_t total_items = sm.total_items;
    out.item = total_items;
    out.q = -1;
    for (;;) {
        ++iters;
        int64_t it = total_items;
        if (SEED) {
            // one item per seeded query: its first one
            if (prune) {
                for (;;) {
                    const int qq = static_cast<int>(atomicAdd(&P->counters[kCntSeed], 1ull));
                    if (qq >= nq) break;
                    if (seeded_query(P, qq, prune)) {
                        it = P->item_off[qq];
                        break;
                    }
                }
            }
        } else {
            it = take_item(P, total_items, sm.victim, probes);
        }
        if (it >= total_items) return;
        const uint4 dsc = P->item_desc[it];
        const uint32_t ub = P->item_ub[it];
        const int iq = static_cast<int>(dsc.x & 0x7fffffffu);
        const bool seeded = (dsc.x >> 31) != 0u;
        const int64_t li = dsc.w;
        const int dense = __ldcg(P->dense + iq);
        uint32_t gk = __ldcg(P->thr_g + iq);
        const int64_t s_near = P->s_near[iq];
        const uint32_t lt = *reinterpret_cast<volatile uint32_t*>(&sm.lt_key);
        if (iq == *reinterpret_cast<volatile int*>(&sm.q) && lt > gk) gk = lt;
        const int64_t chunk = P->chunk;
        const int64_t first = min(chunk, s_near);  // edges of the query's first item
        bool skip = dense != 0;
        if (!SEED && prune && !skip) {
            if (li == 0 && seeded && first <= kSeedEdges) {
                skip = true;  // the seed launch did all of it
            } else if (gk != 0u && __fadd_ru(key2f(ub), P->prune_slack) < keep_threshold(gk, sm.two_err)) {
                skip = true;
                atomicAdd(&sm.c_skipped, 1ull);
            }
        }
        if (skip) continue;
        int64_t e0 = li * chunk, e1 = min(e0 + chunk, s_near);
        uint32_t k0 = dsc.y, k1 = dsc.z;
        if (li == 0 && seeded && first > kSeedEdges) {
            const uint2 sk = P->seed_k[iq];
            if (SEED) {
                e1 = kSeedEdges;  // last edge kSeedEdges - 1
                k1 = sk.x;
            } else {
                e0 = kSeedEdges;  // first edge kSeedEdges
                k0 = sk.y;
            }
        }
        out.item = it;
        out.q = iq;
        out.e0 = static_cast<uint32_t>(e0);
        out.e1 = static_cast<uint32_t>(e1);
        out.k0 = k0;
        out.k1 = k1;
        out.gk = gk;
        out.ub = ub;
        return;
    }
}

// SEED: with bound pruning on, a first launch processes only the first work
// item of every query (its highest-bound rows when rows are ordered), so the
// shared K-th score of every query is set before the main launch starts.
template <int UNROLL, bool SEED, bool TC>
__global__ void __launch_bounds__(kMidThreads, 1) k_middle(const PlanDev* __restrict__ P, DevGraph g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MidSmem& sm = *reinterpret_cast<MidSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = P->K;
    const int nq = P->nq;
    const int sigma = P->sigma;
    Hit* hits = P->hits + static_cast<int64_t>(blockIdx.x) * kMaxChunk;
    uint32_t n_paths_w = 0, n_pruned = 0;  // per lane
    const bool prune = P->prune != 0;
    const float slack = P->prune_slack;
    if (SEED && !prune) return;
#ifdef MHR_PHASE_TIMING
    // cycles per phase, thread 0: 0 fetch + query switch, 1 item setup, 2 scan, 3 score
    unsigned long long ph[4] = {0, 0, 0, 0};
    unsigned long long tph = clock64();
#define MHR_PHASE(i)                                  \
    do {                                              \
        if (threadIdx.x == 0) {                       \
            const unsigned long long now__ = clock64(); \
            ph[i] += now__ - tph;                     \
            tph = now__;                              \
        }                                             \
    } while (0)
    // per warp: own cycles in the scan and score loops (before the closing barrier);
    // thread 0: items taken, fetch-loop iterations, ranges probed, query switches
    unsigned long long wt_scan = 0, wt_score = 0, t_w = 0;
    unsigned long long c_items = 0, c_iter = 0, c_probe = 0, c_switch = 0;
#define MHR_WSTART() (t_w = clock64())
#define MHR_WEND(acc) ((acc) += clock64() - t_w)
#define MHR_COUNT(c) (++(c))
    unsigned long long t_sub = 0;
    unsigned long long subc[6] = {0, 0, 0, 0, 0, 0};  // this warp's cycles of the sub-phases (lane 0)
#define MHR_SUB_START() (t_sub = clock64())
#define MHR_SUB(i)                                               \
    do {                                                         \
        const unsigned long long now__ = clock64();              \
        if (lane == 0) subc[i] += now__ - t_sub;                 \
        t_sub = now__;                                           \
    } while (0)
#else
#define MHR_PHASE(i) \
    do {             \
    } while (0)
#define MHR_WSTART() ((void)0)
#define MHR_WEND(acc) ((void)0)
#define MHR_COUNT(c) ((void)0)
#define MHR_SUB_START() ((void)0)
#define MHR_SUB(i) ((void)0)
#endif
    int cur_q = -1;
    if (threadIdx.x == 0) {
        sm.q = -1;
        sm.two_err = 2.0 * P->err_path;
        sm.total_items = P->item_off[nq];
        sm.c_scanned = sm.c_hits = sm.c_cands = sm.c_skipped = 0ull;
        sm.victim = 0;
        sm.nx_ready = 0;
    }
    // fast hit scorer: fp32 rows of at most 2G vectors per lane group
    const int vec4 = g.d / 4;
    const bool fast = g.dtype == MHR_F32 && (g.d & 3) == 0 && vec4 <= kHitVecs * P->hit_width;
    // the same for bf16 rows (16-byte vectors of eight values)
    const int vec8 = g.d / 8;
    const bool fastb = g.dtype == MHR_BF16 && (g.d & 7) == 0 && vec8 <= kHitVecs * P->hit_width;
    const int relvecs = fast ? g.R * vec4 : (fastb ? g.R * vec8 : kRelCacheVecs + 1);
    const bool relc_ok = relvecs <= kRelCacheVecs;
    if (relc_ok)
        for (int i = threadIdx.x; i < relvecs; i += blockDim.x)
            sm.relc[i] = reinterpret_cast<const float4*>(g.remb)[i];
    // (the first __syncthreads of the item loop publishes the cache)

    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long iters = 0, probes = 0;
            ItemSel sel;
            bool have = false;
            if (!SEED && sm.nx_ready) {
                // the item taken during the last score phase, unless the band rose past it since
                sm.nx_ready = 0;
                sel = sm.nx;
                have = true;
                if (prune && sel.item < sm.total_items) {
                    uint32_t gk = sel.gk;
                    if (sel.q == sm.q && sm.lt_key > gk) gk = sm.lt_key;
                    if (gk != 0u && __fadd_ru(key2f(sel.ub), P->prune_slack) < keep_threshold(gk, sm.two_err)) {
                        ++sm.c_skipped;
                        have = false;
                    } else {
                        sel.gk = gk;
                    }
                }
            }
            if (!have) select_item<SEED>(sm, P, nq, prune, sel, iters, probes);
#ifdef MHR_PHASE_TIMING
            c_iter += iters;
            c_probe += probes;
#endif
            sm.item = sel.item;
            sm.item_q = sel.q;
            sm.e0 = sel.e0;
            sm.e1 = sel.e1;
            sm.k0 = sel.k0;
            sm.k1 = sel.k1;
            sm.f_gk = sel.gk;
            if (sel.item < sm.total_items) MHR_COUNT(c_items);
        }
        __syncthreads();
        const int64_t item = sm.item;
        if (item >= sm.total_items) break;
        const int q = sm.item_q;
        if (q != cur_q) {
            if (cur_q >= 0) finish_query(sm, P, K);
            setup_query(sm, P, q);
            cur_q = q;
            MHR_COUNT(c_switch);
        }
        MHR_PHASE(0);
        if (threadIdx.x == 0) {
            sm.skip = sm.local_dense;
            const uint32_t gk = sm.f_gk;
            if (gk > sm.lt_key) {
                sm.lt_key = gk;
                sm.thr_keep = keep_threshold(gk, sm.two_err);
            }
            sm.hit_cnt = 0;
            sm.batch_next = 0;
            sm.nx_claim = 0;
        }
        __syncthreads();
        if (sm.skip) continue;

        const uint32_t e0 = sm.e0, e1 = sm.e1;
        const int ngroups = static_cast<int>((e1 - e0 + 31) / 32);
        const int near_cnt = sm.near_cnt;
        const uint2* nearP = P->nearP + sm.near_base;
        const float* nearB = P->nearB + sm.near_base;
        const uint32_t s_near32 = static_cast<uint32_t>(sm.s_near);
        const float thr_scan = sm.thr_keep;
        // --- group -> owning near entry (+1) and, for a group inside one near row,
        // the CSR position of its first edge (or a marker: several rows, pruned)
        const uint32_t k0 = sm.k0, k1 = sm.k1;
        if (k1 - k0 < 63u) {
            // At most 63 near rows: every warp holds their prefixes in registers
            // (entry k0 + j at lane j % 32, register j / 32) and each thread finds
            // the row of its group by a search over them.
            const uint32_t nent = k1 - k0 + 1u;
            uint32_t pA = 0xffffffffu, pB = 0xffffffffu, rA = 0u, rB = 0u;
            float bA = 0.f, bB = 0.f;
            if (static_cast<uint32_t>(lane) < nent) {
                const uint2 t = nearP[k0 + lane];
                pA = t.x;
                rA = t.y;
                if (prune) bA = nearB[k0 + lane];
            }
            if (static_cast<uint32_t>(lane) + 32u < nent) {
                const uint2 t = nearP[k0 + 32u + lane];
                pB = t.x;
                rB = t.y;
                if (prune) bB = nearB[k0 + 32u + lane];
            }
            const int gidx = threadIdx.x;  // one group per thread (ngroups <= blockDim.x)
            const uint32_t gs = e0 + 32u * static_cast<uint32_t>(gidx);
            // pos = number of rows whose prefix is <= gs (>= 1: row k0 holds e0)
            int pos = 0;
#pragma unroll
            for (int step = 32; step > 0; step >>= 1) {
                const int j = pos + step - 1;
                const uint32_t va = __shfl_sync(FULL, pA, j & 31), vb = __shfl_sync(FULL, pB, j & 31);
                if ((j < 32 ? va : vb) <= gs) pos += step;
            }
            const int jr = pos - 1, jn = pos;
            const uint32_t ra = __shfl_sync(FULL, rA, jr & 31), rb2 = __shfl_sync(FULL, rB, jr & 31);
            const uint32_t pa = __shfl_sync(FULL, pA, jr & 31), pb = __shfl_sync(FULL, pB, jr & 31);
            const float ba = __shfl_sync(FULL, bA, jr & 31), bb = __shfl_sync(FULL, bB, jr & 31);
            const uint32_t na = __shfl_sync(FULL, pA, jn & 31), nb = __shfl_sync(FULL, pB, jn & 31);
            if (gidx < ngroups) {
                const uint32_t rowstart = jr < 32 ? ra : rb2, pre = jr < 32 ? pa : pb;
                const float rowb = jr < 32 ? ba : bb;
                // the row after it starts at the next prefix; the item's last row reaches e1
                const uint32_t nxt = static_cast<uint32_t>(jn) < nent ? (jn < 32 ? na : nb) : 0xffffffffu;
                const uint32_t ge = min(gs + 32u, e1);
                uint32_t gp = kGposMulti;
                if (ge <= nxt) {
                    gp = rowstart + (gs - pre);
                    if (prune && __fadd_ru(rowb, slack) < thr_scan) gp = kGposPruned;
                }
                sm.gmap[gidx] = k0 + static_cast<uint32_t>(jr) + 1u;
                sm.gpos[gidx] = gp;
            }
        } else {
            // by marking group starts, then a prefix max
            for (int i = threadIdx.x; i < ngroups; i += blockDim.x) sm.gmap[i] = 0u;
            __syncthreads();
            for (uint32_t k = k0 + threadIdx.x; k <= k1; k += blockDim.x) {
                const uint32_t pk = nearP[k].x;
                const uint32_t pk1 = (k + 1 < static_cast<uint32_t>(near_cnt)) ? nearP[k + 1].x : s_near32;
                const uint32_t lo = max(pk, e0), hi = min(pk1, e1);
                const uint32_t gf = (lo - e0 + 31) / 32;
                if (e0 + 32 * gf < hi) sm.gmap[gf] = k + 1;
            }
            __syncthreads();
            // inclusive prefix max over <= 1024 entries (one per thread)
            uint32_t v = threadIdx.x < ngroups ? sm.gmap[threadIdx.x] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, v, o);
                if (lane >= o) v = max(v, y);
            }
            if (lane == 31) sm.redu[warp] = v;
            __syncthreads();
            if (warp == 0) {
                uint32_t w = sm.redu[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(FULL, w, o);
                    if (lane >= o) w = max(w, y);
                }
                sm.redu[lane] = w;
            }
            __syncthreads();
            if (warp > 0) v = max(v, sm.redu[warp - 1]);
            if (threadIdx.x < ngroups) {
                sm.gmap[threadIdx.x] = v;
                const uint32_t kk = v - 1u;
                const uint32_t gs = e0 + 32u * threadIdx.x;
                const uint32_t ge = min(gs + 32u, e1);
                const uint2 pk = nearP[kk];
                const uint32_t nxt = (kk + 1u < static_cast<uint32_t>(near_cnt)) ? nearP[kk + 1u].x : s_near32;
                uint32_t gp = kGposMulti;
                if (ge <= nxt) {
                    gp = pk.y + (gs - pk.x);
                    if (prune && __fadd_ru(nearB[kk], slack) < thr_scan) gp = kGposPruned;
                }
                sm.gpos[threadIdx.x] = gp;
            }
        }
        __syncthreads();

        MHR_PHASE(1);
        // --- scan: stream near rows, probe the far bitmap, stage hits
        const uint32_t* colsrc = sm.dir ? g.col : g.rcol;
        const ListEnt* far = P->list + sm.far_base;
        const uint4* far_start = P->far_start + static_cast<int64_t>(blockIdx.x) * P->far_cap;
        const uint16_t* relsrc = sm.dir ? g.rel : g.rrel;
        MHR_WSTART();
        for (int gb = warp * UNROLL; gb < ngroups; gb += kMidWarps * UNROLL) {
            MHR_SUB_START();
            uint2 ne[UNROLL];
            uint32_t kk[UNROLL], gp[UNROLL];
            float rb[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int gidx = gb + u;
                ne[u] = make_uint2(s_near32, 0u);
                kk[u] = 0;
                gp[u] = kGposPruned;
                rb[u] = 0.f;
                if (gidx < ngroups) {
                    kk[u] = sm.gmap[gidx] - 1u;
                    gp[u] = sm.gpos[gidx];
                    const uint32_t idx = kk[u] + lane;
                    // rows of a group spanning several near rows: 32 row starts from kk on
                    if (gp[u] == kGposMulti && idx < static_cast<uint32_t>(near_cnt)) {
                        ne[u] = nearP[idx];
                        if (prune) rb[u] = nearB[idx];
                    }
                }
            }
            uint32_t xv[UNROLL], rv[UNROLL], epos[UNROLL], nk[UNROLL];
            bool valid[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int gidx = gb + u;
                valid[u] = false;
                xv[u] = 0;
                rv[u] = 0;
                epos[u] = 0;
                nk[u] = 0;
                if (gidx < ngroups) {
                    const uint32_t gs = e0 + 32u * gidx;
                    const uint32_t e = gs + lane;
                    valid[u] = e < e1;
                    if (gp[u] == kGposMulti) {  // warp-uniform
                        // lane -> its row: count the row starts in (gs, e]
                        const uint32_t pos = ne[u].x - gs;
                        const uint32_t bit = (lane >= 1 && pos >= 1 && pos <= 31) ? (1u << pos) : 0u;
                        const uint32_t mask = __reduce_or_sync(FULL, bit);
                        const int c = __popc(mask & lanemask_le());
                        const uint32_t pm = __shfl_sync(FULL, ne[u].x, c);
                        const uint32_t rs = __shfl_sync(FULL, ne[u].y, c);
                        if (prune) {
                            // no path through this row can reach the kept band: skip its edges
                            const float rowb = __fadd_ru(__shfl_sync(FULL, rb[u], c), slack);
                            if (valid[u] && rowb < thr_scan) {
                                valid[u] = false;
                                ++n_pruned;
                            }
                        }
                        epos[u] = rs + (e - pm);
                        nk[u] = kk[u] + c;
                    } else if (gp[u] == kGposPruned) {
                        if (valid[u]) ++n_pruned;
                        valid[u] = false;
                        nk[u] = kk[u];
                    } else {
                        epos[u] = gp[u] + lane;
                        nk[u] = kk[u];
                    }
                }
            }
            MHR_SUB(0);
            // far vertex and relation of every edge (the relation travels with a hit)
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                if (valid[u]) {
                    xv[u] = __ldg(colsrc + epos[u]);
                    rv[u] = __ldg(relsrc + epos[u]);
                }
            // Membership of the UNROLL groups' far vertices, in passes whose
            // loads do not depend on one another across groups, so a warp has
            // all of them in flight at once: bitmap bit (and, for an exact
            // bitmap, its rank: the far-list index) in shared memory, then for a
            // coarse bitmap the set bit's run in the far list from the run
            // table (global), then the rare walk along the run.
            bool hit[UNROLL];
            uint32_t fk[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                hit[u] = false;
                fk[u] = 0;
                if (valid[u]) {
                    const uint32_t x = xv[u];
                    const uint32_t bv = x >> sigma;
                    if ((sm.bm[bv >> 5] >> (bv & 31u)) & 1u) {
                        hit[u] = true;
                        // exact bitmap: the rank of x is its far-list index;
                        // coarse: the bit indexes the run table
                        fk[u] = sigma == 0 ? bm_rank(sm, x) : bv;
                    }
                }
            }
            if (sigma > 0) {
                // coarse bitmap: far_start[bit] (written by this CTA's query set-up:
                // a coherent load) holds the set bit's run in the far list: first
                // entry and vertex, last vertex and entry.  x equal to either end is
                // a hit, x outside them a miss; only x strictly inside a run of three
                // or more walks the run.
                bool walk[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    walk[u] = false;
                    if (hit[u]) {
                        const uint4 st = far_start[fk[u]];
                        const uint32_t x = xv[u];
                        walk[u] = st.y < x && x < st.z;
                        hit[u] = x == st.y || x == st.z;
                        fk[u] = x == st.z ? st.w : st.x;
                    }
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    if (!walk[u]) continue;
                    const uint32_t x = xv[u];
                    uint32_t k = fk[u], v = 0u;
                    do {
                        v = far[++k].vertex;
                    } while (v < x);
                    hit[u] = v == x;
                    fk[u] = k;
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int gidx = gb + u;
                if (gidx >= ngroups) break;
                const unsigned b = __ballot_sync(FULL, hit[u]);
                if (b) {
                    int base = 0;
                    const int leader = __ffs(b) - 1;
                    if (lane == leader) base = atomicAdd(&sm.hit_cnt, __popc(b));
                    base = __shfl_sync(FULL, base, leader);
                    if (hit[u]) {
                        Hit h;
                        h.near_k = nk[u];
                        h.far_k = fk[u];
                        h.r2 = rv[u];
                        hits[base + __popc(b & lanemask_lt())] = h;
                    }
                }
            }
            MHR_SUB(1);
        }
        MHR_WEND(wt_scan);
        if (threadIdx.x == 0) sm.round_cnt = sm.cand_cnt;
        __syncthreads();
        MHR_PHASE(2);
        const int nh = sm.hit_cnt;
        if (threadIdx.x == 0) {
            sm.c_scanned += e1 - e0;
            sm.c_hits += static_cast<unsigned long long>(nh);
        }

        // --- score hits; keep paths that can still reach the top K.
        // A warp takes batches of 32 hits: one lane loads each hit's frontier
        // entries, then groups of G lanes score H = 32 / G hits at a time over
        // G rounds, so every warp keeps H hits' embedding rows in flight.
        const ListEnt* nearL = P->nearL + sm.near_base;  // ordered position
        const float* w1s = P->w32 + sm.a_base;
        const float* w3s = P->w32 + sm.c_base;
        const int G = P->hit_width, H = 32 / G;
        const int sub = lane & (G - 1);
        int b = 0;                 // current batch of 32 hits (taken from a shared counter)
        bool loaded = false;
        unsigned pend = 0;         // lanes whose hit still has combinations to expand
        uint32_t slice = 0;        // this lane's next combination
        uint32_t hu = 0, hv = 0, hr2 = 0, has = 0, hal = 0, hcs = 0, hcl = 0, hnk = 0;
        float hw2 = 0.f, hm1 = 0.f, hm3 = 0.f;  // middle-edge weight; run maxima of the hit's u and v
        NearRow nrow;
        nrow.id = 0xffffffffu;
        for (;;) {
            MHR_WSTART();
            const int budget = (kCandCap - sm.round_cnt) / kMidWarps;
            int used = 0;
            bool done = true;
            if (!sm.local_dense) {
                const float thr = sm.thr_keep;
                for (;;) {
                    if (!loaded) {
                        if (lane == 0) b = atomicAdd(&sm.batch_next, 1);
                        b = __shfl_sync(FULL, b, 0);
                        const int hb = b * 32;
                        if (hb >= nh) {
                            // The first warp to find no batch left takes the next work
                            // item while the other warps finish their last batches.
                            if (!SEED && lane == 0 && atomicCAS(&sm.nx_claim, 0, 1) == 0) {
                                unsigned long long iters = 0, probes = 0;
                                select_item<SEED>(sm, P, nq, prune, sm.nx, iters, probes);
                                sm.nx_ready = 1;
                            }
                            break;
                        }
                        MHR_SUB_START();
                        const int hi = hb + lane;
                        const bool live = hi < nh;
                        float mw1 = 0.f, mw3 = 0.f;
                        hu = hv = hr2 = 0;
                        has = hal = hcs = hcl = 0;
                        bool alive = false;
                        if (live) {
                            const Hit ht = hits[hi];
                            hnk = ht.near_k;
                            const ListEnt ne = nearL[ht.near_k];
                            const ListEnt fe = far[ht.far_k];
                            const ListEnt& ea = sm.dir ? ne : fe;  // hop-1 side (u)
                            const ListEnt& ec = sm.dir ? fe : ne;  // hop-3 side (v)
                            hu = ea.vertex;
                            hv = ec.vertex;
                            hr2 = ht.r2;
                            has = ea.run_start;
                            hal = ea.run_len;
                            hcs = ec.run_start;
                            hcl = ec.run_len;
                            mw1 = ea.maxw;
                            mw3 = ec.maxw;
                            alive = true;
                            if (P->cons && !P->cons[g.R + hr2]) {
                                // constrained query: a disallowed middle relation ends the hit
                                alive = false;
                                hal = 0;
                            }
                            n_paths_w += hal * hcl;
                            if (prune && alive) {
                                // w2 <= the largest weight of any out-edge of u and of any in-edge of v,
                                // and of those of relation r2 when the graph keeps that table
                                const float mw2 = fminf(ea.midw, ec.midw);
                                if (__fadd_ru(__fadd_rn(__fadd_rn(mw1, mw2), mw3), slack) < thr) {
                                    alive = false;
                                    ++n_pruned;
                                } else if (g.maxw_out_r) {
                                    const float mr = fminf(g.maxw_out_r[static_cast<int64_t>(hu) * g.R + hr2],
                                                           g.maxw_in_r[static_cast<int64_t>(hv) * g.R + hr2]);
                                    if (__fadd_ru(__fadd_rn(__fadd_rn(mw1, mr), mw3), slack) < thr) {
                                        alive = false;
                                        ++n_pruned;
                                    }
                                }
                            }
                        }
                        // move the surviving hits to the low lanes
                        MHR_SUB(2);
                        const unsigned am = __ballot_sync(FULL, alive);
                        const int nsurv = __popc(am);
                        if (prune) {
                            if (alive) sm.compact[warp][__popc(am & lanemask_lt())] = static_cast<uint8_t>(lane);
                            __syncwarp();
                            const int src = lane < nsurv ? sm.compact[warp][lane] : lane;
                            __syncwarp();
                            hu = __shfl_sync(FULL, hu, src);
                            hv = __shfl_sync(FULL, hv, src);
                            hr2 = __shfl_sync(FULL, hr2, src);
                            has = __shfl_sync(FULL, has, src);
                            hal = __shfl_sync(FULL, hal, src);
                            hcs = __shfl_sync(FULL, hcs, src);
                            hcl = __shfl_sync(FULL, hcl, src);
                            mw1 = __shfl_sync(FULL, mw1, src);
                            mw3 = __shfl_sync(FULL, mw3, src);
                        }
                        const bool live2 = prune ? (lane < nsurv) : live;
                        const int rounds = prune ? (nsurv + H - 1) / H : G;
                        float w2m = 0.f;
                        if (TC) {
                            w2m = tc_batch_w2(g, P->wsplit, hu, hv, hr2, lane);
                        } else
                        for (int r = 0; r < rounds; ++r) {
                            const int src = r * H + lane / G;
                            const uint32_t u = __shfl_sync(FULL, hu, src);
                            const uint32_t v = __shfl_sync(FULL, hv, src);
                            const uint32_t rr = __shfl_sync(FULL, hr2, src);
                            float w;
                            if (fast) {
                                const bool fwd = sm.dir != 0;
                                w = hit_w32_f32(g, nrow, fwd ? u : v, fwd ? v : u, rr, fwd, sub, G, vec4,
                                                relc_ok ? sm.relc : nullptr);
                            } else if (fastb) {
                                const bool fwd = sm.dir != 0;
                                w = hit_w32_bf16(g, nrow, fwd ? u : v, fwd ? v : u, rr, fwd, sub, G, vec8,
                                                 relc_ok ? sm.relc : nullptr);
                            } else {
                                w = edge_w32_group(g, u, rr, v, sub, G);
                            }
                            const float tw = __shfl_sync(FULL, w, ((lane - r * H) & (H - 1)) * G);
                            if (lane / H == r) w2m = tw;
                        }
                        hw2 = w2m;
                        hm1 = mw1;
                        hm3 = mw3;
                        // a hit with no combination (disallowed middle relation) stays out
                        if (hal == 0u) hw2 = neg_inf();
                        MHR_SUB(3);
                        const float smax = __fadd_rn(__fadd_rn(mw1, hw2), mw3);
                        // training labels (plain runs only): best path score through the near entry
                        if (P->label && live2) atomicMax(&P->ubest[sm.near_base + hnk], f2key(smax));
                        pend = __ballot_sync(FULL, live2 && hal != 0u && smax >= thr);
                        loaded = true;
                        slice = 0;
                    }
                    // The (r1, r3) combinations of the pending hits, flattened: lane h's
                    // remaining combinations take positions [excl, excl + rem) of one
                    // sequence that the warp walks 32 at a time, so a hit with many
                    // parallel edges does not serialise the warp.
                    bool stop = false;
                    const bool mine0 = (pend >> lane) & 1u;
                    if (__all_sync(FULL, !mine0 || (hal * hcl == 1u && slice == 0u))) {
                        // Every pending hit has one combination (runs of one edge on both
                        // sides, the common case): its path score is the hit's smax, which
                        // already passed the threshold.  One candidate per pending lane.
                        const int np = __popc(pend);
                        if (used + np > budget) {
                            stop = true;
                        } else if (np) {
                            int base = 0;
                            const int leader = __ffs(pend) - 1;
                            if (lane == leader) base = atomicAdd(&sm.cand_cnt, np);
                            base = __shfl_sync(FULL, base, leader);
                            if (mine0) {
                                Cand cd;
                                cd.s32 = __fadd_rn(__fadd_rn(hm1, hw2), hm3);
                                cd.a_idx = has;
                                cd.c_idx = hcs;
                                cd.r2 = static_cast<uint16_t>(hr2);
                                cd.pad = 0;
                                sm.cand[base + __popc(pend & lanemask_lt())] = cd;
                            }
                            used += np;
                            pend = 0u;
                        }
                    } else {
                        const bool mine = mine0;
                        const uint32_t ncomb = hal * hcl;
                        const uint32_t rem = mine ? ncomb - slice : 0u;
                        uint32_t incl = rem;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(FULL, incl, o);
                            if (lane >= o) incl += y;
                        }
                        const uint32_t total = __shfl_sync(FULL, incl, 31);
                        const uint32_t excl = incl - rem;
                        uint32_t c0 = 0;
                        for (; c0 < total; c0 += 32) {
                            const uint32_t f = c0 + lane;
                            // owner of position f: the number of lanes whose inclusive prefix is <= f
                            int own = 0;
#pragma unroll
                            for (int step = 16; step > 0; step >>= 1) {
                                const uint32_t pv = __shfl_sync(FULL, incl, own + step - 1);
                                if (pv <= f) own += step;
                            }
                            const uint32_t o_excl = __shfl_sync(FULL, excl, own);
                            const uint32_t o_slice = __shfl_sync(FULL, slice, own);
                            const uint32_t o_hcl = __shfl_sync(FULL, hcl, own);
                            const uint32_t o_has = __shfl_sync(FULL, has, own);
                            const uint32_t o_hcs = __shfl_sync(FULL, hcs, own);
                            const uint32_t o_r2 = __shfl_sync(FULL, hr2, own);
                            const float o_w2 = __shfl_sync(FULL, hw2, own);
                            // a run of one edge: its weight is the run's maximum (no slot load)
                            const uint32_t o_hal = __shfl_sync(FULL, hal, own);
                            const float o_m1 = __shfl_sync(FULL, hm1, own);
                            const float o_m3 = __shfl_sync(FULL, hm3, own);
                            bool keep = false;
                            Cand cd;
                            if (f < total) {
                                const uint32_t sl = o_slice + (f - o_excl);
                                uint32_t i = sl, j = 0;
                                if (o_hcl != 1) {
                                    i = sl / o_hcl;
                                    j = sl - i * o_hcl;
                                }
                                const float w1 = o_hal == 1u ? o_m1 : w1s[o_has + i];
                                const float w3 = o_hcl == 1u ? o_m3 : w3s[o_hcs + j];
                                const float s32 = __fadd_rn(__fadd_rn(w1, o_w2), w3);
                                // -inf: a slot of a disallowed relation (constrained queries)
                                keep = s32 >= thr && s32 != neg_inf();
                                cd.s32 = s32;
                                cd.a_idx = o_has + i;
                                cd.c_idx = o_hcs + j;
                                cd.r2 = static_cast<uint16_t>(o_r2);
                                cd.pad = 0;
                            }
                            const unsigned bal = __ballot_sync(FULL, keep);
                            const int nk2 = __popc(bal);
                            if (used + nk2 > budget) {
                                stop = true;
                                break;
                            }
                            if (nk2) {
                                int base = 0;
                                const int leader = __ffs(bal) - 1;
                                if (lane == leader) base = atomicAdd(&sm.cand_cnt, nk2);
                                base = __shfl_sync(FULL, base, leader);
                                if (keep) sm.cand[base + __popc(bal & lanemask_lt())] = cd;
                            }
                            used += nk2;
                        }
                        // positions [0, c0) are done
                        if (mine) slice += c0 > excl ? min(c0 - excl, rem) : 0u;
                        pend = __ballot_sync(FULL, mine && slice < ncomb);
                    }
                    MHR_SUB(4);
                    if (stop) {
                        done = false;
                        break;
                    }
                    loaded = false;
                }
            }
            MHR_WEND(wt_score);
            if (!__syncthreads_or(done ? 0 : 1)) break;
            flush_cands(sm, P, K);
        }
        __syncthreads();
        if (!sm.local_dense && (sm.lt_key == 0u ? sm.cand_cnt >= K : sm.cand_cnt > kCandCap / 2))
            flush_cands(sm, P, K);
        MHR_PHASE(3);
    }
    if (cur_q >= 0) finish_query(sm, P, K);
    MHR_PHASE(0);
#ifdef MHR_PHASE_TIMING
    if (threadIdx.x == 0) printf("MHR_PHASE %d %llu %llu %llu %llu\n", blockIdx.x, ph[0], ph[1], ph[2], ph[3]);
    {
        unsigned long long* wr = reinterpret_cast<unsigned long long*>(sm.red);
        __syncthreads();
        if (threadIdx.x < 4) wr[threadIdx.x] = 0ull;
        __syncthreads();
        if (lane == 0) {
            atomicMax(&wr[0], wt_scan);
            atomicAdd(&wr[1], wt_scan);
            atomicMax(&wr[2], wt_score);
            atomicAdd(&wr[3], wt_score);
        }
        __syncthreads();
        __syncthreads();
        if (threadIdx.x < 6) wr[4 + threadIdx.x] = 0ull;
        __syncthreads();
        if (lane == 0)
            for (int i = 0; i < 6; ++i) atomicAdd(&wr[4 + i], subc[i]);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a[6];
            for (int i = 0; i < 6; ++i) a[i] = wr[4 + i];
            printf("MHR_SUB %d %d nearP %llu col_bitmap_hits %llu hit_load %llu w2 %llu combos %llu\n", blockIdx.x,
                   SEED ? 1 : 0, a[0] / kMidWarps, a[1] / kMidWarps, a[2] / kMidWarps, a[3] / kMidWarps,
                   a[4] / kMidWarps);
        }
        if (threadIdx.x == 0)
            printf("MHR_WARPS %d %d items %llu iters %llu probes %llu switches %llu scan_max %llu scan_mean %llu "
                   "score_max %llu score_mean %llu\n",
                   blockIdx.x, SEED ? 1 : 0, c_items, c_iter, c_probe, c_switch, wr[0], wr[1] / kMidWarps, wr[2],
                   wr[3] / kMidWarps);
    }
#endif
    if (threadIdx.x == 0) {
        atomicAdd(&P->counters[kCntScanned], sm.c_scanned);
        atomicAdd(&P->counters[kCntHits], sm.c_hits);
        atomicAdd(&P->counters[kCntCands], sm.c_cands);
        if (sm.c_skipped) atomicAdd(&P->counters[kCntSkippedItems], sm.c_skipped);
    }
    unsigned long long wp = n_pruned, wq = n_paths_w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wp += __shfl_xor_sync(FULL, wp, o);
        wq += __shfl_xor_sync(FULL, wq, o);
    }
    if (lane == 0 && wp) atomicAdd(&P->counters[kCntPruned], wp);
    if (lane == 0 && wq) atomicAdd(&P->counters[kCntPaths], wq);
}

// ===========================================================================
// merge: exact K-th fp32 score, band, fp64 rescoring, final order
// ===========================================================================
__global__ void __launch_bounds__(1024) k_merge1(const PlanDev* __restrict__ P) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t bc[4];
    __shared__ int red[33];
    __shared__ float s_thr;
    const int K = P->K;
    const double two_err = 2.0 * P->err_path;
    for (int q = blockIdx.x; q < P->nq; q += gridDim.x) {
        if (P->status[q] != 0 || P->dense[q] != 0) continue;
        const int pc = P->pool_cnt[q];
        if (pc > P->pq) continue;
        const Cand* pool = P->pool + static_cast<int64_t>(q) * P->pq;
        if (threadIdx.x == 0) s_thr = neg_inf();
        __syncthreads();
        if (pc >= K) {
            const uint32_t key = block_select_kth([&](int64_t i) { return f2key(pool[i].s32); }, pc, K, hist, bc);
            if (threadIdx.x == 0) s_thr = keep_threshold(key, two_err);
        }
        __syncthreads();
        const float thr = s_thr;
        Cand* band = P->band_cand + static_cast<int64_t>(q) * P->band_cap;
        int w = 0;
        for (int base = 0; base < pc; base += blockDim.x) {
            const int i = base + threadIdx.x;
            bool keep = false;
            Cand c;
            if (i < pc) {
                c = pool[i];
                keep = c.s32 >= thr;
            }
            int tot;
            const int pos = block_excl_scan(keep ? 1 : 0, red, &tot);
            if (keep && w + pos < P->band_cap) band[w + pos] = c;
            w += tot;
        }
        // fp64 sums the band needs: every middle edge, and each hop-1 / hop-3 edge once
        if (w <= P->band_cap) {
            __syncthreads();
            const int64_t a0 = P->a_off[q], c0 = P->totA + P->c_off[q];
            uint32_t* ch = P->chains + static_cast<int64_t>(q) * 3 * P->band_cap;
            int nch = 0;
            for (int base = 0; base < w; base += blockDim.x) {
                const int i = base + threadIdx.x;
                int n = 0;
                bool o1 = false, o3 = false;
                Cand c;
                if (i < w) {
                    c = band[i];
                    o1 = atomicExch(&P->w64own[a0 + c.a_idx], 1) == 0;
                    o3 = atomicExch(&P->w64own[c0 + c.c_idx], 1) == 0;
                    n = 1 + (o1 ? 1 : 0) + (o3 ? 1 : 0);
                }
                int tot;
                int pos = nch + block_excl_scan(n, red, &tot);
                if (i < w) {
                    ch[pos++] = (2u << 30) | static_cast<uint32_t>(i);
                    if (o1) ch[pos++] = (0u << 30) | c.a_idx;
                    if (o3) ch[pos++] = (1u << 30) | c.c_idx;
                }
                nch += tot;
            }
            if (threadIdx.x == 0) P->chain_cnt[q] = nch;
        }
        if (threadIdx.x == 0) {
            if (w > P->band_cap) {
                atomicExch(&P->dense[q], 1);
                P->band_cnt[q] = 0;
                P->chain_cnt[q] = 0;
#ifdef MHR_PHASE_TIMING
                printf("MHR_DENSE band q %d w %d pc %d thr %.6f\n", q, w, pc, thr);
#endif
            } else {
                P->band_cnt[q] = w;
                atomicAdd(&P->counters[kCntRescored], static_cast<unsigned long long>(w));
            }
        }
        __syncthreads();
    }
}

// fp64 rescoring of the band.  The canonical order fixes the accumulation
// acc = acc + y_j (j ascending) of each edge; the terms y_j = |(a_j + b_j) - c_j|
// (or (a_j * b_j) * c_j) are formed from the stored values converted exactly.
// k_merge1 lists the sums a query's band needs (every middle edge; each hop-1
// and hop-3 edge once, however many band entries share it); each lane runs one
// sum straight from the three embedding rows (16-byte loads, several in
// flight), and k_merge2 adds the three weights of every entry.
constexpr int kRsWarps = 4;
#ifndef MHR_RS_LANES
#define MHR_RS_LANES 32
#endif
constexpr int kRsLanes = MHR_RS_LANES;  // sums per warp (the other lanes idle)

// Exact binary32 -> binary64 widening done with integer operations (the value
// is finite: the graph load rejects NaN and infinity), keeping the slow fp64
// pipe for the arithmetic: sign and mantissa move over, the exponent is
// re-biased (1023 - 127 = 896), and a subnormal is first normalised.
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = static_cast<uint64_t>(u >> 31) << 63;
    uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0u) {
        if (m == 0u) return __longlong_as_double(static_cast<long long>(sign));
        const int sh = __clz(m) - 8;  // moves the top set bit to position 23
        m = (m << sh) & 0x7fffffu;
        e = static_cast<uint32_t>(1 - sh);
    }
    const uint64_t bits = sign | (static_cast<uint64_t>(e + 896u) << 52) | (static_cast<uint64_t>(m) << 29);
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ double term1(float a, float b, float c, bool transe) {
    const double x = widen(a), y = widen(b), z = widen(c);
    return transe ? fabs(__dsub_rn(__dadd_rn(x, y), z)) : __dmul_rn(__dmul_rn(x, y), z);
}

__device__ __forceinline__ double acc4(double acc, const float4& a, const float4& b, const float4& c, bool transe) {
    acc = __dadd_rn(acc, term1(a.x, b.x, c.x, transe));
    acc = __dadd_rn(acc, term1(a.y, b.y, c.y, transe));
    acc = __dadd_rn(acc, term1(a.z, b.z, c.z, transe));
    acc = __dadd_rn(acc, term1(a.w, b.w, c.w, transe));
    return acc;
}

// fp64 weight of edge (h, r, t) in the canonical order
__device__ __forceinline__ double edge_w64_seq(const DevGraph& g, uint32_t h, uint32_t r, uint32_t t) {
    const int d = g.d;
    const bool transe = g.fn == MHR_SCORE_TRANSE_L1;
    double acc = 0.0;
    if (g.dtype == MHR_F32 && (d & 3) == 0) {
        const float4* A = reinterpret_cast<const float4*>(static_cast<const float*>(g.vemb) + static_cast<int64_t>(h) * d);
        const float4* B = reinterpret_cast<const float4*>(static_cast<const float*>(g.remb) + static_cast<int64_t>(r) * d);
        const float4* C = reinterpret_cast<const float4*>(static_cast<const float*>(g.vemb) + static_cast<int64_t>(t) * d);
        const int n4 = d >> 2;
#pragma unroll 4
        for (int j = 0; j < n4; ++j) acc = acc4(acc, __ldg(A + j), __ldg(B + j), __ldg(C + j), transe);
    } else {
        for (int j = 0; j < d; ++j)
            acc = __dadd_rn(acc, term1(emb_f32(g.vemb, g.dtype, h, d, j), emb_f32(g.remb, g.dtype, r, d, j),
                                       emb_f32(g.vemb, g.dtype, t, d, j), transe));
    }
    return transe ? __dsub_rn(g.gamma, acc) : acc;
}

__global__ void __launch_bounds__(kRsWarps * 32) k_rescore(const PlanDev* __restrict__ P, DevGraph g) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nq = P->nq, cap = P->band_cap;
    const int64_t gw = blockIdx.x * static_cast<int64_t>(kRsWarps) + w;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kRsWarps;
    // work unit u = (group of kRsLanes sums) * nq + query: the units that have work
    // (the first groups of every query) fill the first warps, spread over all
    // SMs by the small blocks; lane = one sequential fp64 sum
    const int64_t groups_per_q = (3 * static_cast<int64_t>(cap) + kRsLanes - 1) / kRsLanes;
    for (int64_t u = gw; u < static_cast<int64_t>(nq) * groups_per_q; u += nw) {
        const int q = static_cast<int>(u % nq);
        const int i0 = static_cast<int>(u / nq) * kRsLanes;
        const int nc = P->chain_cnt[q];
        if (i0 >= nc || P->dense[q]) continue;
        const int i = i0 + lane;
        if (lane >= kRsLanes || i >= nc) continue;
        const uint32_t chv = P->chains[static_cast<int64_t>(q) * 3 * cap + i];
        const uint32_t kind = chv >> 30, idx = chv & 0x3fffffffu;
        const uint32_t s = P->S[q], t = P->T[q];
        // the edge and where its weight goes; then one converged call for all lanes
        uint32_t h, r, tt;
        double* dst;
        if (kind == 0u) {  // hop-1 edge (s, r1, u)
            const int64_t p1 = g.off[s] + idx;
            h = s;
            r = g.rel[p1];
            tt = g.col[p1];
            dst = P->w64s + P->a_off[q] + idx;
        } else if (kind == 1u) {  // hop-3 edge (v, r3, t)
            const int64_t p3 = g.roff[t] + idx;
            h = g.rcol[p3];
            r = g.rrel[p3];
            tt = t;
            dst = P->w64s + P->totA + P->c_off[q] + idx;
        } else {  // middle edge (u, r2, v) of band entry idx
            const Cand cd = P->band_cand[static_cast<int64_t>(q) * cap + idx];
            h = g.col[g.off[s] + cd.a_idx];
            r = cd.r2;
            tt = g.rcol[g.roff[t] + cd.c_idx];
            dst = P->band_w2 + static_cast<int64_t>(q) * cap + idx;
        }
        *dst = edge_w64_seq(g, h, r, tt);
    }
}

__global__ void __launch_bounds__(1024) k_merge2(const PlanDev* __restrict__ P, DevGraph g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    mhr_path* buf = reinterpret_cast<mhr_path*>(smem_raw);
    const int K = P->K;
    for (int q = blockIdx.x; q < P->nq; q += gridDim.x) {
        if (P->status[q] != 0) {
            if (threadIdx.x == 0) P->n_out[q] = -1;
            continue;
        }
        if (P->dense[q]) continue;
        const int nb = P->band_cnt[q];
        int m = 2;
        while (m < nb) m <<= 1;
        // band entries with their fp64 score (w1 + w2) + w3 in the canonical order
        const Cand* bc = P->band_cand + static_cast<int64_t>(q) * P->band_cap;
        const double* bw2 = P->band_w2 + static_cast<int64_t>(q) * P->band_cap;
        const uint32_t s = P->S[q], t = P->T[q];
        const int64_t a0 = P->a_off[q], c0 = P->totA + P->c_off[q];
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            mhr_path p = worst_path();
            if (i < nb) {
                const Cand cd = bc[i];
                const int64_t p1 = g.off[s] + cd.a_idx, p3 = g.roff[t] + cd.c_idx;
                p.u = g.col[p1];
                p.r1 = g.rel[p1];
                p.v = g.rcol[p3];
                p.r3 = g.rrel[p3];
                p.r2 = cd.r2;
                p.pad = 0;
                p.score = __dadd_rn(__dadd_rn(P->w64s[a0 + cd.a_idx], bw2[i]), P->w64s[c0 + cd.c_idx]);
            }
            buf[i] = p;
        }
        __syncthreads();
        block_sort_paths(buf, m);
        const int nout = min(nb, K);
        mhr_path* dst = P->out + static_cast<int64_t>(q) * K;
        for (int i = threadIdx.x; i < nout; i += blockDim.x) dst[i] = buf[i];
        if (threadIdx.x == 0) P->n_out[q] = nout;
        __syncthreads();
    }
}

// ===========================================================================
// exact path for tie-heavy queries: fp64 keys for every candidate that the
// fp32 screen cannot separate from the running K-th score
// ===========================================================================
constexpr int kExactBuf = 4096;
constexpr int kExactTile = 1024;

struct ExactSmem {
    mhr_path buf[kExactBuf];  // [0, K) top K, [K, ...) staging
    uint32_t hnk[kExactTile], hfk[kExactTile], hep[kExactTile];
    float hw2[kExactTile];
    int64_t hcomb[kExactTile + 1];
    int64_t red[33];
    int nt, ns, hit_cnt;
    double thr64;
};

__device__ void exact_flush(ExactSmem& sm, int K) {
    __syncthreads();
    const int nt = sm.nt, ns = sm.ns;
    for (int i = threadIdx.x; i < kExactBuf; i += blockDim.x) {
        const bool live = (i < nt) || (i >= K && i < K + ns);
        if (!live) sm.buf[i] = worst_path();
    }
    __syncthreads();
    block_sort_paths(sm.buf, kExactBuf);
    if (threadIdx.x == 0) {
        sm.nt = min(K, nt + ns);
        sm.ns = 0;
        if (sm.nt == K) sm.thr64 = sm.buf[K - 1].score;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_exact(const PlanDev* __restrict__ P, DevGraph g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ExactSmem& sm = *reinterpret_cast<ExactSmem*>(smem_raw);
    const int K = P->K;
    const double err = P->err_path;
    for (int q = blockIdx.x; q < P->nq; q += gridDim.x) {
        if (P->status[q] != 0 || !P->dense[q]) continue;
        if (threadIdx.x == 0) {
            sm.nt = 0;
            sm.ns = 0;
            sm.thr64 = __longlong_as_double(0xfff0000000000000ll);
            atomicAdd(&P->counters[kCntDense], 1ull);
        }
        __syncthreads();
        const uint32_t s = P->S[q], t = P->T[q];
        const int dir = P->dir[q];
        const int64_t a_base = P->a_off[q], c_base = P->totA + P->c_off[q];
        const int64_t nb = dir ? a_base : c_base, fb = dir ? c_base : a_base;
        const int near_cnt = P->near_cnt[q], far_cnt = P->far_cnt[q];
        const int64_t s_near = P->s_near[q];
        const uint2* nearP = P->nearP + nb;
        const ListEnt* nearL = P->list + nb;
        const uint32_t* nperm = P->nperm + nb;  // ordered position -> list entry
        const ListEnt* far = P->list + fb;
        const uint32_t* colsrc = dir ? g.col : g.rcol;
        const uint16_t* relsrc = dir ? g.rel : g.rrel;
        for (int64_t eb = 0; eb < s_near; eb += kExactTile) {
            if (threadIdx.x == 0) sm.hit_cnt = 0;
            __syncthreads();
            const int64_t e = eb + threadIdx.x;
            if (e < s_near) {
                int lo = 0, hi = near_cnt;
                while (lo + 1 < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (static_cast<int64_t>(nearP[mid].x) <= e) lo = mid;
                    else hi = mid;
                }
                const uint32_t ep = nearP[lo].y + static_cast<uint32_t>(e - nearP[lo].x);
                const uint32_t x = colsrc[ep];
                int a = 0, b = far_cnt;
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if (far[mid].vertex < x) a = mid + 1;
                    else b = mid;
                }
                if (a < far_cnt && far[a].vertex == x) {
                    const ListEnt& ne = nearL[nperm[lo]];
                    const ListEnt& fe = far[a];
                    const ListEnt& ea = dir ? ne : fe;
                    const ListEnt& ec = dir ? fe : ne;
                    const int slot = atomicAdd(&sm.hit_cnt, 1);
                    sm.hnk[slot] = lo;
                    sm.hfk[slot] = a;
                    sm.hep[slot] = ep;
                    const uint32_t r2 = relsrc[ep];
                    sm.hw2[slot] = (P->cons && !P->cons[g.R + r2]) ? neg_inf()
                                                                   : edge_w32_group(g, ea.vertex, r2, ec.vertex, 0, 1);
                }
            }
            __syncthreads();
            const int nh = sm.hit_cnt;
            int64_t comb = 0;
            if (threadIdx.x < nh) {
                const ListEnt& ne = nearL[nperm[sm.hnk[threadIdx.x]]];
                const ListEnt& fe = far[sm.hfk[threadIdx.x]];
                comb = static_cast<int64_t>(ne.run_len) * fe.run_len;
            }
            int64_t tot;
            const int64_t ex = block_excl_scan(comb, sm.red, &tot);
            if (threadIdx.x < nh) sm.hcomb[threadIdx.x] = ex;
            if (threadIdx.x == 0) sm.hcomb[nh] = tot;
            __syncthreads();
            for (int64_t cb = 0; cb < tot; cb += blockDim.x) {
                if (sm.ns + static_cast<int>(blockDim.x) > kExactBuf - K) exact_flush(sm, K);
                const int64_t c = cb + threadIdx.x;
                if (c < tot) {
                    int lo = 0, hi = nh;  // largest h with hcomb[h] <= c
                    while (lo + 1 < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sm.hcomb[mid] <= c) lo = mid;
                        else hi = mid;
                    }
                    const ListEnt& ne = nearL[nperm[sm.hnk[lo]]];
                    const ListEnt& fe = far[sm.hfk[lo]];
                    const ListEnt& ea = dir ? ne : fe;
                    const ListEnt& ec = dir ? fe : ne;
                    const int64_t local = c - sm.hcomb[lo];
                    const uint32_t i = static_cast<uint32_t>(local / ec.run_len);
                    const uint32_t j = static_cast<uint32_t>(local - static_cast<int64_t>(i) * ec.run_len);
                    const float w1 = P->w32[a_base + ea.run_start + i];
                    const float w3 = P->w32[c_base + ec.run_start + j];
                    const float s32 = __fadd_rn(__fadd_rn(w1, sm.hw2[lo]), w3);
                    const double thr = sm.thr64;
                    if (s32 != neg_inf() && static_cast<double>(s32) + err >= thr) {
                        const int64_t p1 = g.off[s] + ea.run_start + i;
                        const int64_t p3 = g.roff[t] + ec.run_start + j;
                        mhr_path p;
                        p.u = ea.vertex;
                        p.v = ec.vertex;
                        p.r1 = g.rel[p1];
                        p.r3 = g.rrel[p3];
                        p.r2 = relsrc[sm.hep[lo]];
                        p.pad = 0;
                        const double w1d = edge_w64(g, s, p.r1, p.u);
                        const double w2d = edge_w64(g, p.u, p.r2, p.v);
                        const double w3d = edge_w64(g, p.v, p.r3, t);
                        p.score = __dadd_rn(__dadd_rn(w1d, w2d), w3d);
                        if (p.score >= thr) {
                            const int slot = atomicAdd(&sm.ns, 1);
                            sm.buf[K + slot] = p;
                        }
                    }
                }
                __syncthreads();
            }
            __syncthreads();
        }
        exact_flush(sm, K);
        mhr_path* dst = P->out + static_cast<int64_t>(q) * K;
        for (int i = threadIdx.x; i < sm.nt; i += blockDim.x) dst[i] = sm.buf[i];
        if (threadIdx.x == 0) P->n_out[q] = sm.nt;
        __syncthreads();
    }
}

// training rows from a label run (one per near entry that lies on a path)
__global__ void k_dump_labels(const PlanDev* __restrict__ P, int64_t cap, uint32_t* __restrict__ near_v,
                              uint32_t* __restrict__ end_v, float* __restrict__ own, float* __restrict__ best,
                              unsigned long long* __restrict__ count) {
    const int64_t X = P->X;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < X; x += stride) {
        int q;
        int64_t base;
        bool sideA;
        if (!near_slot(P, x, q, base, sideA)) continue;
        const uint32_t k = P->ubest[x];
        if (k == 0u) continue;
        const int64_t nat = base + P->nperm[x];
        const ListEnt e = P->list[nat];
        const unsigned long long i = atomicAdd(count, 1ull);
        if (static_cast<int64_t>(i) < cap) {
            near_v[i] = e.vertex;
            end_v[i] = sideA ? P->T[q] : P->S[q];
            own[i] = P->bnat[nat];  // the row's provable score bound
            best[i] = key2f(k);
        }
    }
}

// ===========================================================================
// host side: plans (buffers + captured graph) per (nq, K, chunk)
// ===========================================================================
struct Plan {
    int nq = 0, K = 0, chunk = 0, grid = 0, precision = 0, tile = kDefaultTile;
    int expand_per_sm = 8;  // resident expansion blocks per SM
    void (*expand_fn)(const PlanDev*, DevGraph) = nullptr;  // the expansion kernel for the graph's rows
    PlanDev h{};
    unsigned char* dregion = nullptr;  // [PlanDev][S][T][a_off][c_off]
    size_t region_bytes = 0;
    unsigned char* pin = nullptr;      // pinned host mirror of dregion
    std::vector<void*> fixed;
    void* slot_mem = nullptr;
    int64_t slot_cap = 0;
    void* item_mem = nullptr;
    void* far_mem = nullptr;
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr;
    cudaEvent_t h2d_done = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // before / join / after / end
    cudaEvent_t ev_x[2] = {nullptr, nullptr};  // around the expansion kernel (recorded inside the first graph)
    bool h2d_pending = false;
    void drop_graphs() {
        for (cudaGraphExec_t& x : exec)
            if (x) {
                cudaGraphExecDestroy(x);
                x = nullptr;
            }
    }
    ~Plan() {
        drop_graphs();
        if (cap) cudaStreamDestroy(cap);
        if (h2d_done) cudaEventDestroy(h2d_done);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_x)
            if (e) cudaEventDestroy(e);
        for (void* p : fixed) cudaFree(p);
        if (slot_mem) cudaFree(slot_mem);
        if (item_mem) cudaFree(item_mem);
        if (far_mem) cudaFree(far_mem);
        if (dregion) cudaFree(dregion);
        if (pin) cudaFreeHost(pin);
    }
};

struct PlanCache {
    std::map<std::tuple<int, int, int, int, int>, Plan*> plans;  // (nq, K, chunk, precision, tile)
    ~PlanCache() {
        for (auto& kv : plans) delete kv.second;
    }
};

void destroy_plans(mhr_graph* g) {
    delete g->plans;
    g->plans = nullptr;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct RegionLayout {
    size_t off_S, off_T, off_a, off_c, off_cons, total;
};

// bytes of the constraint flags: three relation sets and two type sets
static size_t cons_bytes(int R) { return 3 * static_cast<size_t>(R) + 512; }

static RegionLayout region_layout(int nq, int R) {
    RegionLayout L;
    size_t o = align_up(sizeof(PlanDev), 256);
    L.off_S = o;
    o = align_up(o + sizeof(uint32_t) * nq, 256);
    L.off_T = o;
    o = align_up(o + sizeof(uint32_t) * nq, 256);
    L.off_a = o;
    o = align_up(o + sizeof(int64_t) * (nq + 1), 256);
    L.off_c = o;
    o = align_up(o + sizeof(int64_t) * (nq + 1), 256);
    L.off_cons = o;
    o = align_up(o + cons_bytes(R), 256);
    L.total = o;
    return L;
}

template <typename T>
static mhr_status plan_alloc(Plan* p, T** out, size_t count) {
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (query plan)");
    p->fixed.push_back(ptr);
    *out = static_cast<T*>(ptr);
    return MHR_OK;
}

static size_t mid_smem_bytes() { return sizeof(MidSmem); }
static_assert(sizeof(MidSmem) <= 232448, "the join's shared memory fits one CTA per SM (227 KB)");
static size_t exact_smem_bytes() { return sizeof(ExactSmem); }
static size_t merge2_smem_bytes(int band_cap) {
    int m = 2;
    while (m < band_cap) m <<= 1;
    return sizeof(mhr_path) * m;
}

static mhr_status ensure_slots(Plan* p, int64_t X) {
    if (X <= p->slot_cap && p->slot_mem) return MHR_OK;
    int64_t cap = std::max<int64_t>(X, std::max<int64_t>(p->slot_cap * 2, 1 << 16));
    // per slot: w32 4, flag 4, scan1 8, list 32, nearP 8, nearL 32, nearB 4,
    // okey 4, orank 4, bnat 4, nperm 4, degv3 4, scan4 8, mlp_pred 4, ubest 4, w64s 8, w64own 4
    const size_t a8 = 256;
    size_t o = 0;
    const size_t o_w32 = o; o = align_up(o + 4 * cap, a8);
    const size_t o_flag = o; o = align_up(o + 4 * cap, a8);
    const size_t o_s1 = o; o = align_up(o + 8 * (cap + 1), a8);
    const size_t o_list = o; o = align_up(o + sizeof(ListEnt) * cap, a8);
    const size_t o_near = o; o = align_up(o + sizeof(uint2) * cap, a8);
    const size_t o_nearl = o; o = align_up(o + sizeof(ListEnt) * cap, a8);
    const size_t o_nb = o; o = align_up(o + sizeof(float) * cap, a8);
    const size_t o_okey = o; o = align_up(o + 4 * cap, a8);
    const size_t o_orank = o; o = align_up(o + 4 * cap, a8);
    const size_t o_bnat = o; o = align_up(o + 4 * cap, a8);
    const size_t o_nperm = o; o = align_up(o + 4 * cap, a8);
    const size_t o_degv3 = o; o = align_up(o + 4 * cap, a8);
    const size_t o_s4 = o; o = align_up(o + 8 * (cap + 1), a8);
    const size_t o_mlp = o; o = align_up(o + 4 * cap, a8);
    const size_t o_ub = o; o = align_up(o + 4 * cap, a8);
    const size_t o_w64 = o; o = align_up(o + 8 * cap, a8);
    const size_t o_own = o; o = align_up(o + 4 * cap, a8);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, o);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (frontier slots)");
    if (p->slot_mem) {
        cudaDeviceSynchronize();
        cudaFree(p->slot_mem);
    }
    p->slot_mem = mem;
    p->slot_cap = cap;
    unsigned char* b = static_cast<unsigned char*>(mem);
    p->h.w32 = reinterpret_cast<float*>(b + o_w32);
    p->h.flag = reinterpret_cast<uint32_t*>(b + o_flag);
    p->h.scan1 = reinterpret_cast<int64_t*>(b + o_s1);
    p->h.list = reinterpret_cast<ListEnt*>(b + o_list);
    p->h.nearP = reinterpret_cast<uint2*>(b + o_near);
    p->h.nearL = reinterpret_cast<ListEnt*>(b + o_nearl);
    p->h.nearB = reinterpret_cast<float*>(b + o_nb);
    p->h.okey = reinterpret_cast<uint32_t*>(b + o_okey);
    p->h.orank = reinterpret_cast<uint32_t*>(b + o_orank);
    p->h.bnat = reinterpret_cast<float*>(b + o_bnat);
    p->h.nperm = reinterpret_cast<uint32_t*>(b + o_nperm);
    p->h.degv3 = reinterpret_cast<uint32_t*>(b + o_degv3);
    p->h.scan4 = reinterpret_cast<int64_t*>(b + o_s4);
    p->h.mlp_pred = reinterpret_cast<float*>(b + o_mlp);
    p->h.ubest = reinterpret_cast<uint32_t*>(b + o_ub);
    p->h.w64s = reinterpret_cast<double*>(b + o_w64);
    p->h.w64own = reinterpret_cast<int32_t*>(b + o_own);
    // scan kernels take raw pointers, so a new buffer needs a new capture
    p->drop_graphs();
    return MHR_OK;
}

// The sequence is captured as three graphs (before, the join, after) so that
// timing events recorded between their launches on the caller's stream bracket
// the join kernel exactly.
// run table of the coarse far bitmap, one entry per coarse bit and join CTA
// (only graphs too large for the exact shared-memory bitmap need it)
static mhr_status ensure_far(Plan* p, int64_t cap) {
    if (p->h.sigma == 0) return MHR_OK;
    cap = std::max<int64_t>(cap, 1);
    if (cap <= p->h.far_cap && p->h.far_start) return MHR_OK;
    cap = std::max(cap, 2 * p->h.far_cap);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, sizeof(uint4) * static_cast<size_t>(cap) * p->grid);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (far-set run starts)");
    if (p->far_mem) {
        cudaDeviceSynchronize();
        cudaFree(p->far_mem);
    }
    p->far_mem = mem;
    p->h.far_start = static_cast<uint4*>(mem);
    p->h.far_cap = cap;
    return MHR_OK;
}

static mhr_status ensure_items(Plan* p, int64_t cap) {
    cap = std::max<int64_t>(cap, 1);
    if (cap <= p->h.item_cap && p->h.item_ub) return MHR_OK;
    cap = std::max(cap, 2 * p->h.item_cap);
    void* mem = nullptr;
    const size_t o_desc = align_up(sizeof(uint32_t) * cap, 256);
    cudaError_t e = cudaMalloc(&mem, o_desc + sizeof(uint4) * cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (work-item bounds)");
    if (p->item_mem) {
        cudaDeviceSynchronize();
        cudaFree(p->item_mem);
    }
    p->item_mem = mem;
    p->h.item_ub = static_cast<uint32_t*>(mem);
    p->h.item_desc = reinterpret_cast<uint4*>(static_cast<unsigned char*>(mem) + o_desc);
    p->h.item_cap = cap;
    return MHR_OK;
}

static cudaError_t launch_part(Plan* p, const mhr_graph* G, cudaStream_t st, int part) {
    const PlanDev* d = reinterpret_cast<const PlanDev*>(p->dregion);
    const int sms = std::max(1, G->num_sms);
    const DevGraph& g = G->dg;
    const int64_t* nX = reinterpret_cast<const int64_t*>(p->dregion + offsetof(PlanDev, X));
    if (part == 0) {
        k_init<<<sms * 2, 256, 0, st>>>(d, g);
        cudaError_t ee = cudaEventRecordWithFlags(p->ev_x[0], st, cudaEventRecordExternal);
        if (ee != cudaSuccess) return ee;
        p->expand_fn<<<sms * p->expand_per_sm, 256, 0, st>>>(d, g);
        ee = cudaEventRecordWithFlags(p->ev_x[1], st, cudaEventRecordExternal);
        if (ee != cudaSuccess) return ee;
        cudaError_t e = device_excl_scan<uint32_t>(p->h.flag, nX, p->h.partials, p->h.scan1, st);
        if (e != cudaSuccess) return e;
        k_lists<<<sms * 4, 256, 0, st>>>(d, g);
        k_plan<<<1, 1024, 0, st>>>(d);
        k_order_key<<<sms * 4, 256, 0, st>>>(d, g);
        k_mlp_qbias<<<std::min(p->nq, sms * 4), kMlpHid, 0, st>>>(d, g);
        k_mlp_keys<<<sms, kTcThreads, sizeof(MlpTcSmem<128>), st>>>(d, g);
        k_order_hist<<<sms * 4, 256, 0, st>>>(d);
        const int64_t* nH = reinterpret_cast<const int64_t*>(p->dregion + offsetof(PlanDev, nhist));
        e = device_excl_scan<uint32_t>(p->h.hist, nH, p->h.partials, p->h.hscan, st);
        if (e != cudaSuccess) return e;
        k_order_perm<<<sms * 4, 256, 0, st>>>(d);
        e = device_excl_scan<uint32_t>(p->h.degv3, nX, p->h.partials, p->h.scan4, st);
        if (e != cudaSuccess) return e;
        k_near<<<sms * 4, 256, 0, st>>>(d, g);
    } else if (part == 1) {
        const size_t sb = mid_smem_bytes();
        if (p->tile == 8) {
            if (p->precision) {
                k_middle<8, true, true><<<p->grid, kMidThreads, sb, st>>>(d, g);
                k_middle<8, false, true><<<p->grid, kMidThreads, sb, st>>>(d, g);
            } else {
                k_middle<8, true, false><<<p->grid, kMidThreads, sb, st>>>(d, g);
                k_middle<8, false, false><<<p->grid, kMidThreads, sb, st>>>(d, g);
            }
        } else {
            if (p->precision) {
                k_middle<4, true, true><<<p->grid, kMidThreads, sb, st>>>(d, g);
                k_middle<4, false, true><<<p->grid, kMidThreads, sb, st>>>(d, g);
            } else {
                k_middle<4, true, false><<<p->grid, kMidThreads, sb, st>>>(d, g);
                k_middle<4, false, false><<<p->grid, kMidThreads, sb, st>>>(d, g);
            }
        }
    } else {
        k_merge1<<<std::min(p->nq, sms * 2), 1024, 0, st>>>(d);
        k_rescore<<<sms * 4, kRsWarps * 32, 0, st>>>(d, g);
        k_merge2<<<std::min(p->nq, sms * 2), 1024, merge2_smem_bytes(p->h.band_cap), st>>>(d, g);
        k_exact<<<std::min(p->nq, sms * 2), 1024, exact_smem_bytes(), st>>>(d, g);
    }
    return cudaGetLastError();
}

static mhr_status capture(Plan* p, const mhr_graph* G) {
    if (p->exec[0]) return MHR_OK;
    for (int part = 0; part < 3; ++part) {
        cudaGraph_t graph = nullptr;
        MHR_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_part(p, G, p->cap, part);
        cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            p->drop_graphs();
            return cuda_fail(e != cudaSuccess ? e : e2, "kernel launch during capture");
        }
        e = cudaGraphInstantiate(&p->exec[part], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->drop_graphs();
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    return MHR_OK;
}

static cudaError_t launch_graphs(Plan* p, cudaStream_t st) {
    cudaError_t e;
    for (int part = 0; part < 3; ++part) {
        if ((e = cudaEventRecord(p->ev[part], st)) != cudaSuccess) return e;
        if ((e = cudaGraphLaunch(p->exec[part], st)) != cudaSuccess) return e;
    }
    return cudaEventRecord(p->ev[3], st);
}

// lanes that score one edge together: about `per` 16-byte vectors per lane per row
static int hit_group_width(int d, int dtype, int per) {
    const int vec = (dtype == MHR_F32) ? ((d & 3) == 0 ? d / 4 : d) : ((d & 7) == 0 ? d / 8 : d);
    const int want = (vec + per - 1) / per;
    int w = 1;
    while (w < want && w < 32) w <<= 1;
    return w;
}

static float __double2float_ru_host(double x) {
    float f = static_cast<float>(x);
    if (static_cast<double>(f) < x) f = std::nextafter(f, INFINITY);
    return f;
}

static int choose_sigma(int64_t n) {
    int sigma = 0;
    while (((n - 1) >> sigma) >= static_cast<int64_t>(kMaxBmWords) * 32) ++sigma;
    return sigma;
}

static mhr_status make_plan(mhr_graph* G, int nq, int K, int chunk, int precision, int tile, Plan** out) {
    Plan* p = new Plan();
    p->nq = nq;
    p->tile = tile;
    p->K = K;
    p->chunk = chunk;
    p->precision = precision;
    p->grid = std::max(1, G->num_sms);
    PlanDev& h = p->h;
    h.nq = nq;
    h.K = K;
    h.chunk = chunk;
    h.sigma = choose_sigma(G->dg.n);
    h.nbw = static_cast<int32_t>(((G->dg.n - 1) >> h.sigma) / 32 + 1);
    h.pq = 16 * K + 4096;  // room for the final candidates of every CTA that worked on the query
    h.band_cap = K + 2048;
    h.err_path = precision ? G->err_path_tc : G->err_path;
    h.precision = precision;
    h.prune_slack = precision ? __double2float_ru_host((G->epstc_edge + G->eps32_edge) * 1.01) : 0.f;
    h.wsplit = G->wsplit;
    h.score_width = hit_group_width(G->dg.d, G->dg.dtype, 2);
    h.hit_width = hit_group_width(G->dg.d, G->dg.dtype, kHitVecs);
    mhr_status rc = MHR_OK;
    auto bail = [&](mhr_status r) {
        delete p;
        return r;
    };
    if ((rc = plan_alloc(p, &h.status, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.dir, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.near_cnt, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.far_cnt, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.s_near, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.item_off, nq + 1)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.near_off, nq + 1)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.thr_g, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.seed_k, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.mlp_qbias, static_cast<size_t>(nq) * kMlpHid)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.qmax, 2 * static_cast<size_t>(nq))) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.sdeg_q, 2 * static_cast<size_t>(nq))) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.qkey, 2 * static_cast<size_t>(nq))) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.hist, 256 * static_cast<size_t>(nq))) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.hscan, 256 * static_cast<size_t>(nq) + 1)) != MHR_OK) return bail(rc);
    h.nhist = 256 * static_cast<int64_t>(nq);
    if ((rc = plan_alloc(p, &h.dense, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.pool_cnt, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.band_cnt, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.hits, static_cast<size_t>(p->grid) * kMaxChunk)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.pool, static_cast<size_t>(nq) * h.pq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.band_cand, static_cast<size_t>(nq) * h.band_cap)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.band_w2, static_cast<size_t>(nq) * h.band_cap)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.chains, static_cast<size_t>(nq) * 3 * h.band_cap)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.chain_cnt, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.out, static_cast<size_t>(nq) * K)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.n_out, nq)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.counters, kCntCount)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.partials, kScanPartials)) != MHR_OK) return bail(rc);
    if (cudaMemset(h.partials, 0, sizeof(int64_t) * kScanPartials) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaMemset (scan counter)"));
    if ((rc = plan_alloc(p, &h.cursors, p->grid)) != MHR_OK) return bail(rc);
    if ((rc = plan_alloc(p, &h.drained, (p->grid + 31) / 32)) != MHR_OK) return bail(rc);
    h.grid = p->grid;
    const RegionLayout L = region_layout(nq, G->dg.R);
    p->region_bytes = L.total;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->dregion), L.total);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc (plan region)"));
    e = cudaMallocHost(reinterpret_cast<void**>(&p->pin), L.total);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocHost (plan region)"));
    h.S = reinterpret_cast<const uint32_t*>(p->dregion + L.off_S);
    h.T = reinterpret_cast<const uint32_t*>(p->dregion + L.off_T);
    h.a_off = reinterpret_cast<const int64_t*>(p->dregion + L.off_a);
    h.c_off = reinterpret_cast<const int64_t*>(p->dregion + L.off_c);
    e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    e = cudaEventCreateWithFlags(&p->h2d_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    for (cudaEvent_t& ev : p->ev_x) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    for (cudaEvent_t& ev : p->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    {
        const int sb = static_cast<int>(mid_smem_bytes());
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        e = cudaFuncSetAttribute(k_middle<4, true, false>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<4, false, false>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<4, true, true>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<4, false, true>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<8, true, false>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<8, false, false>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<8, true, true>, a, sb);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_middle<8, false, true>, a, sb);
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute (middle join)"));
    {
        // one resident wave of the grid-stride expansion kernel
        int nb = 0;
        p->expand_fn = expand_kernel(G->dg, h.score_width);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, p->expand_fn, 256, 0) == cudaSuccess && nb > 0)
            p->expand_per_sm = nb;
        cudaGetLastError();
    }
    e = cudaFuncSetAttribute(k_mlp_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(MlpTcSmem<128>)));
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute (ordering MLP)"));
    e = cudaFuncSetAttribute(k_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(exact_smem_bytes()));
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute (exact)"));
    e = cudaFuncSetAttribute(k_merge2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(merge2_smem_bytes(h.band_cap)));
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute (merge)"));
    *out = p;
    return MHR_OK;
}

static mhr_status get_plan(mhr_graph* G, int nq, int K, int chunk, int precision, int tile, Plan** out) {
    if (!G->plans) G->plans = new PlanCache();
    auto key = std::make_tuple(nq, K, chunk, precision, tile);
    auto it = G->plans->plans.find(key);
    if (it != G->plans->plans.end()) {
        *out = it->second;
        return MHR_OK;
    }
    if (G->plans->plans.size() >= 8) {
        cudaDeviceSynchronize();
        delete G->plans->plans.begin()->second;
        G->plans->plans.erase(G->plans->plans.begin());
    }
    Plan* p = nullptr;
    MHR_TRY(make_plan(G, nq, K, chunk, precision, tile, &p));
    G->plans->plans[key] = p;
    *out = p;
    return MHR_OK;
}

static mhr_status run_batch(mhr_graph* G, int nq, const uint32_t* hS, const uint32_t* hT, int K,
                            const mhr_query_opts* opts, cudaStream_t st, Plan** plan_out, bool label = false) {
    int chunk = (opts && opts->chunk > 0) ? opts->chunk : kDefaultChunk;
    if (chunk > kMaxChunk || chunk < 32 || (chunk & 31))
        return fail(MHR_EINVAL, "opts->chunk must be a multiple of 32 in [32, 32768]");
    const int precision = opts ? opts->precision : 0;
    if (precision != 0 && precision != 1) return fail(MHR_EINVAL, "opts->precision must be 0 or 1");
    const int tile = (opts && opts->tile) ? opts->tile : kDefaultTile;
    if (tile != 4 && tile != 8) return fail(MHR_EINVAL, "opts->tile must be 0, 4 or 8");
    if (precision == 1 && (G->fn != MHR_SCORE_DISTMULT || G->dg.R > 16 || !G->wsplit))
        return fail(MHR_EINVAL, "the tensor-core screen (precision 1) needs DistMult and at most 16 relations");
    if (precision == 1 && label) return fail(MHR_EINVAL, "label runs use the plain search");
    Plan* p = nullptr;
    MHR_TRY(get_plan(G, nq, K, chunk, precision, tile, &p));
    // sizes from the host copy of the row starts
    const RegionLayout L = region_layout(nq, G->dg.R);
    if (p->h2d_pending) {
        MHR_CUDA_TRY(cudaEventSynchronize(p->h2d_done));
        p->h2d_pending = false;
    }
    uint32_t* pS = reinterpret_cast<uint32_t*>(p->pin + L.off_S);
    uint32_t* pT = reinterpret_cast<uint32_t*>(p->pin + L.off_T);
    int64_t* pa = reinterpret_cast<int64_t*>(p->pin + L.off_a);
    int64_t* pc = reinterpret_cast<int64_t*>(p->pin + L.off_c);
    const int64_t n = G->dg.n;
    int64_t ta = 0, tc = 0;
    for (int q = 0; q < nq; ++q) {
        const uint32_t s = hS[q], t = hT[q];
        pS[q] = s;
        pT[q] = t;
        pa[q] = ta;
        pc[q] = tc;
        if (s < n && t < n && s != t) {
            ta += G->h_off[s + 1] - G->h_off[s];
            tc += G->h_roff[t + 1] - G->h_roff[t];
        }
    }
    pa[nq] = ta;
    pc[nq] = tc;
    MHR_TRY(ensure_slots(p, ta + tc));
    // work items per query are at most ceil(S_near / chunk), and S_near is at
    // most min(E, deg(s) * max out-degree, deg(t) * max in-degree)
    int64_t icap = 0;
    for (int q = 0; q < nq; ++q) {
        const int64_t da = pa[q + 1] - pa[q], dc = pc[q + 1] - pc[q];
        const int64_t bound = std::min<int64_t>(G->dg.E, std::min(da * G->max_out_deg, dc * G->max_in_deg));
        icap += (bound + chunk - 1) / chunk;
    }
    MHR_TRY(ensure_items(p, icap));
    // the coarse bitmap's run table has one entry per bit
    MHR_TRY(ensure_far(p, static_cast<int64_t>(p->h.nbw) * 32));
    p->h.X = ta + tc;
    p->h.totA = ta;
    p->h.prune = (opts && opts->prune) ? 1 : 0;
    p->h.order = opts ? opts->order : 0;
    if (p->h.order < 0 || p->h.order > 2) return fail(MHR_EINVAL, "opts->order must be 0, 1 or 2");
    p->h.mlp = MlpDev{};
    if (p->h.order == 2) {
        const mhr_mlp* m = opts->mlp;
        if (!m || !m->W1 || !m->b1 || !m->w2 || !m->b2) return fail(MHR_EINVAL, "order 2 needs opts->mlp weights");
        p->h.mlp.W1 = m->W1;
        p->h.mlp.b1 = m->b1;
        p->h.mlp.w2 = m->w2;
        p->h.mlp.b2 = m->b2;
    }
    p->h.label = label ? 1 : 0;
    if (label && (p->h.prune || p->h.order)) return fail(MHR_EINVAL, "label runs use the plain search");
    // vertex partition of the paths by their hop-1 vertex
    p->h.part_count = opts ? opts->part_count : 0;
    p->h.part_index = opts ? opts->part_index : 0;
    if (p->h.part_count < 0 || (p->h.part_count > 1 && (p->h.part_index < 0 || p->h.part_index >= p->h.part_count)) ||
        (p->h.part_count <= 1 && p->h.part_index != 0))
        return fail(MHR_EINVAL, "opts->part_index must be in [0, part_count)");
    if (label && p->h.part_count > 1) return fail(MHR_EINVAL, "label runs use the unpartitioned search");
    // constraint flags (Sec. 3.1 query shape), copied with the call's queries
    p->h.cons = nullptr;
    if (opts && opts->constraints) {
        if (label) return fail(MHR_EINVAL, "label runs use the unconstrained search");
        const mhr_constraints* c = opts->constraints;
        const int R = G->dg.R;
        uint8_t* f = p->pin + L.off_cons;
        const uint8_t* rel[3] = {c->rel1, c->rel2, c->rel3};
        for (int h = 0; h < 3; ++h)
            for (int r = 0; r < R; ++r) f[h * R + r] = rel[h] ? (rel[h][r] != 0) : 1;
        const uint8_t* ty[2] = {c->types_u, c->types_v};
        for (int h = 0; h < 2; ++h)
            for (int y = 0; y < 256; ++y) f[3 * R + h * 256 + y] = ty[h] ? (ty[h][y] != 0) : 1;
        p->h.cons = p->dregion + L.off_cons;
    }
    std::memcpy(p->pin, &p->h, sizeof(PlanDev));
    MHR_CUDA_TRY(cudaMemcpyAsync(p->dregion, p->pin, L.total, cudaMemcpyHostToDevice, st));
    MHR_CUDA_TRY(cudaEventRecord(p->h2d_done, st));
    p->h2d_pending = true;
    MHR_TRY(capture(p, G));
    MHR_CUDA_TRY(launch_graphs(p, st));
    *plan_out = p;
    return MHR_OK;
}

static mhr_status read_stats(Plan* p, cudaStream_t st, mhr_stats* stats) {
    unsigned long long c[kCntCount];
    MHR_CUDA_TRY(cudaMemcpyAsync(c, p->h.counters, sizeof c, cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    stats->edges_scanned = static_cast<int64_t>(c[kCntScanned]);
    stats->hits = static_cast<int64_t>(c[kCntHits]);
    stats->paths = static_cast<int64_t>(c[kCntPaths]);
    stats->candidates = static_cast<int64_t>(c[kCntCands]);
    stats->rescored = static_cast<int64_t>(c[kCntRescored]);
    stats->pruned_edges = static_cast<int64_t>(c[kCntPruned]);
    stats->dense_queries = static_cast<int64_t>(c[kCntDense]);
    float a = -1.f, b = -1.f;
    if (cudaEventElapsedTime(&a, p->ev[0], p->ev[3]) != cudaSuccess) a = -1.f;
    // ev[1] .. ev[2] bracket the join graph
    if (cudaEventElapsedTime(&b, p->ev[1], p->ev[2]) != cudaSuccess) b = -1.f;
    float x = -1.f;
    if (cudaEventElapsedTime(&x, p->ev_x[0], p->ev_x[1]) != cudaSuccess) x = -1.f;
    stats->ms_expand = x;
    cudaGetLastError();
    stats->ms_device = a;
    stats->ms_join = b;
    return MHR_OK;
}

}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_topk_paths_batched(const mhr_graph* gc, int32_t nq, const uint32_t* s,
                                             const uint32_t* t, int32_t K, mhr_path* out, int32_t* n_out,
                                             mhr_mem mem, const mhr_query_opts* opts, mhr_stats* stats,
                                             void* cuda_stream) {
    MHR_TRY(check_graph(gc));
    mhr_graph* G = const_cast<mhr_graph*>(gc);
    if (nq < 0) return fail(MHR_EINVAL, "nq must be >= 0");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_K_MAX");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    if (nq == 0) {
        if (stats) *stats = mhr_stats{};
        return MHR_OK;
    }
    if (!s || !t || !out || !n_out) return fail(MHR_EINVAL, "a required pointer is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<uint32_t> hs, ht;
    const uint32_t *ps = s, *pt = t;
    if (mem == MHR_MEM_DEVICE) {
        hs.resize(nq);
        ht.resize(nq);
        MHR_CUDA_TRY(cudaMemcpyAsync(hs.data(), s, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(ht.data(), t, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
        ps = hs.data();
        pt = ht.data();
    }
    Plan* p = nullptr;
    MHR_TRY(run_batch(G, nq, ps, pt, K, opts, st, &p));
    const cudaMemcpyKind kind = mem == MHR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    MHR_CUDA_TRY(cudaMemcpyAsync(out, p->h.out, sizeof(mhr_path) * static_cast<size_t>(nq) * K, kind, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(n_out, p->h.n_out, sizeof(int32_t) * nq, kind, st));
    if (mem == MHR_MEM_HOST) MHR_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats) {
        *stats = mhr_stats{};
        MHR_TRY(read_stats(p, st, stats));
    }
    return MHR_OK;
}

// Autotuner of the join's launch shape and middle-edge screen: every
// (screen, work-item size, scan tile) candidate runs the same batch (results
// do not depend on any of them), timed by the plan's own events; the plans of
// the losing candidates are released.
extern "C" mhr_status mhr_autotune(const mhr_graph* gc, int32_t nq, const uint32_t* s, const uint32_t* t, int32_t K,
                                   mhr_mem mem, const mhr_query_opts* opts, const int32_t* chunks, int32_t n_chunks,
                                   const int32_t* tiles, int32_t n_tiles, int32_t reps, int32_t* best_chunk,
                                   int32_t* best_tile, int32_t* best_precision, float* ms_out, void* cuda_stream) {
    MHR_TRY(check_graph(gc));
    mhr_graph* G = const_cast<mhr_graph*>(gc);
    static const int32_t kChunks[3] = {8192, 16384, 32768};
    static const int32_t kTiles[2] = {4, 8};
    if (!chunks) {
        chunks = kChunks;
        n_chunks = 3;
    }
    if (!tiles) {
        tiles = kTiles;
        n_tiles = 2;
    }
    if (nq < 1 || !s || !t || !best_chunk || !best_tile || n_chunks < 1 || n_tiles < 1 || reps < 1)
        return fail(MHR_EINVAL, "bad autotune arguments");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_K_MAX");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    for (int i = 0; i < n_chunks; ++i)
        if (chunks[i] > kMaxChunk || chunks[i] < 32 || (chunks[i] & 31))
            return fail(MHR_EINVAL, "chunk candidates must be multiples of 32 in [32, 32768]");
    for (int i = 0; i < n_tiles; ++i)
        if (tiles[i] != 4 && tiles[i] != 8) return fail(MHR_EINVAL, "tile candidates must be 4 or 8");
    mhr_query_opts o = opts ? *opts : mhr_query_opts{};
    // screens to try: the requested one, or both when opts->precision < 0 and
    // the tensor-core screen applies (DistMult, at most 16 relations)
    int precs[2] = {o.precision, 0};
    int n_prec = 1;
    if (o.precision < 0) {
        precs[0] = 0;
        if (G->fn == MHR_SCORE_DISTMULT && G->dg.R <= 16 && G->wsplit) {
            precs[1] = 1;
            n_prec = 2;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<uint32_t> hs(nq), ht(nq);
    MHR_CUDA_TRY(cudaMemcpyAsync(hs.data(), s, sizeof(uint32_t) * nq, cudaMemcpyDefault, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(ht.data(), t, sizeof(uint32_t) * nq, cudaMemcpyDefault, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    const int per = n_chunks * n_tiles;
    int best = -1;
    float best_ms = 0.f;
    for (int i = 0; i < n_prec * per; ++i) {
        o.precision = precs[i / per];
        o.chunk = chunks[(i % per) / n_tiles];
        o.tile = tiles[i % n_tiles];
        Plan* p = nullptr;
        MHR_TRY(run_batch(G, nq, hs.data(), ht.data(), K, &o, st, &p));  // warm-up (capture, buffers)
        float ms = 0.f;
        for (int r = 0; r < reps; ++r) {
            MHR_TRY(run_batch(G, nq, hs.data(), ht.data(), K, &o, st, &p));
            mhr_stats sts{};
            MHR_TRY(read_stats(p, st, &sts));
            if (sts.ms_device < 0) return fail(MHR_ECUDA, "autotune: event timing failed");
            ms = r == 0 ? static_cast<float>(sts.ms_device) : std::min(ms, static_cast<float>(sts.ms_device));
        }
        if (ms_out) ms_out[i] = ms;
        if (best < 0 || ms < best_ms) {
            best = i;
            best_ms = ms;
        }
    }
    const int bp = precs[best / per];
    *best_chunk = chunks[(best % per) / n_tiles];
    *best_tile = tiles[best % n_tiles];
    if (best_precision) *best_precision = bp;
    // keep only the winner's plan
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n_prec * per; ++i) {
        const int pr = precs[i / per], c = chunks[(i % per) / n_tiles], tl = tiles[i % n_tiles];
        if (pr == bp && c == *best_chunk && tl == *best_tile) continue;
        auto it = G->plans->plans.find(std::make_tuple(static_cast<int>(nq), static_cast<int>(K), c, pr, tl));
        if (it != G->plans->plans.end()) {
            delete it->second;
            G->plans->plans.erase(it);
        }
    }
    return MHR_OK;
}

extern "C" mhr_status mhr_training_labels(const mhr_graph* gc, int32_t nq, const uint32_t* s, const uint32_t* t,
                                          int64_t cap, uint32_t* near_v, uint32_t* end_v, float* own, float* best,
                                          int64_t* n_written, void* cuda_stream) {
    MHR_TRY(check_graph(gc));
    mhr_graph* G = const_cast<mhr_graph*>(gc);
    if (nq < 1 || !s || !t || !n_written || cap < 0 || (cap && (!near_v || !end_v || !own || !best)))
        return fail(MHR_EINVAL, "bad training-label arguments");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Plan* p = nullptr;
    mhr_query_opts plain{};
    MHR_TRY(run_batch(G, nq, s, t, 1, &plain, st, &p, true));
    unsigned long long* cnt = p->h.counters + kCntLabels;
    MHR_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    k_dump_labels<<<std::max(1, G->num_sms) * 4, 256, 0, st>>>(reinterpret_cast<const PlanDev*>(p->dregion), cap,
                                                               near_v, end_v, own, best, cnt);
    MHR_CUDA_TRY(cudaGetLastError());
    unsigned long long h = 0;
    MHR_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    *n_written = static_cast<int64_t>(h);
    if (static_cast<int64_t>(h) > cap) return fail(MHR_ERANGE, "more training rows than cap");
    return MHR_OK;
}

extern "C" mhr_status mhr_topk_paths(const mhr_graph* g, uint32_t s, uint32_t t, int32_t K, mhr_path* out,
                                     int32_t* n_out, const mhr_query_opts* opts, mhr_stats* stats) {
    MHR_TRY(check_graph(g));
    if (!out || !n_out) return fail(MHR_EINVAL, "out and n_out are required");
    if (s >= g->dg.n || t >= g->dg.n) return fail(MHR_EINVAL, "s or t is out of range");
    if (s == t) return fail(MHR_EINVAL, "s == t");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_K_MAX");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);
    std::vector<mhr_path> buf(K);
    int32_t n = 0;
    mhr_status rc = mhr_topk_paths_batched(g, 1, &s, &t, K, buf.data(), &n, MHR_MEM_HOST, opts, stats, nullptr);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MHR_OK) return rc;
    std::memcpy(out, buf.data(), sizeof(mhr_path) * std::max(0, n));
    *n_out = n;
    if (stats) stats->ms = ms;
    return MHR_OK;
}
