// Generic H-hop search with a per-path beam (Alg. 6, Alg. 7), batched over
// queries, exact.
//
// Level l holds, per query, up to K^l paths in fixed slots (slot j of level
// l+1 is child j mod K of slot j / K of level l).  One CTA per held path:
//   - every out-edge (x, r, y) of the path's last vertex x is scored in fp32;
//     the K-th largest fp32 weight among the path's extensions sets a band (the
//     graph's proven fp32 error, twice, plus the spacing of the rounded path
//     scores), and only the extensions inside it and the edges into t are
//     scored in fp64 in the canonical operation order (the path score is the
//     parent's score plus the edge weight, left to right, as the reference
//     definition);
//   - y already on the path: skipped (Alg. 7); y == t: a result (reaching the
//     target ends the path); otherwise an extension;
//   - the path keeps its K best extensions (score desc, then relation, then
//     vertex ascending) and its K best results, merged chunk by chunk (256
//     edges) into shared-memory lists with a bitonic sort;
//   - the K best extensions become the children's slots of level l+1 (unused
//     child slots are marked empty), the K best results are appended to the
//     query's result list.
// A final CTA per query keeps the K best results (score desc, hop count asc,
// then (y_1, r_1, ..., y_{h-1}, r_{h-1}, r_h) asc) and writes them in order.
// Every kept score is fp64 with the reference's operation order, so selection
// decisions and output equal the fp64 brute force exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "mhr_internal.cuh"

namespace mhr {
namespace {

constexpr int kBeamThreads = 256;
constexpr int kBeamChunk = 256;      // edges per merge step
constexpr int kBeamMaxK = 64;        // MHR_BEAM_K_MAX
constexpr int kBeamMaxH = 8;         // MHR_BEAM_MAX_H
constexpr int kBeamBuf = 512;        // >= kBeamMaxK + kBeamChunk, power of two

struct BeamPath {                    // same layout as mhr_beam_path (64 B)
    double score;
    int32_t hops;                    // -1: empty slot
    uint32_t v[kBeamMaxH + 1];
    uint16_t r[kBeamMaxH];
};
static_assert(sizeof(BeamPath) == 64, "beam path record is 64 bytes");
static_assert(kBeamBuf >= kBeamMaxK + kBeamChunk, "merge buffer holds the kept list and one chunk");

struct Ext {                         // one scored out-edge of a held path
    double score;
    uint32_t y;
    uint32_t r;                      // relation; 0xffffffff pads the sort
};

// extensions of one path: score desc, then relation asc, then vertex asc
__device__ __forceinline__ bool ext_before(const Ext& a, const Ext& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.r != b.r) return a.r < b.r;
    return a.y < b.y;
}

// results: score desc, hop count asc, then (y_1, r_1, ..., y_{h-1}, r_{h-1}, r_h) asc
__device__ __forceinline__ bool result_before(const BeamPath& a, const BeamPath& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.hops != b.hops) return a.hops < b.hops;
    for (int i = 1; i < a.hops; ++i) {
        if (a.v[i] != b.v[i]) return a.v[i] < b.v[i];
        if (a.r[i - 1] != b.r[i - 1]) return a.r[i - 1] < b.r[i - 1];
    }
    return a.r[a.hops - 1] < b.r[b.hops - 1];
}

__device__ __forceinline__ Ext ext_pad() { return Ext{-INFINITY, 0xffffffffu, 0xffffffffu}; }

// bitonic sort of P (power of two) records in shared memory, best first
template <typename T, typename Before>
__device__ void block_bitonic(T* a, unsigned P, Before before) {
    for (unsigned size = 2; size <= P; size <<= 1) {
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
                const unsigned j = i ^ stride;
                if (j > i) {
                    const T x = a[i], y = a[j];
                    const bool best_first = (i & size) == 0;
                    if (best_first ? before(y, x) : before(x, y)) {
                        a[i] = y;
                        a[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ unsigned pow2_at_least(unsigned m) {
    unsigned P = 1;
    while (P < m) P <<= 1;
    return P;
}

// level 0: the one-vertex path (s) of every query
__global__ void k_beam_init(const uint32_t* __restrict__ s, int nq, BeamPath* __restrict__ level0,
                            unsigned* __restrict__ n_res) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    BeamPath p;
    p.score = 0.0;
    p.hops = 0;
    for (int i = 0; i <= kBeamMaxH; ++i) p.v[i] = 0u;
    for (int i = 0; i < kBeamMaxH; ++i) p.r[i] = 0;
    p.v[0] = s[q];
    level0[q] = p;
    n_res[q] = 0u;
}

struct LevelArgs {
    DevGraph g;
    const uint32_t* t;             // [nq] targets
    int level, H, K;
    int64_t slots;                 // K^level slots per query at this level
    const BeamPath* cur;           // [nq * slots]
    BeamPath* next;                // [nq * slots * K] when level + 1 < H
    BeamPath* res;                 // [nq * res_cap]
    int64_t res_cap;
    unsigned* n_res;               // [nq]
    unsigned long long* n_scored;  // edges scored (one counter)
    unsigned long long* n_exact;   // extensions scored in fp64 (one counter)
    double e1;                     // bound on |w32 - w64| of one edge
};

// Screening of a path's extensions.  With T the K-th largest fp32 weight
// w32 among them and E1 the bound on |w32 - w64|, every extension of the true
// K best (by fl64(score(p) + w64), then relation, then vertex) has
//   w32 >= T - 2 E1 - 2^-51 (|score(p)| + |w32| + E1)   (rounded down below):
// at least one of the K extensions with w32 >= T ranks after it, so its w64 is
// at least that one's w64 minus the spacing of the doubles around the
// (equal) rounded path scores.  Only those extensions are scored in fp64.
__device__ __forceinline__ bool in_band(float w32, float T, double P, double e1) {
    if (T == -INFINITY) return true;
    const double a = fabs(P) + fabs(static_cast<double>(w32)) + e1 + 1.0;
    return static_cast<double>(w32) >= static_cast<double>(T) - 2.0 * e1 - ldexp(a, -50);
}

// one CTA per held path of this level
__global__ void __launch_bounds__(kBeamThreads) k_beam_level(LevelArgs a) {
    __shared__ Ext ext[kBeamBuf];
    __shared__ Ext res[kBeamBuf];
    __shared__ unsigned n_ext, n_rl, c_ext, c_res, res_base;
    const int64_t slot = blockIdx.x;
    const int64_t q = slot / a.slots;
    const BeamPath p = a.cur[slot];
    const bool more = a.level + 1 < a.H;
    const int K = a.K;
    if (p.hops != a.level) {  // an empty slot has empty children
        if (more)
            for (int c = threadIdx.x; c < K; c += blockDim.x) a.next[slot * K + c].hops = -1;
        return;
    }
    const uint32_t x = p.v[a.level];
    const uint32_t tq = a.t[q];
    const int64_t e0 = a.g.off[x], e1 = a.g.off[x + 1];
    __shared__ float topw[kBeamBuf];  // screening: the K largest fp32 extension weights, then staging
    __shared__ unsigned n_top, c_top;
    __shared__ float thr_adm;         // admission threshold of the staging (K-th largest so far)
    __shared__ unsigned long long n_fp64;
    if (threadIdx.x == 0) {
        n_ext = 0u;
        n_rl = 0u;
        n_top = 0u;
        n_fp64 = 0ull;
        thr_adm = -INFINITY;
        if (e1 > e0) atomicAdd(a.n_scored, static_cast<unsigned long long>(e1 - e0));
    }
    __syncthreads();
    // 0. fp32 pass over the extensions: T = the K-th largest w32 (-inf when
    //    there are at most K extensions: every one is kept)
    float T = -INFINITY;
    if (more && e1 - e0 > K) {
        for (int64_t base = e0; base < e1; base += kBeamChunk) {
            if (threadIdx.x == 0) c_top = 0u;
            __syncthreads();
            const int64_t e = base + threadIdx.x;
            if (threadIdx.x < kBeamChunk && e < e1) {
                const uint32_t y = a.g.col[e];
                bool on_path = y == tq;
                for (int i = 0; i <= a.level; ++i) on_path |= (p.v[i] == y);
                if (!on_path) {
                    const float w = edge_w32_group(a.g, x, a.g.rel[e], y, 0, 1);
                    if (w >= thr_adm) topw[n_top + atomicAdd(&c_top, 1u)] = w;
                }
            }
            __syncthreads();
            const unsigned m = n_top + c_top;
            const bool last = base + kBeamChunk >= e1;
            // keep the K largest once the staging could not take another chunk, and
            // at the end (sorted, so that entry K - 1 is the K-th largest)
            if (m + kBeamChunk > static_cast<unsigned>(kBeamBuf) || last) {
                if (m > static_cast<unsigned>(K) || (last && m == static_cast<unsigned>(K))) {
                    const unsigned P2 = pow2_at_least(m);
                    for (unsigned i = m + threadIdx.x; i < P2; i += blockDim.x) topw[i] = -INFINITY;
                    __syncthreads();
                    block_bitonic(topw, P2, [](float u, float v) { return u > v; });
                    if (threadIdx.x == 0) {
                        n_top = static_cast<unsigned>(K);
                        thr_adm = topw[K - 1];
                    }
                } else if (threadIdx.x == 0) {
                    n_top = m;
                }
            } else if (threadIdx.x == 0) {
                n_top = m;
            }
            __syncthreads();
        }
        if (n_top >= static_cast<unsigned>(K)) T = topw[K - 1];
        __syncthreads();
    }
    for (int64_t base = e0; base < e1; base += kBeamChunk) {
        if (threadIdx.x == 0) {
            c_ext = 0u;
            c_res = 0u;
        }
        __syncthreads();
        // 1. score this chunk's edges; append behind the kept lists
        const int64_t e = base + threadIdx.x;
        if (threadIdx.x < kBeamChunk && e < e1) {
            const uint32_t y = a.g.col[e];
            const uint32_t r = a.g.rel[e];
            bool on_path = false;
            for (int i = 0; i <= a.level; ++i) on_path |= (p.v[i] == y);
            if (!on_path && (y == tq || more)) {
                // an extension outside the screening band cannot be among the K best
                const bool keep = y == tq || T == -INFINITY ||
                                  in_band(edge_w32_group(a.g, x, r, y, 0, 1), T, p.score, a.e1);
                if (keep) {
                    const double sc = __dadd_rn(p.score, edge_w64(a.g, x, r, y));
                    if (y == tq) res[n_rl + atomicAdd(&c_res, 1u)] = Ext{sc, y, r};
                    else ext[n_ext + atomicAdd(&c_ext, 1u)] = Ext{sc, y, r};
                    atomicAdd(&n_fp64, 1ull);
                }
            }
        }
        __syncthreads();
        // 2. keep the K best of each list
        const unsigned me = n_ext + c_ext, mr = n_rl + c_res;
        if (me > static_cast<unsigned>(K)) {
            const unsigned P = pow2_at_least(me);
            for (unsigned i = me + threadIdx.x; i < P; i += blockDim.x) ext[i] = ext_pad();
            __syncthreads();
            block_bitonic(ext, P, ext_before);
        }
        if (mr > static_cast<unsigned>(K)) {
            const unsigned P = pow2_at_least(mr);
            for (unsigned i = mr + threadIdx.x; i < P; i += blockDim.x) res[i] = ext_pad();
            __syncthreads();
            block_bitonic(res, P, ext_before);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            n_ext = min(me, static_cast<unsigned>(K));
            n_rl = min(mr, static_cast<unsigned>(K));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && n_fp64) atomicAdd(a.n_exact, n_fp64);
    // 3. children: the kept extensions (any order); the other child slots empty
    if (more) {
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            BeamPath* ch = a.next + slot * K + c;
            if (static_cast<unsigned>(c) < n_ext) {
                BeamPath cp = p;
                cp.score = ext[c].score;
                cp.r[a.level] = static_cast<uint16_t>(ext[c].r);
                cp.hops = a.level + 1;
                cp.v[a.level + 1] = ext[c].y;
                *ch = cp;
            } else {
                ch->hops = -1;
            }
        }
    }
    // 4. results: appended to the query's list
    if (n_rl) {
        if (threadIdx.x == 0) res_base = atomicAdd(a.n_res + q, n_rl);
        __syncthreads();
        for (unsigned c = threadIdx.x; c < n_rl; c += blockDim.x) {
            const int64_t pos = static_cast<int64_t>(res_base) + c;
            if (pos >= a.res_cap) continue;
            BeamPath rp = p;
            rp.score = res[c].score;
            rp.r[a.level] = static_cast<uint16_t>(res[c].r);
            rp.hops = a.level + 1;
            rp.v[a.level + 1] = tq;
            a.res[q * a.res_cap + pos] = rp;
        }
    }
}

__device__ __forceinline__ BeamPath result_pad() {
    BeamPath p;
    p.score = -INFINITY;
    p.hops = 0x7fffffff;
    for (int i = 0; i <= kBeamMaxH; ++i) p.v[i] = 0xffffffffu;
    for (int i = 0; i < kBeamMaxH; ++i) p.r[i] = 0xffff;
    return p;
}

// one CTA per query: the K best results in order
__global__ void __launch_bounds__(kBeamThreads) k_beam_final(const BeamPath* __restrict__ res, int64_t res_cap,
                                                             const unsigned* __restrict__ n_res, int K,
                                                             BeamPath* __restrict__ out, int32_t* __restrict__ n_out) {
    __shared__ BeamPath buf[kBeamBuf];
    const int64_t q = blockIdx.x;
    const int64_t n = min(static_cast<int64_t>(n_res[q]), res_cap);
    const BeamPath* a = res + q * res_cap;
    unsigned kept = 0;
    for (int64_t base = 0; base < n; base += kBeamChunk) {
        const unsigned c = static_cast<unsigned>(min(static_cast<int64_t>(kBeamChunk), n - base));
        for (unsigned i = threadIdx.x; i < c; i += blockDim.x) buf[kept + i] = a[base + i];
        __syncthreads();
        const unsigned m = kept + c;
        if (m > static_cast<unsigned>(K)) {
            const unsigned P = pow2_at_least(m);
            for (unsigned i = m + threadIdx.x; i < P; i += blockDim.x) buf[i] = result_pad();
            __syncthreads();
            block_bitonic(buf, P, result_before);
        }
        kept = min(m, static_cast<unsigned>(K));
        __syncthreads();
    }
    const unsigned P = pow2_at_least(kept);
    for (unsigned i = kept + threadIdx.x; i < P; i += blockDim.x) buf[i] = result_pad();
    __syncthreads();
    block_bitonic(buf, P, result_before);
    for (unsigned i = threadIdx.x; i < kept; i += blockDim.x) out[q * K + i] = buf[i];
    if (threadIdx.x == 0) n_out[q] = static_cast<int32_t>(kept);
}

}  // namespace
}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_beam_paths(const mhr_graph* g, int32_t nq, const uint32_t* s, const uint32_t* t,
                                     int32_t H, int32_t K, mhr_beam_path* out, int32_t* n_out, mhr_mem mem,
                                     mhr_stats* stats, void* cuda_stream) {
    const auto t_start = std::chrono::steady_clock::now();
    MHR_TRY(check_graph(g));
    if (nq < 0) return fail(MHR_EINVAL, "nq must be >= 0");
    if (H < 1 || H > MHR_BEAM_MAX_H) return fail(MHR_EINVAL, "H must be in [1, MHR_BEAM_MAX_H]");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_BEAM_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_BEAM_K_MAX");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    // level l holds K^l slots per query; the widest level is H - 1
    int64_t widest = 1, held_total = 0;
    for (int l = 0; l < H; ++l) {
        held_total += widest;
        if (l + 1 < H) {
            widest *= K;
            if (widest > (int64_t(1) << 16)) return fail(MHR_ERANGE, "K^(H-1) exceeds 65536");
        }
    }
    const int64_t res_cap = held_total * K;
    if (stats) *stats = mhr_stats{};
    if (nq == 0) return MHR_OK;
    if (!s || !t || !out || !n_out) return fail(MHR_EINVAL, "NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    std::vector<uint32_t> hs(nq), ht(nq);
    if (mem == MHR_MEM_HOST) {
        std::copy(s, s + nq, hs.begin());
        std::copy(t, t + nq, ht.begin());
    } else {
        MHR_CUDA_TRY(cudaMemcpyAsync(hs.data(), s, 4ull * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(ht.data(), t, 4ull * nq, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < nq; ++i) {
        if (static_cast<int64_t>(hs[i]) >= g->dg.n || static_cast<int64_t>(ht[i]) >= g->dg.n)
            return fail(MHR_EINVAL, "vertex out of range");
        if (hs[i] == ht[i]) return fail(MHR_EINVAL, "s == t");
    }

    // queries per round so that the level buffers and results stay within 1 GiB
    const size_t per_query = sizeof(BeamPath) * static_cast<size_t>(2 * widest + res_cap) + 64;
    const int QB = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t(1) << 30) / per_query)));
    std::vector<void*> bufs;
    auto cleanup = [&]() {
        for (void* b : bufs) cudaFree(b);
    };
    auto alloc = [&](void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) bufs.push_back(*p);
        return e;
    };
    BeamPath *A = nullptr, *B = nullptr, *R = nullptr, *d_out = reinterpret_cast<BeamPath*>(out);
    uint32_t *d_s = const_cast<uint32_t*>(s), *d_t = const_cast<uint32_t*>(t);
    unsigned* d_nres = nullptr;
    int32_t* d_nout = n_out;
    unsigned long long* d_scored = nullptr;  // [0] edges scored in fp32, [1] scored in fp64
    cudaError_t e = alloc(reinterpret_cast<void**>(&A), sizeof(BeamPath) * QB * widest);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&B), sizeof(BeamPath) * QB * widest);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&R), sizeof(BeamPath) * QB * res_cap);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&d_nres), 4ull * QB);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&d_scored), 16);
    if (e == cudaSuccess && mem == MHR_MEM_HOST) {
        e = alloc(reinterpret_cast<void**>(&d_out), sizeof(BeamPath) * static_cast<size_t>(nq) * K);
        if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&d_nout), 4ull * nq);
        if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&d_s), 4ull * nq);
        if (e == cudaSuccess) e = alloc(reinterpret_cast<void**>(&d_t), 4ull * nq);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, hs.data(), 4ull * nq, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, ht.data(), 4ull * nq, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_scored, 0, 16, st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "beam buffers");
    }
    for (int c0 = 0; c0 < nq && e == cudaSuccess; c0 += QB) {
        const int qb = std::min(QB, nq - c0);
        k_beam_init<<<(qb + 255) / 256, 256, 0, st>>>(d_s + c0, qb, A, d_nres);
        BeamPath *cur = A, *nxt = B;
        int64_t slots = 1;
        for (int l = 0; l < H; ++l) {
            LevelArgs a;
            a.g = g->dg;
            a.t = d_t + c0;
            a.level = l;
            a.H = H;
            a.K = K;
            a.slots = slots;
            a.cur = cur;
            a.next = nxt;
            a.res = R;
            a.res_cap = res_cap;
            a.n_res = d_nres;
            a.n_scored = d_scored;
            a.n_exact = d_scored + 1;
            a.e1 = (g->eps32_edge + g->eps64_edge) * (1.0 + 1e-6);
            k_beam_level<<<static_cast<unsigned>(qb * slots), kBeamThreads, 0, st>>>(a);
            std::swap(cur, nxt);
            slots *= K;
        }
        k_beam_final<<<qb, kBeamThreads, 0, st>>>(R, res_cap, d_nres, K, d_out + static_cast<int64_t>(c0) * K,
                                                  d_nout + c0);
        e = cudaGetLastError();
    }
    unsigned long long scored[2] = {0ull, 0ull};
    if (e == cudaSuccess && mem == MHR_MEM_HOST) {
        e = cudaMemcpyAsync(out, d_out, sizeof(BeamPath) * static_cast<size_t>(nq) * K, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(n_out, d_nout, 4ull * nq, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(scored, d_scored, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "beam search");
    if (stats) {
        stats->edges_scanned = static_cast<int64_t>(scored[0]);
        stats->rescored = static_cast<int64_t>(scored[1]);
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    return MHR_OK;
}
