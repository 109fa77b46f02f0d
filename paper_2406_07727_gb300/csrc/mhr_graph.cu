// Graph residency: upload, validation, reverse CSR, error bounds, edge scores.
//
// The graph is the paper's three inputs (Sec. 3.1): the (h, r, t) edge list
// as a CSR by head, the entity embedding table and the relation embedding
// table.  Per-relation edge tables and hash-table embedding stores of the
// CPU design (Alg. 1, Sec. 3.3) become one CSR with a relation id per edge,
// its transpose, and dense row-major embedding arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "mhr_internal.cuh"
#include "mhr_util.cuh"
#include <cuda_bf16.h>

static_assert(sizeof(mhr_graph_desc) == 104, "mhr_graph_desc layout");
static_assert(sizeof(mhr_path) == 24, "mhr_path layout");
static_assert(sizeof(mhr_query_opts) == 48, "mhr_query_opts layout");
static_assert(sizeof(mhr_constraints) == 40, "mhr_constraints layout");
static_assert(sizeof(mhr_graph_info) == 80, "mhr_graph_info layout");
static_assert(sizeof(mhr_mlp) == 32, "mhr_mlp layout");
static_assert(sizeof(mhr_stats) == 88, "mhr_stats layout");

namespace mhr {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

mhr_status fail(mhr_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

mhr_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MHR_ENOMEM : MHR_ECUDA;
}

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

mhr_status check_graph(const mhr_graph* g) {
    if (!g) return fail(MHR_EINVAL, "graph handle is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return fail(MHR_EINVAL, "the graph was loaded on another device than the current one");
    return MHR_OK;
}

// ---------------------------------------------------------------------------
// validation kernels (flags, never traps)
// ---------------------------------------------------------------------------
enum {
    kErrOffsets = 0,
    kErrColRange = 1,
    kErrRelRange = 2,
    kErrRowOrder = 3,
    kErrSelfLoop = 4,
    kErrNonFinite = 5,
    kErrCount = 8
};

__global__ void k_validate_offsets(const int64_t* __restrict__ off, int64_t n, int64_t E,
                                   int* __restrict__ err) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n; u += stride)
        if (off[u] > off[u + 1]) err[kErrOffsets] = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != E)) err[kErrOffsets] = 1;
}

__global__ void k_validate_rows(const int64_t* __restrict__ off, const uint32_t* __restrict__ col,
                                const uint16_t* __restrict__ rel, int64_t n, int32_t R,
                                int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t lo = off[u], hi = off[u + 1];
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const uint32_t c = col[p];
            const uint32_t r = rel[p];
            if (c >= static_cast<uint64_t>(n)) err[kErrColRange] = 1;
            if (r >= static_cast<uint32_t>(R)) err[kErrRelRange] = 1;
            if (c == static_cast<uint64_t>(u)) err[kErrSelfLoop] = 1;
            if (p > lo) {
                const uint32_t pc = col[p - 1];
                const uint32_t pr = rel[p - 1];
                if (!(pc < c || (pc == c && pr < r))) err[kErrRowOrder] = 1;
            }
        }
    }
}

__global__ void k_validate_finite(const void* __restrict__ tab, int dtype, int64_t count,
                                  int* __restrict__ err) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count; i += stride) {
        float x = dtype == MHR_F32 ? static_cast<const float*>(tab)[i]
                                   : bf16_to_f32(static_cast<const uint16_t*>(tab)[i]);
        if (!isfinite(x)) err[kErrNonFinite] = 1;
    }
}

// ---------------------------------------------------------------------------
// reverse CSR
// ---------------------------------------------------------------------------
__global__ void k_count_in(const uint32_t* __restrict__ col, int64_t E, uint32_t* __restrict__ indeg) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < E; p += stride)
        atomicAdd(&indeg[col[p]], 1u);
}

__global__ void k_make_keys(const uint32_t* __restrict__ col, int64_t E, int64_t N,
                            uint64_t* __restrict__ keys) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < N; p += stride)
        keys[p] = p < E ? ((static_cast<uint64_t>(col[p]) << 32) | static_cast<uint64_t>(p))
                        : ~0ull;
}

__device__ __forceinline__ int64_t row_of_edge(const int64_t* __restrict__ off, int64_t n, int64_t p) {
    // largest u with off[u] <= p (rows may be empty)
    int64_t lo = 0, hi = n;  // answer in [0, n)
    while (lo + 1 < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_fill_reverse(const uint64_t* __restrict__ keys, int64_t E,
                               const int64_t* __restrict__ off, int64_t n,
                               const uint16_t* __restrict__ rel, uint32_t* __restrict__ rcol,
                               uint16_t* __restrict__ rrel) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < E; i += stride) {
        const int64_t p = static_cast<int64_t>(keys[i] & 0xffffffffull);
        rcol[i] = static_cast<uint32_t>(row_of_edge(off, n, p));
        rrel[i] = rel[p];
    }
}

// ---------------------------------------------------------------------------
// norms behind the fp32 error bound
// ---------------------------------------------------------------------------
__global__ void k_row_norms(const void* __restrict__ tab, int dtype, int64_t rows, int d,
                            unsigned long long* __restrict__ max_l1,
                            unsigned long long* __restrict__ max_aux, int aux_is_inf) {
    // max over rows of ||x||_1 and of ||x||_2^2 (or ||x||_inf); non-negative
    // doubles compare like their bit patterns, so atomicMax on the bits works.
    __shared__ double s1[32], s2[32];
    double m1 = 0.0, m2 = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows; r += stride) {
        double l1 = 0.0, aux = 0.0;
        for (int j = 0; j < d; ++j) {
            double x = fabs(static_cast<double>(emb_f32(tab, dtype, r, d, j)));
            l1 += x;
            aux = aux_is_inf ? fmax(aux, x) : aux + x * x;
        }
        m1 = fmax(m1, l1);
        m2 = fmax(m2, aux);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s1[wid] = m1;
        s2[wid] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            m1 = fmax(m1, s1[w]);
            m2 = fmax(m2, s2[w]);
        }
        atomicMax(max_l1, static_cast<unsigned long long>(__double_as_longlong(m1)));
        atomicMax(max_aux, static_cast<unsigned long long>(__double_as_longlong(m2)));
    }
}

static double gam(double n, double u) { return n * u / (1.0 - n * u); }

// Bound on |S32 - S64| for one path (three edges), valid for any summation
// order of the fp32 screening arithmetic:
//   TransE: |fl32(w) - w| <= |gamma - fl32(gamma)| + g_{d+4}(2^-24) (N + |gamma| + 1)
//           with N = 2 max ||e||_1 + max ||w_r||_1 bounding sum |a|+|b|+|c|
//   DistMult: <= g_{d+3}(2^-24) M with M = max ||w_r||_inf * max ||e||_2^2
//           bounding sum |a b c| (Cauchy-Schwarz)
//   the same with 2^-53 for the fp64 value, plus the two path additions.
static void compute_bounds(mhr_graph* g) {
    const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
    const int d = g->dg.d;
    const double gamma = g->dg.gamma;
    double eps32, eps64, wmax;
    if (g->fn == MHR_SCORE_TRANSE_L1) {
        const double N = 2.0 * g->max_l1 + g->max_rel_l1;
        const double gerr = std::fabs(gamma - static_cast<double>(static_cast<float>(gamma)));
        eps32 = gerr + gam(d + 4, u32) * (N + std::fabs(gamma) + 1.0);
        eps64 = gam(d + 4, u64) * (N + std::fabs(gamma) + 1.0);
        wmax = std::fabs(gamma) + N;
    } else {
        const double M = g->max_rel_inf * g->max_l2sq;
        eps32 = gam(d + 3, u32) * M;
        eps64 = gam(d + 3, u64) * M;
        wmax = M;
    }
    g->eps32_edge = eps32;
    g->eps64_edge = eps64;
    const double path = 3.0 * (eps32 + eps64) +
                        (gam(2, u32) + gam(2, u64)) * 3.0 * (wmax + eps32 + eps64);
    g->err_path = path * (1.0 + 1e-6) + 1e-300;
    // Tensor-core middle-edge screen (DistMult): p_j = fl32(e_u[j] e_v[j]) is
    // split p = p_hi + p_lo + r with bf16 parts, |r| <= 2^-16 |p|; w_r likewise;
    // the products p_hi w_hi + p_hi w_lo + p_lo w_hi are exact in fp32 and the
    // dropped p_lo w_lo is <= 2^-16 |p w|, so each term is within
    // (2^-24 + 4 * 2^-16) |e_u e_v w| of the exact one.  The tensor-core fp32
    // accumulation (3 products per term, order unspecified) is bounded with a
    // unit roundoff of 2^-22 to allow for its alignment truncation.
    if (g->fn == MHR_SCORE_DISTMULT) {
        const double M = g->max_rel_inf * g->max_l2sq;
        const double term = std::ldexp(1.0, -24) + 4.0 * std::ldexp(1.0, -16);
        const double epstc = (term + gam(3.0 * d + 3, std::ldexp(1.0, -22)) * (1.0 + term)) * M;
        g->epstc_edge = epstc;
        const double ptc = 2.0 * eps32 + epstc + 3.0 * eps64 +
                           (gam(2, u32) + gam(2, u64)) * 3.0 * (wmax + epstc + eps32 + eps64);
        g->err_path_tc = ptc * (1.0 + 1e-6) + 1e-300;
    }
}

// bf16 hi / lo split of the relation table (tensor-core middle-edge screen)
__global__ void k_split_rel(const void* __restrict__ remb, int dtype, int64_t count, uint16_t* __restrict__ hi,
                            uint16_t* __restrict__ lo) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count; i += stride) {
        const float w = dtype == MHR_F32 ? static_cast<const float*>(remb)[i]
                                         : bf16_to_f32(static_cast<const uint16_t*>(remb)[i]);
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        hi[i] = __bfloat16_as_ushort(h);
        lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w - __bfloat162float(h)));
    }
}

// ---------------------------------------------------------------------------
// edge scores
// ---------------------------------------------------------------------------
__global__ void k_edge_scores32(DevGraph g, const uint32_t* __restrict__ src,
                                const uint16_t* __restrict__ rel, const uint32_t* __restrict__ dst,
                                int64_t m, int width, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (width - 1);
    const int64_t group = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / width;
    const int64_t ngroups = (static_cast<int64_t>(gridDim.x) * blockDim.x) / width;
    // every lane of the warp runs the same number of iterations (shuffles)
    const int64_t warp_first_group = group - (lane / width);
    const int64_t iters = (m + ngroups - 1) / ngroups;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = group + it * ngroups;
        const bool live = i < m;
        uint32_t u = 0, r = 0, v = 0;
        if (live) {
            if (src) {
                u = src[i];
                r = rel[i];
                v = dst[i];
            } else {
                u = static_cast<uint32_t>(row_of_edge(g.off, g.n, i));
                r = g.rel[i];
                v = g.col[i];
            }
        }
        const float w = edge_w32_group(g, u, r, v, sub, width);
        if (live && sub == 0) out[i] = w;
    }
    (void)warp_first_group;
}

__global__ void k_edge_scores64(DevGraph g, const uint32_t* __restrict__ src,
                                const uint16_t* __restrict__ rel, const uint32_t* __restrict__ dst,
                                int64_t m, double* __restrict__ out) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m; i += stride) {
        uint32_t u, r, v;
        if (src) {
            u = src[i];
            r = rel[i];
            v = dst[i];
        } else {
            u = static_cast<uint32_t>(row_of_edge(g.off, g.n, i));
            r = g.rel[i];
            v = g.col[i];
        }
        out[i] = edge_w64(g, u, r, v);
    }
}

// per-vertex maximum fp32 weight over out-edges and in-edges (order keys)
// Per-vertex maxima of the fp32 weight of its out- and in-edges and, when the
// tables are given, per (vertex, relation) maxima (kout_r[u * R + r]).
__global__ void k_vertex_maxw(DevGraph g, int width, uint32_t* __restrict__ kout, uint32_t* __restrict__ kin,
                              uint32_t* __restrict__ kout_r, uint32_t* __restrict__ kin_r) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (width - 1);
    const int64_t group = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / width;
    const int64_t ngroups = (static_cast<int64_t>(gridDim.x) * blockDim.x) / width;
    const int64_t iters = (g.E + ngroups - 1) / ngroups;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = group + it * ngroups;
        const bool live = i < g.E;
        uint32_t u = 0, r = 0, v = 0;
        if (live) {
            u = static_cast<uint32_t>(row_of_edge(g.off, g.n, i));
            r = g.rel[i];
            v = g.col[i];
        }
        const float w = edge_w32_group(g, u, r, v, sub, width);
        if (live && sub == 0) {
            const uint32_t k = f2key(w);
            atomicMax(&kout[u], k);
            atomicMax(&kin[v], k);
            if (kout_r) {
                atomicMax(&kout_r[static_cast<int64_t>(u) * g.R + r], k);
                atomicMax(&kin_r[static_cast<int64_t>(v) * g.R + r], k);
            }
        }
    }
}

// keys -> fp32 upper bounds: + slack (two fp32 evaluations of one edge in
// different summation orders differ by at most 2 * eps32), rounded up
__global__ void k_maxw_finish(uint32_t* __restrict__ a, int64_t n, double slack) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const uint32_t k = a[i];
        float f;
        if (k == 0u) f = __int_as_float(0xff800000);
        else f = __double2float_ru(__dadd_ru(static_cast<double>(key2f(k)), slack));
        a[i] = __float_as_uint(f);
    }
}

}  // namespace mhr

using namespace mhr;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

struct Scoped {
    std::vector<void*> ptrs;
    ~Scoped() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t bytes) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 1);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

void free_graph(mhr_graph* g);

// Device-memory cap of a resident graph (bytes), from MHR_GRAPH_MEMORY_CAP_BYTES;
// 0 = none.  Read at every load.
size_t graph_memory_cap() {
    const char* v = std::getenv("MHR_GRAPH_MEMORY_CAP_BYTES");
    if (!v || !*v) return 0;
    char* end = nullptr;
    const unsigned long long c = std::strtoull(v, &end, 10);
    return (end && *end == '\0') ? static_cast<size_t>(c) : 0;
}

mhr_status graph_alloc(mhr_graph* g, void** p, size_t bytes) {
    const size_t want = bytes ? bytes : 16;
    if (g->memory_cap && g->alloc_bytes + want > g->memory_cap) {
        *p = nullptr;
        return fail(MHR_ENOMEM, "graph device memory would exceed MHR_GRAPH_MEMORY_CAP_BYTES (" +
                                    std::to_string(g->memory_cap) + " bytes)");
    }
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc (graph)");
    }
    g->allocations.push_back(*p);
    g->alloc_bytes += want;
    return MHR_OK;
}

mhr_status load_impl(const mhr_graph_desc* desc, mhr_graph* g, cudaStream_t st) {
    const int64_t n = desc->n_vertices, E = desc->n_edges;
    const int R = desc->n_relations, d = desc->dim;
    const bool host = desc->mem == MHR_MEM_HOST;
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t esz = desc->emb_dtype == MHR_F32 ? 4 : 2;
    g->num_sms = device_sm_count();
    const int grid = std::max(1, g->num_sms) * 8;

    int64_t* off;
    uint32_t* col;
    uint16_t* rel;
    uint8_t* vt;
    void *vemb, *remb;
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&off), sizeof(int64_t) * (n + 1)));
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&col), sizeof(uint32_t) * E));
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&rel), sizeof(uint16_t) * E));
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&vt), n));
    MHR_TRY(graph_alloc(g, &vemb, esz * n * d));
    MHR_TRY(graph_alloc(g, &remb, esz * R * d));
    MHR_CUDA_TRY(cudaMemcpyAsync(off, desc->offsets, sizeof(int64_t) * (n + 1), kind, st));
    if (E) {
        MHR_CUDA_TRY(cudaMemcpyAsync(col, desc->cols, sizeof(uint32_t) * E, kind, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(rel, desc->rels, sizeof(uint16_t) * E, kind, st));
    }
    if (desc->vtypes) MHR_CUDA_TRY(cudaMemcpyAsync(vt, desc->vtypes, n, kind, st));
    else MHR_CUDA_TRY(cudaMemsetAsync(vt, 0, n, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(vemb, desc->vertex_emb, esz * n * d, kind, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(remb, desc->rel_emb, esz * R * d, kind, st));

    // --- validation
    Scoped tmp;
    int* err;
    MHR_CUDA_TRY(tmp.alloc(&err, sizeof(int) * kErrCount));
    MHR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int) * kErrCount, st));
    k_validate_offsets<<<grid, 256, 0, st>>>(off, n, E, err);
    int herr[kErrCount];
    MHR_CUDA_TRY(cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr[kErrOffsets])
        return fail(MHR_EINVAL, "offsets must start at 0, be non-decreasing and end at n_edges");
    k_validate_rows<<<grid, 256, 0, st>>>(off, col, rel, n, R, err);
    k_validate_finite<<<grid, 256, 0, st>>>(vemb, desc->emb_dtype, n * d, err);
    k_validate_finite<<<grid, 256, 0, st>>>(remb, desc->emb_dtype, static_cast<int64_t>(R) * d, err);
    MHR_CUDA_TRY(cudaGetLastError());
    MHR_CUDA_TRY(cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr[kErrColRange]) return fail(MHR_EINVAL, "a destination id is >= n_vertices");
    if (herr[kErrRelRange]) return fail(MHR_EINVAL, "a relation id is >= n_relations");
    if (herr[kErrSelfLoop]) return fail(MHR_EINVAL, "self loops are not allowed");
    if (herr[kErrRowOrder])
        return fail(MHR_EINVAL, "each row must be sorted by (col, rel) without repeated (col, rel)");
    if (herr[kErrNonFinite]) return fail(MHR_EINVAL, "an embedding value is NaN or infinite");

    // --- reverse CSR (in-edges of each vertex, rows sorted by (source, relation))
    int64_t* roff;
    uint32_t* rcol;
    uint16_t* rrel;
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&roff), sizeof(int64_t) * (n + 1)));
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&rcol), sizeof(uint32_t) * E));
    MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&rrel), sizeof(uint16_t) * E));
    {
        uint32_t* indeg;
        int64_t *n_dev, *partials;
        MHR_CUDA_TRY(tmp.alloc(&indeg, sizeof(uint32_t) * n));
        MHR_CUDA_TRY(tmp.alloc(&n_dev, sizeof(int64_t)));
        MHR_CUDA_TRY(tmp.alloc(&partials, sizeof(int64_t) * kScanPartials));
        MHR_CUDA_TRY(cudaMemsetAsync(partials, 0, sizeof(int64_t) * kScanPartials, st));
        MHR_CUDA_TRY(cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * n, st));
        MHR_CUDA_TRY(cudaMemcpyAsync(n_dev, &n, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        if (E) k_count_in<<<grid, 256, 0, st>>>(col, E, indeg);
        MHR_CUDA_TRY(device_excl_scan<uint32_t>(indeg, n_dev, partials, roff, st));
        if (E) {
            int64_t N = kBitonicTile;
            while (N < E) N <<= 1;
            uint64_t* keys;
            MHR_CUDA_TRY(tmp.alloc(&keys, sizeof(uint64_t) * N));
            k_make_keys<<<grid, 256, 0, st>>>(col, E, N, keys);
            MHR_CUDA_TRY(bitonic_sort_u64(keys, static_cast<uint64_t>(N), std::max(1, g->num_sms), st));
            k_fill_reverse<<<grid, 256, 0, st>>>(keys, E, off, n, rel, rcol, rrel);
            MHR_CUDA_TRY(cudaGetLastError());
        }
        // the scan wrote n_dev-long output plus the total at roff[n]
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // --- host copies of row starts (query sizing)
    g->h_off.resize(n + 1);
    g->h_roff.resize(n + 1);
    MHR_CUDA_TRY(cudaMemcpyAsync(g->h_off.data(), off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(g->h_roff.data(), roff, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));

    // --- norms
    unsigned long long* mx;
    MHR_CUDA_TRY(tmp.alloc(&mx, sizeof(unsigned long long) * 4));
    MHR_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 4, st));
    k_row_norms<<<grid, 256, 0, st>>>(vemb, desc->emb_dtype, n, d, mx + 0, mx + 1, 0);
    k_row_norms<<<std::max(1, std::min(grid, (R + 255) / 256)), 256, 0, st>>>(remb, desc->emb_dtype, R, d,
                                                                               mx + 2, mx + 3, 1);
    MHR_CUDA_TRY(cudaGetLastError());
    unsigned long long hm[4];
    MHR_CUDA_TRY(cudaMemcpyAsync(hm, mx, sizeof hm, cudaMemcpyDeviceToHost, st));
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    double dm[4];
    std::memcpy(dm, hm, sizeof dm);
    g->max_l1 = dm[0];
    g->max_l2sq = dm[1];
    g->max_rel_l1 = dm[2];
    g->max_rel_inf = dm[3];
    if (g->h_roff[n] != E) return fail(MHR_ECUDA, "reverse CSR construction is inconsistent");
    for (int64_t u = 0; u < n; ++u) {
        g->max_out_deg = std::max(g->max_out_deg, g->h_off[u + 1] - g->h_off[u]);
        g->max_in_deg = std::max(g->max_in_deg, g->h_roff[u + 1] - g->h_roff[u]);
    }

    DevGraph& dg = g->dg;
    dg.n = n;
    dg.E = E;
    dg.R = R;
    dg.d = d;
    dg.dtype = desc->emb_dtype;
    dg.fn = desc->score_fn;
    dg.gamma = desc->gamma;
    dg.gamma32 = static_cast<float>(desc->gamma);
    dg.off = off;
    dg.col = col;
    dg.rel = rel;
    dg.roff = roff;
    dg.rcol = rcol;
    dg.rrel = rrel;
    dg.vtypes = vt;
    dg.vemb = vemb;
    dg.remb = remb;
    g->fn = desc->score_fn;
    compute_bounds(g);
    if (g->fn == MHR_SCORE_DISTMULT) {
        const int64_t cnt = static_cast<int64_t>(R) * d;
        MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&g->wsplit), sizeof(uint16_t) * 2 * cnt));
        k_split_rel<<<std::max(1, std::min(grid, static_cast<int>((cnt + 255) / 256))), 256, 0, st>>>(
            remb, desc->emb_dtype, cnt, g->wsplit, g->wsplit + cnt);
        MHR_CUDA_TRY(cudaGetLastError());
    }
    // per-vertex bounds on the fp32 weight of adjacent edges (bound pruning),
    // and per (vertex, relation) bounds when n x R entries stay within
    // kMaxRelBoundEntries (4 bytes each, two tables)
    {
        uint32_t *kout, *kin, *kout_r = nullptr, *kin_r = nullptr;
        MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&kout), sizeof(uint32_t) * n));
        MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&kin), sizeof(uint32_t) * n));
        MHR_CUDA_TRY(cudaMemsetAsync(kout, 0, sizeof(uint32_t) * n, st));
        MHR_CUDA_TRY(cudaMemsetAsync(kin, 0, sizeof(uint32_t) * n, st));
        const int64_t nr = n * static_cast<int64_t>(R);
        if (nr <= kMaxRelBoundEntries) {
            MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&kout_r), sizeof(uint32_t) * nr));
            MHR_TRY(graph_alloc(g, reinterpret_cast<void**>(&kin_r), sizeof(uint32_t) * nr));
            MHR_CUDA_TRY(cudaMemsetAsync(kout_r, 0, sizeof(uint32_t) * nr, st));
            MHR_CUDA_TRY(cudaMemsetAsync(kin_r, 0, sizeof(uint32_t) * nr, st));
        }
        if (E)
            k_vertex_maxw<<<grid, 256, 0, st>>>(dg, score_group_width(d, desc->emb_dtype), kout, kin, kout_r, kin_r);
        k_maxw_finish<<<grid, 256, 0, st>>>(kout, n, 2.0 * g->eps32_edge);
        k_maxw_finish<<<grid, 256, 0, st>>>(kin, n, 2.0 * g->eps32_edge);
        if (kout_r) {
            k_maxw_finish<<<grid, 256, 0, st>>>(kout_r, nr, 2.0 * g->eps32_edge);
            k_maxw_finish<<<grid, 256, 0, st>>>(kin_r, nr, 2.0 * g->eps32_edge);
        }
        MHR_CUDA_TRY(cudaGetLastError());
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
        dg.maxw_out = reinterpret_cast<const float*>(kout);
        dg.maxw_in = reinterpret_cast<const float*>(kin);
        dg.maxw_out_r = reinterpret_cast<const float*>(kout_r);
        dg.maxw_in_r = reinterpret_cast<const float*>(kin_r);
    }
    const double big = 1e30;
    if (!(g->max_l1 < big && g->max_rel_l1 < big && g->max_l2sq < big && g->max_rel_inf < big &&
          g->err_path < 1e20))
        return fail(MHR_EINVAL, "embedding magnitudes are too large for fp32 screening");
    return MHR_OK;
}

void free_graph(mhr_graph* g);

}  // namespace

namespace mhr {
void destroy_plans(mhr_graph* g);  // mhr_query.cu
void destroy_tail(mhr_graph* g);   // mhr_tail.cu
}

namespace {
void free_graph(mhr_graph* g) {
    if (!g) return;
    mhr::destroy_plans(g);
    mhr::destroy_tail(g);
    for (void* p : g->allocations) cudaFree(p);
    delete g;
}
}  // namespace

extern "C" mhr_status mhr_graph_load(const mhr_graph_desc* desc, mhr_graph** out, void* cuda_stream) {
    if (!out) return fail(MHR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(MHR_EINVAL, "desc is NULL");
    if (desc->n_vertices < 1 || desc->n_vertices >= (1ll << 32))
        return fail(MHR_EINVAL, "n_vertices must be in [1, 2^32)");
    if (desc->n_edges < 0 || desc->n_edges >= (1ll << 32)) return fail(MHR_EINVAL, "n_edges must be in [0, 2^32)");
    if (desc->n_relations < 1 || desc->n_relations > 65536) return fail(MHR_EINVAL, "n_relations must be in [1, 65536]");
    if (desc->dim < 1 || desc->dim > 65536) return fail(MHR_EINVAL, "dim must be in [1, 65536]");
    if (desc->emb_dtype != MHR_F32 && desc->emb_dtype != MHR_BF16) return fail(MHR_EINVAL, "unknown emb_dtype");
    if (desc->mem != MHR_MEM_HOST && desc->mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    if (desc->score_fn != MHR_SCORE_TRANSE_L1 && desc->score_fn != MHR_SCORE_DISTMULT)
        return fail(MHR_EINVAL, "unknown score_fn");
    if (!std::isfinite(desc->gamma)) return fail(MHR_EINVAL, "gamma must be finite");
    if (!desc->offsets || (desc->n_edges && (!desc->cols || !desc->rels)) || !desc->vertex_emb || !desc->rel_emb)
        return fail(MHR_EINVAL, "a required array pointer is NULL");
    if (desc->mem == MHR_MEM_HOST) {
        const int64_t* o = desc->offsets;
        if (o[0] != 0 || o[desc->n_vertices] != desc->n_edges)
            return fail(MHR_EINVAL, "offsets must start at 0 and end at n_edges");
    }
    mhr_graph* g = new (std::nothrow) mhr_graph();
    if (!g) return fail(MHR_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(MHR_ECUDA, "no CUDA device");
    }
    g->memory_cap = graph_memory_cap();
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    mhr_status rc = load_impl(desc, g, st);
    if (rc != MHR_OK) {
        cudaStreamSynchronize(st);
        std::string keep = mhr_last_error();
        free_graph(g);
        set_error(keep);
        return rc;
    }
    *out = g;
    return MHR_OK;
}

extern "C" mhr_status mhr_graph_free(mhr_graph* g) {
    if (!g) return MHR_OK;
    cudaDeviceSynchronize();
    free_graph(g);
    return MHR_OK;
}

extern "C" mhr_status mhr_edge_scores(const mhr_graph* g, const uint32_t* src, const uint16_t* rel,
                                      const uint32_t* dst, int64_t n, int32_t precision, void* out,
                                      mhr_mem mem, void* cuda_stream) {
    MHR_TRY(check_graph(g));
    if (n < 0) return fail(MHR_EINVAL, "n must be >= 0");
    if (precision != 0 && precision != 2) return fail(MHR_EINVAL, "precision must be 0 (fp32) or 2 (fp64)");
    if (!out && n) return fail(MHR_EINVAL, "out is NULL");
    if (!src != !rel || !src != !dst) return fail(MHR_EINVAL, "src, rel and dst must all be given or all NULL");
    if (!src && n != g->dg.E) return fail(MHR_EINVAL, "with src == NULL, n must equal n_edges");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    if (n == 0) return MHR_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t osz = precision == 0 ? 4 : 8;
    Scoped tmp;
    const uint32_t *ds = src, *dd = dst;
    const uint16_t* dr = rel;
    void* dout = out;
    if (mem == MHR_MEM_HOST) {
        if (src) {
            uint32_t *a, *c;
            uint16_t* b;
            MHR_CUDA_TRY(tmp.alloc(&a, 4 * n));
            MHR_CUDA_TRY(tmp.alloc(&b, 2 * n));
            MHR_CUDA_TRY(tmp.alloc(&c, 4 * n));
            MHR_CUDA_TRY(cudaMemcpyAsync(a, src, 4 * n, cudaMemcpyHostToDevice, st));
            MHR_CUDA_TRY(cudaMemcpyAsync(b, rel, 2 * n, cudaMemcpyHostToDevice, st));
            MHR_CUDA_TRY(cudaMemcpyAsync(c, dst, 4 * n, cudaMemcpyHostToDevice, st));
            ds = a;
            dr = b;
            dd = c;
        }
        void* o;
        MHR_CUDA_TRY(tmp.alloc(&o, osz * n));
        dout = o;
    }
    // ids must be in range: checked on the device copy is costly; validate host
    // arrays here when they are on the host
    if (mem == MHR_MEM_HOST && src) {
        for (int64_t i = 0; i < n; ++i)
            if (src[i] >= g->dg.n || dst[i] >= g->dg.n || rel[i] >= g->dg.R)
                return fail(MHR_EINVAL, "edge id out of range");
    }
    const int sms = std::max(1, g->num_sms);
    if (precision == 0) {
        const int width = score_group_width(g->dg.d, g->dg.dtype);
        k_edge_scores32<<<sms * 8, 256, 0, st>>>(g->dg, ds, dr, dd, n, width, static_cast<float*>(dout));
    } else {
        k_edge_scores64<<<sms * 16, 128, 0, st>>>(g->dg, ds, dr, dd, n, static_cast<double*>(dout));
    }
    MHR_CUDA_TRY(cudaGetLastError());
    if (mem == MHR_MEM_HOST) {
        MHR_CUDA_TRY(cudaMemcpyAsync(out, dout, osz * n, cudaMemcpyDeviceToHost, st));
        MHR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MHR_OK;
}

extern "C" mhr_status mhr_graph_get_info(const mhr_graph* g, mhr_graph_info* out) {
    MHR_TRY(check_graph(g));
    if (!out) return fail(MHR_EINVAL, "out is NULL");
    out->n_vertices = g->dg.n;
    out->n_edges = g->dg.E;
    out->n_relations = g->dg.R;
    out->dim = g->dg.d;
    out->max_out_degree = g->max_out_deg;
    out->max_in_degree = g->max_in_deg;
    out->eps32_edge = g->eps32_edge;
    out->eps64_edge = g->eps64_edge;
    out->err_path = g->err_path;
    out->epstc_edge = g->epstc_edge;
    out->err_path_tc = g->err_path_tc;
    return MHR_OK;
}

extern "C" const char* mhr_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* mhr_version(void) { return "mhr-gb300 0.1 (sm_103a)"; }
