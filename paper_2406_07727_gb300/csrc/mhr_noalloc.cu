// One-query top-K search that allocates nothing.
//
// The batched engine sizes its work buffers per call and grows them with
// cudaMalloc.  Some callers cannot allow that: code running inside a stream
// capture it does not own (an allocation there breaks the capture), services
// that must keep a fixed device-memory footprint after start-up, and hosts
// that hand the library a stream inside a latency-critical section where the
// implicit synchronisation of cudaMalloc/cudaFree is not acceptable.  For them,
// mhr_topk_paths_noalloc runs one fused kernel whose only global scratch is a
// file-scope array of fixed size declared below; the caller passes the inputs
// (the loaded graph, s, t, K) and the output buffers.
//
// The kernel is the single-query form of the exact (tie-safe) path: fp32
// screening weights of the hop-1 and hop-3 edges in the scratch array, a
// brute-force walk over the middle edges with a binary search in the reverse
// row of t, and an exact top-K (fp64 rescoring in the canonical order of every
// candidate the fp32 screen cannot separate from the running K-th score).
#include <cuda_runtime.h>

#include <mutex>

#include "mhr_internal.cuh"
#include "mhr_util.cuh"

namespace mhr {

// Largest hop-1 row (out-degree of s) and hop-3 row (in-degree of t) the
// no-allocation entry point accepts.
constexpr int kNoAllocMaxFrontier = 65536;

// Scratch shared by every call on a device, kept between calls:
//   [0, M)            fp32 weight of hop-1 entry i  (w(s, r1, u))
//   [M, 2M)           fp32 weight of hop-3 entry j  (w(v, r3, t))
//   [2M, 2M + 2M + 2) uint64 prefix of middle-row lengths over hop-1 entries
// (M = kNoAllocMaxFrontier).  Every cell a call reads is written earlier in
// the same call, so nothing needs clearing.  About 1 MiB per device.
constexpr size_t kNoAllocScratchWords = 2 * kNoAllocMaxFrontier + 2 * (kNoAllocMaxFrontier + 1);
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchWords];

constexpr int kNaThreads = 1024;
constexpr int kNaBuf = 4096;

struct NoAllocSmem {
    mhr_path buf[kNaBuf];  // [0, K) running top K, [K, kNaBuf) staging
    uint32_t hi[kNaThreads], hp[kNaThreads], hc0[kNaThreads], hcn[kNaThreads];
    float hw2[kNaThreads];
    int64_t hcomb[kNaThreads + 1];
    int64_t red[33];
    int nt, ns, hit_cnt;
    double thr64;
};

__device__ bool na_before(const mhr_path& a, const mhr_path& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.u != b.u) return a.u < b.u;
    if (a.r1 != b.r1) return a.r1 < b.r1;
    if (a.v != b.v) return a.v < b.v;
    if (a.r2 != b.r2) return a.r2 < b.r2;
    return a.r3 < b.r3;
}

__device__ mhr_path na_worst() {
    mhr_path p;
    p.score = __longlong_as_double(0xfff0000000000000ll);
    p.u = p.v = 0xffffffffu;
    p.r1 = p.r2 = p.r3 = p.pad = 0xffff;
    return p;
}

// keep the K best of the running top K and the staged candidates
__device__ void na_flush(NoAllocSmem& sm, int K) {
    __syncthreads();
    const int nt = sm.nt, ns = sm.ns;
    for (int i = threadIdx.x; i < kNaBuf; i += blockDim.x)
        if (!((i < nt) || (i >= K && i < K + ns))) sm.buf[i] = na_worst();
    __syncthreads();
    for (int k = 2; k <= kNaBuf; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < kNaBuf / 2; t += blockDim.x) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const bool asc = (i & k) == 0;
                mhr_path x = sm.buf[i], y = sm.buf[i + j];
                if (asc ? na_before(y, x) : na_before(x, y)) {
                    sm.buf[i] = y;
                    sm.buf[i + j] = x;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        sm.nt = min(K, nt + ns);
        sm.ns = 0;
        if (sm.nt == K) sm.thr64 = sm.buf[K - 1].score;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kNaThreads) k_topk_noalloc(DevGraph g, uint32_t s, uint32_t t, int K, double err,
                                                             uint32_t* __restrict__ scratch,
                                                             mhr_path* __restrict__ out,
                                                             int32_t* __restrict__ n_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NoAllocSmem& sm = *reinterpret_cast<NoAllocSmem*>(smem_raw);
    float* wA = reinterpret_cast<float*>(scratch);
    float* wC = reinterpret_cast<float*>(scratch + kNoAllocMaxFrontier);
    uint64_t* pref = reinterpret_cast<uint64_t*>(scratch + 2 * kNoAllocMaxFrontier);
    const int64_t os = g.off[s], na = g.off[s + 1] - os;
    const int64_t rs = g.roff[t], nc = g.roff[t + 1] - rs;

    // hop-1 and hop-3 fp32 weights; excluded endpoints get -inf
    for (int64_t i = threadIdx.x; i < na; i += blockDim.x) {
        const uint32_t u = g.col[os + i];
        wA[i] = (u == s || u == t) ? __int_as_float(0xff800000) : edge_w32_group(g, s, g.rel[os + i], u, 0, 1);
    }
    for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
        const uint32_t v = g.rcol[rs + j];
        wC[j] = (v == s || v == t) ? __int_as_float(0xff800000) : edge_w32_group(g, v, g.rrel[rs + j], t, 0, 1);
    }
    // prefix of middle-row lengths over hop-1 entries (excluded entries: 0)
    int64_t carry = 0;
    for (int64_t b = 0; b < na; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        int64_t len = 0;
        if (i < na) {
            const uint32_t u = g.col[os + i];
            if (u != s && u != t) len = g.off[u + 1] - g.off[u];
        }
        int64_t tot;
        const int64_t ex = block_excl_scan(len, sm.red, &tot);
        if (i < na) pref[i] = static_cast<uint64_t>(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        pref[na] = static_cast<uint64_t>(carry);
        sm.nt = 0;
        sm.ns = 0;
        sm.thr64 = __longlong_as_double(0xfff0000000000000ll);
    }
    __syncthreads();
    const int64_t total = carry;
    const uint32_t* rcolt = g.rcol + rs;

    for (int64_t eb = 0; eb < total; eb += blockDim.x) {
        if (threadIdx.x == 0) sm.hit_cnt = 0;
        __syncthreads();
        const int64_t e = eb + threadIdx.x;
        if (e < total) {
            int lo = 0, hi = static_cast<int>(na);  // hop-1 entry: largest i with pref[i] <= e
            while (lo + 1 < hi) {
                const int mid = (lo + hi) >> 1;
                if (pref[mid] <= static_cast<uint64_t>(e)) lo = mid;
                else hi = mid;
            }
            const uint32_t u = g.col[os + lo];
            const int64_t p2 = g.off[u] + (e - static_cast<int64_t>(pref[lo]));
            const uint32_t v = g.col[p2];
            if (v != s && v != t && v != u) {
                int a = 0, b = static_cast<int>(nc);  // first hop-3 entry with source >= v
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if (rcolt[mid] < v) a = mid + 1;
                    else b = mid;
                }
                int c1 = a;
                while (c1 < nc && rcolt[c1] == v) ++c1;
                if (c1 > a) {
                    const int slot = atomicAdd(&sm.hit_cnt, 1);
                    sm.hi[slot] = static_cast<uint32_t>(lo);
                    sm.hp[slot] = static_cast<uint32_t>(p2);
                    sm.hc0[slot] = static_cast<uint32_t>(a);
                    sm.hcn[slot] = static_cast<uint32_t>(c1 - a);
                    sm.hw2[slot] = edge_w32_group(g, u, g.rel[p2], v, 0, 1);
                }
            }
        }
        __syncthreads();
        const int nh = sm.hit_cnt;
        const int64_t comb = threadIdx.x < nh ? static_cast<int64_t>(sm.hcn[threadIdx.x]) : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(comb, sm.red, &tot);
        if (threadIdx.x < nh) sm.hcomb[threadIdx.x] = ex;
        if (threadIdx.x == 0) sm.hcomb[nh] = tot;
        __syncthreads();
        for (int64_t cb = 0; cb < tot; cb += blockDim.x) {
            if (sm.ns + static_cast<int>(blockDim.x) > kNaBuf - K) na_flush(sm, K);
            const int64_t c = cb + threadIdx.x;
            if (c < tot) {
                int lo = 0, hi = nh;
                while (lo + 1 < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.hcomb[mid] <= c) lo = mid;
                    else hi = mid;
                }
                const uint32_t ia = sm.hi[lo];
                const uint32_t jc = sm.hc0[lo] + static_cast<uint32_t>(c - sm.hcomb[lo]);
                const float s32 = __fadd_rn(__fadd_rn(wA[ia], sm.hw2[lo]), wC[jc]);
                const double thr = sm.thr64;
                if (static_cast<double>(s32) + err >= thr) {
                    mhr_path p;
                    p.u = g.col[os + ia];
                    p.r1 = g.rel[os + ia];
                    p.v = g.col[sm.hp[lo]];
                    p.r2 = g.rel[sm.hp[lo]];
                    p.r3 = g.rrel[rs + jc];
                    p.pad = 0;
                    const double w1 = edge_w64(g, s, p.r1, p.u);
                    const double w2 = edge_w64(g, p.u, p.r2, p.v);
                    const double w3 = edge_w64(g, p.v, p.r3, t);
                    p.score = __dadd_rn(__dadd_rn(w1, w2), w3);
                    if (p.score >= thr) sm.buf[K + atomicAdd(&sm.ns, 1)] = p;
                }
            }
            __syncthreads();
        }
    }
    na_flush(sm, K);
    for (int i = threadIdx.x; i < sm.nt; i += blockDim.x) out[i] = sm.buf[i];
    if (threadIdx.x == 0) *n_out = sm.nt;
}

// per-device address of the scratch array (host code cannot use the symbol
// itself: in host code it names a host-side stand-in, not device memory)
static std::mutex g_na_mu;
static void* g_na_ptr[256];
static bool g_na_attr[256];

static mhr_status noalloc_setup(int dev, uint32_t** ptr) {
    if (dev < 0 || dev >= 256) return fail(MHR_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress (no-allocation scratch)");
        g_na_ptr[dev] = p;
    }
    if (!g_na_attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_topk_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sizeof(NoAllocSmem)));
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute (no-allocation kernel)");
        g_na_attr[dev] = true;
    }
    *ptr = static_cast<uint32_t*>(g_na_ptr[dev]);
    return MHR_OK;
}

}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_topk_paths_noalloc(const mhr_graph* g, uint32_t s, uint32_t t, int32_t K, mhr_path* out,
                                             int32_t* n_out, void* cuda_stream) {
    MHR_TRY(check_graph(g));
    if (!out || !n_out) return fail(MHR_EINVAL, "out and n_out (device pointers) are required");
    if (s >= g->dg.n || t >= g->dg.n) return fail(MHR_EINVAL, "s or t is out of range");
    if (s == t) return fail(MHR_EINVAL, "s == t");
    if (K < 1) return fail(MHR_EINVAL, "K must be >= 1");
    if (K > MHR_K_MAX) return fail(MHR_ERANGE, "K exceeds MHR_K_MAX");
    const int64_t na = g->h_off[s + 1] - g->h_off[s];
    const int64_t nc = g->h_roff[t + 1] - g->h_roff[t];
    if (na > kNoAllocMaxFrontier || nc > kNoAllocMaxFrontier)
        return fail(MHR_ERANGE,
                    "mhr_topk_paths_noalloc: out-degree of s and in-degree of t must each be <= 65536 "
                    "(the size of its fixed scratch); use mhr_topk_paths_batched for larger frontiers");
    uint32_t* scratch = nullptr;
    MHR_TRY(noalloc_setup(g->device, &scratch));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_topk_noalloc<<<1, kNaThreads, sizeof(NoAllocSmem), st>>>(g->dg, s, t, K, g->err_path, scratch, out, n_out);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}
