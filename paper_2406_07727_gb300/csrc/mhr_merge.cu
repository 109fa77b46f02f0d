// Merge of partial top-K path lists (Alg. 2, ReduceTopKTree).
//
// The paper's threads each keep a K-best heap and merge them pairwise in a
// tree after a barrier.  Here the partial lists come from the parts of a
// vertex-partitioned search (one per GPU) and are already sorted in the
// result order; each tree round merges pairs of lists with one CTA per
// (query, pair): output position i finds, by a binary search along the merge
// path, how many of its predecessors come from each list, so all K outputs
// are placed in parallel.  A list pairs with nothing in a round when the
// number of lists is odd and is copied through.
#include <cuda_runtime.h>

#include <vector>

#include "mhr_internal.cuh"

namespace mhr {
namespace {

// device scratch of one call, freed when the call returns
struct MergeScratch {
    std::vector<void*> ptrs;
    ~MergeScratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t bytes) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

__device__ __forceinline__ bool path_before(const mhr_path& a, const mhr_path& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.u != b.u) return a.u < b.u;
    if (a.r1 != b.r1) return a.r1 < b.r1;
    if (a.v != b.v) return a.v < b.v;
    if (a.r2 != b.r2) return a.r2 < b.r2;
    return a.r3 < b.r3;
}

// lists [n_in][nq][K] with counts [n_in][nq] -> [ceil(n_in / 2)][nq][K]
__global__ void k_merge_round(int nq, int K, int n_in, const mhr_path* __restrict__ in, const int32_t* __restrict__ n_in_cnt,
                              mhr_path* __restrict__ out, int32_t* __restrict__ n_out_cnt) {
    const int q = blockIdx.x;
    const int pr = blockIdx.y;  // output list
    const int la = 2 * pr, lb = 2 * pr + 1;
    const mhr_path* A = in + (static_cast<int64_t>(la) * nq + q) * K;
    const int32_t ca = n_in_cnt[static_cast<int64_t>(la) * nq + q];
    const bool has_b = lb < n_in;
    const mhr_path* B = has_b ? in + (static_cast<int64_t>(lb) * nq + q) * K : nullptr;
    const int32_t cb = has_b ? n_in_cnt[static_cast<int64_t>(lb) * nq + q] : 0;
    mhr_path* C = out + (static_cast<int64_t>(pr) * nq + q) * K;
    if (ca < 0 || cb < 0) {  // an invalid query stays invalid
        if (threadIdx.x == 0) n_out_cnt[static_cast<int64_t>(pr) * nq + q] = -1;
        return;
    }
    const int na = min(ca, K), nb = min(cb, K);
    const int m = min(K, na + nb);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        // a = outputs before i taken from A
        int lo = max(0, i - nb), hi = min(i, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (path_before(A[mid], B[i - mid - 1])) lo = mid + 1;
            else hi = mid;
        }
        const int a = lo, b = i - lo;
        const bool from_a = a < na && (b >= nb || path_before(A[a], B[b]));
        C[i] = from_a ? A[a] : B[b];
    }
    if (threadIdx.x == 0) n_out_cnt[static_cast<int64_t>(pr) * nq + q] = m;
}

}  // namespace
}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_merge_paths(int32_t nq, int32_t K, int32_t n_parts, const mhr_path* parts,
                                      const int32_t* n_parts_out, mhr_path* out, int32_t* n_out, mhr_mem mem,
                                      void* cuda_stream) {
    if (nq < 0 || n_parts < 1) return fail(MHR_EINVAL, "nq must be >= 0 and n_parts >= 1");
    if (K < 1 || K > MHR_K_MAX) return fail(MHR_EINVAL, "K must be in [1, MHR_K_MAX]");
    if (mem != MHR_MEM_HOST && mem != MHR_MEM_DEVICE) return fail(MHR_EINVAL, "unknown mem kind");
    if (nq == 0) return MHR_OK;
    if (!parts || !n_parts_out || !out || !n_out) return fail(MHR_EINVAL, "a required pointer is NULL");
    if (nq > 65535 * 8) return fail(MHR_EINVAL, "nq too large for one merge call");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t lists = static_cast<size_t>(n_parts) * nq;
    const size_t pbytes = sizeof(mhr_path) * lists * K, cbytes = sizeof(int32_t) * lists;
    // two ping-pong buffers of lists and counts
    MergeScratch tmp;
    mhr_path *buf0 = nullptr, *buf1 = nullptr;
    int32_t *cnt0 = nullptr, *cnt1 = nullptr;
    MHR_CUDA_TRY(tmp.alloc(&buf0, pbytes));
    MHR_CUDA_TRY(tmp.alloc(&buf1, pbytes));
    MHR_CUDA_TRY(tmp.alloc(&cnt0, cbytes));
    MHR_CUDA_TRY(tmp.alloc(&cnt1, cbytes));
    const cudaMemcpyKind in_kind = mem == MHR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    MHR_CUDA_TRY(cudaMemcpyAsync(buf0, parts, pbytes, in_kind, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(cnt0, n_parts_out, cbytes, in_kind, st));
    int n = n_parts;
    if (n == 1) {
        // one list: still clamp counts above K and keep -1
        k_merge_round<<<dim3(nq, 1), 256, 0, st>>>(nq, K, 1, buf0, cnt0, buf1, cnt1);
        MHR_CUDA_TRY(cudaGetLastError());
        std::swap(buf0, buf1);
        std::swap(cnt0, cnt1);
    }
    while (n > 1) {
        const int m = (n + 1) / 2;
        k_merge_round<<<dim3(nq, m), 256, 0, st>>>(nq, K, n, buf0, cnt0, buf1, cnt1);
        MHR_CUDA_TRY(cudaGetLastError());
        std::swap(buf0, buf1);
        std::swap(cnt0, cnt1);
        n = m;
    }
    const cudaMemcpyKind out_kind = mem == MHR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    MHR_CUDA_TRY(cudaMemcpyAsync(out, buf0, sizeof(mhr_path) * static_cast<size_t>(nq) * K, out_kind, st));
    MHR_CUDA_TRY(cudaMemcpyAsync(n_out, cnt0, sizeof(int32_t) * nq, out_kind, st));
    // the scratch is freed when `tmp` leaves scope: wait for the copies first
    MHR_CUDA_TRY(cudaStreamSynchronize(st));
    return MHR_OK;
}
