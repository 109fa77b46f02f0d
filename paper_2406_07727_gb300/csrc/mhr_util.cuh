// Device-wide building blocks: block scans, a fixed-grid exclusive scan whose
// length is read from device memory (so it can live inside a captured CUDA
// graph while the length changes between replays), and a bitonic sort of
// 64-bit keys used once per graph load.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mhr {

constexpr int kScanThreads = 1024;
constexpr int kScanGrid = 256;  // fixed number of blocks for the device-wide scan

// inclusive warp scan
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan (blockDim.x a multiple of 32, <= 1024).  `smem` holds
// 33 values.  Returns the exclusive prefix; *total receives the block total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* smem, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(x);
    if (lane == 31) smem[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T v = lane < nw ? smem[lane] : T(0);
        T vi = warp_incl_scan(v);
        if (lane < nw) smem[lane] = vi - v;
        if (lane == nw - 1) smem[32] = vi;
    }
    __syncthreads();
    T res = inc - x + smem[wid];
    if (total) *total = smem[32];
    __syncthreads();
    return res;
}

template <typename T>
__device__ __forceinline__ T block_sum(T x, T* smem) {
    T tot;
    block_excl_scan(x, smem, &tot);
    return tot;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan over n = *n_dev elements: out[i] = sum in[0..i),
// out[n] = total.  Two launches with a fixed grid of kScanGrid blocks; each
// block owns one contiguous range.  `partials` holds kScanPartials int64: the
// block sums, the total, and a completion counter that must be zero before
// the first scan (the last block resets it).
// ---------------------------------------------------------------------------
constexpr int kScanPartials = kScanGrid + 2;

// block sums; the last block to finish turns them into exclusive offsets
template <typename TIn>
__global__ void __launch_bounds__(kScanThreads)
scan_partials_kernel(const TIn* __restrict__ in, const int64_t* __restrict__ n_dev, int64_t* __restrict__ partials) {
    __shared__ int64_t sm[33];
    __shared__ int last;
    const int64_t n = *n_dev;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
    int64_t acc = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += static_cast<int64_t>(in[i]);
    const int64_t tot = block_sum(acc, sm);
    unsigned long long* done = reinterpret_cast<unsigned long long*>(partials + gridDim.x + 1);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        __threadfence();
        last = atomicAdd(done, 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int64_t carry = 0;
    for (int base = 0; base < static_cast<int>(gridDim.x); base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int64_t v = i < static_cast<int>(gridDim.x) ? __ldcg(partials + i) : 0;
        int64_t t;
        const int64_t ex = block_excl_scan(v, sm, &t);
        if (i < static_cast<int>(gridDim.x)) partials[i] = ex + carry;
        carry += t;
    }
    if (threadIdx.x == 0) {
        partials[gridDim.x] = carry;
        *done = 0ull;
    }
}

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(const TIn* __restrict__ in, const int64_t* __restrict__ n_dev,
                  const int64_t* __restrict__ partials, int64_t* __restrict__ out) {
    __shared__ int64_t sm[33];
    const int64_t n = *n_dev;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
    int64_t carry = partials[blockIdx.x];
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < hi ? static_cast<int64_t>(in[i]) : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, sm, &tot);
        if (i < hi) out[i] = carry + ex;
        carry += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = partials[gridDim.x];
}

template <typename TIn>
inline cudaError_t device_excl_scan(const TIn* in, const int64_t* n_dev, int64_t* partials,
                                    int64_t* out, cudaStream_t st) {
    scan_partials_kernel<TIn><<<kScanGrid, kScanThreads, 0, st>>>(in, n_dev, partials);
    scan_apply_kernel<TIn><<<kScanGrid, kScanThreads, 0, st>>>(in, n_dev, partials, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bitonic sort of N = 2^k uint64 keys, ascending.  Stages with stride below
// kBitonicTile/2 run inside shared memory.
// ---------------------------------------------------------------------------
constexpr int kBitonicThreads = 1024;
constexpr int kBitonicTile = 2 * kBitonicThreads;

static __global__ void __launch_bounds__(kBitonicThreads)
bitonic_shared_kernel(uint64_t* __restrict__ keys, uint64_t kmin, uint64_t kmax_stage) {
    // runs stages (k, j) for k in [kmin, kmax_stage] (k == kmin only when kmin > tile)
    __shared__ uint64_t s[kBitonicTile];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kBitonicTile;
    s[threadIdx.x] = keys[base + threadIdx.x];
    s[threadIdx.x + kBitonicThreads] = keys[base + threadIdx.x + kBitonicThreads];
    __syncthreads();
    for (uint64_t k = kmin; k <= kmax_stage; k <<= 1) {
        uint64_t jstart = (k > static_cast<uint64_t>(kBitonicTile)) ? (kBitonicTile >> 1) : (k >> 1);
        for (uint64_t j = jstart; j > 0; j >>= 1) {
            // thread t handles pair (i, i+j) with i having bit j clear
            uint64_t t = threadIdx.x;
            uint64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
            uint64_t gi = base + i;
            bool asc = (gi & k) == 0;
            uint64_t a = s[i], b = s[i + j];
            if ((a > b) == asc) {
                s[i] = b;
                s[i + j] = a;
            }
            __syncthreads();
        }
    }
    keys[base + threadIdx.x] = s[threadIdx.x];
    keys[base + threadIdx.x + kBitonicThreads] = s[threadIdx.x + kBitonicThreads];
}

static __global__ void bitonic_global_kernel(uint64_t* __restrict__ keys, uint64_t N, uint64_t k, uint64_t j) {
    for (uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; t < N / 2;
         t += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        bool asc = (i & k) == 0;
        uint64_t a = keys[i], b = keys[i + j];
        if ((a > b) == asc) {
            keys[i] = b;
            keys[i + j] = a;
        }
    }
}

inline cudaError_t bitonic_sort_u64(uint64_t* keys, uint64_t N, int num_sms, cudaStream_t st) {
    // N is a power of two >= kBitonicTile
    const unsigned nblk = static_cast<unsigned>(N / kBitonicTile);
    bitonic_shared_kernel<<<nblk, kBitonicThreads, 0, st>>>(keys, 2, kBitonicTile);
    for (uint64_t k = 2ull * kBitonicTile; k <= N; k <<= 1) {
        for (uint64_t j = k >> 1; j >= static_cast<uint64_t>(kBitonicTile); j >>= 1)
            bitonic_global_kernel<<<num_sms * 8, 512, 0, st>>>(keys, N, k, j);
        bitonic_shared_kernel<<<nblk, kBitonicThreads, 0, st>>>(keys, k, k);
    }
    return cudaGetLastError();
}

}  // namespace mhr
