// Ordering MLP first layer on the 5th-generation tensor cores (tcgen05).
//
// A CTA of 256 threads runs tiles of 128 rows: Z = X W1^T with X the tile's
// bf16 features (KC columns) and W1 the bf16 first-layer weights (256 hidden
// units x KC), one tcgen05.mma chain of KC / 16 instructions (M = 128,
// N = 256, K = 16 each) issued by one thread, the fp32 accumulator in 256
// TMEM columns.  The epilogue reads the accumulator back with tcgen05.ld
// (warp w: TMEM lanes 32 (w % 4).., hidden units 128 (w / 4)..), adds the
// bias, applies the ReLU and the dot product with w2; the two half-row
// partial sums meet in shared memory.  W1 is staged into shared memory once
// per CTA; each tile's rows are staged by the caller's loader.
#pragma once

#include "mhr_mlp.cuh"
#include "mhr_tcgen05.cuh"

namespace mhr {

constexpr int kTcRows = 128;                 // rows per tile (MMA M)
constexpr int kTcThreads = 256;              // 8 warps: two per TMEM lane quarter
constexpr uint32_t kTcCols = 256;            // TMEM columns (fp32 accumulator, N = 256)
constexpr uint64_t kTcWaitNs = 1000000000ull;  // give up on an MMA after 1 s

template <int KC>
struct MlpTcSmem {
    alignas(128) uint8_t B[kMlpHid * KC * 2];  // W1[:, 0:KC], K-major core-matrix layout
    alignas(128) uint8_t A[kTcRows * KC * 2];  // the tile's features, same layout
    float part[kTcRows][2];
    uint64_t bar;      // MMA completion
    uint64_t tma_bar;  // TMA tile loads (the dense forward)
    uint32_t tmem;
    int failed;
};

// W1[:, 0:KC] -> shared memory (16-byte chunks; W1 rows hold kMlpIn bf16 values)
template <int KC>
__device__ __forceinline__ void tc_stage_w1(MlpTcSmem<KC>& sm, const uint16_t* __restrict__ W1) {
    const uint4* W = reinterpret_cast<const uint4*>(W1);
    constexpr int chunks = KC / 8;
    for (int i = threadIdx.x; i < kMlpHid * chunks; i += blockDim.x) {
        const int n = i / chunks, c = i - n * chunks;
        *reinterpret_cast<uint4*>(sm.B + tc::core_offset(n, c * 8, KC)) = __ldg(W + n * (kMlpIn / 8) + c);
    }
}

// TMEM and the MMA barrier; every thread calls (warp 0 allocates)
template <int KC>
__device__ __forceinline__ void tc_setup(MlpTcSmem<KC>& sm) {
    if (threadIdx.x < 32) tc::tmem_alloc(&sm.tmem, kTcCols);
    if (threadIdx.x == 0) {
        tc::mbar_init(&sm.bar, 1);
        tc::mbar_init(&sm.tma_bar, 1);
        tc::mbar_fence_init();
        sm.failed = 0;
    }
}

// After the A (and B) stores of every thread: publish them to the tensor
// cores, issue the MMA chain from thread 0 and wait for it.  Returns false on
// every thread when the wait gave up.
template <int KC>
__device__ __forceinline__ bool tc_mma_tile(MlpTcSmem<KC>& sm, uint32_t& phase) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcRows, kMlpHid);
        const uint32_t a = tc::smem_u32(sm.A), b = tc::smem_u32(sm.B);
        constexpr uint32_t sbo = (KC / 8) * 128;  // next 8-row group
#pragma unroll
        for (int kk = 0; kk < KC / 16; ++kk)
            tc::mma_bf16(tmem, tc::smem_desc(a + kk * 256, 128, sbo), tc::smem_desc(b + kk * 256, 128, sbo), idesc,
                         kk > 0 ? 1u : 0u);
        tc::mma_commit(&sm.bar);
    }
    const bool ok = tc::mbar_wait(&sm.bar, phase, kTcWaitNs);
    phase ^= 1u;
    tc::fence_after_sync();
    return !__syncthreads_or(ok ? 0 : 1);
}

// Epilogue for this thread's row (r = 32 (warp % 4) + lane) and half of the
// hidden units; bias(c) acts on that row, store_z(c0, z) receives the row's
// pre-activations of hidden units c0 .. c0 + 31.  Returns the partial output
// sum; the caller adds the halves (part) and b2.
template <typename Bias, typename StoreZ>
__device__ __forceinline__ float tc_row_half(uint32_t tmem, const float* __restrict__ w2, Bias bias, StoreZ store_z) {
    const int warp = threadIdx.x >> 5;
    const int q = warp & 3, h = warp >> 2;
    float p = 0.f;
#pragma unroll 1
    for (int cc = 0; cc < 4; ++cc) {
        const int c0 = h * 128 + cc * 32;
        float v[32];
        tc::tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(c0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            v[i] += bias(c0 + i);
            p += fmaxf(v[i], 0.f) * __ldg(w2 + c0 + i);
        }
        store_z(c0, v);
    }
    return p;
}

template <int KC>
__device__ __forceinline__ void tc_teardown(MlpTcSmem<KC>& sm) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sm.tmem, kTcCols);
    }
}

}  // namespace mhr
