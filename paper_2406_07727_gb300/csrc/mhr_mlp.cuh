// Ordering MLP: y = w2 . relu(W1 x + b1) + b2, x = 256 bfloat16 features,
// 256 hidden units.  The first layer runs on the tensor cores (bf16 inputs,
// fp32 accumulation, mma m16n8k16); bias, ReLU and the output dot product are
// fused into the epilogue.  A tile of 32 rows x 256 hidden units per block of
// 8 warps: warp w owns rows (w & 1) * 16 .. +15 and hidden units
// (w >> 1) * 64 .. +63.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mhr_internal.cuh"

namespace mhr {

constexpr int kMlpIn = 256;
constexpr int kMlpHid = 256;
constexpr int kMlpRows = 32;     // rows per block tile
constexpr int kMlpThreads = 256;

struct MlpDev {
    const uint16_t* W1;  // bf16 [256 hidden x 256 in], row-major
    const float* b1;     // [256]
    const float* w2;     // [256]
    const float* b2;     // [1]
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// features of a row: [e_a[0:128]; e_b[0:128]] of two vertices, as bf16 pairs
// (columns k, k+1; k even); dimensions beyond d are zero
__device__ __forceinline__ uint32_t feature_pair(const DevGraph& g, uint32_t va, uint32_t vb, int k) {
    const uint32_t v = (k < 128) ? va : vb;
    const int j = k & 127;
    if (j >= g.d) return 0u;
    const bool two = j + 1 < g.d;
    const int64_t base = static_cast<int64_t>(v) * g.d + j;
    if (g.dtype == MHR_BF16) {
        const uint16_t* e = static_cast<const uint16_t*>(g.vemb);
        const uint32_t lo = e[base];
        const uint32_t hi = two ? e[base + 1] : 0u;
        return lo | (hi << 16);
    }
    const float* e = static_cast<const float*>(g.vemb);
    return pack_bf16x2(e[base], two ? e[base + 1] : 0.f);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One 32-row tile over the first KT*16 input columns.  a_pair(r, k) returns
// the bf16 pair of row r (0..31 within the tile), columns k, k+1; bias(r, c)
// the first-layer bias of hidden unit c for row r (b1[c], or b1[c] plus the
// product of the columns beyond KT*16 when the caller folded them in).
// Writes y for the tile's rows through store_y(r, y) and, if want_z, the
// pre-activations through store_z(r, c, z).  part: shared [32][4] floats.
// All 256 threads call.
template <int KT, typename APair, typename Bias, typename StoreY, typename StoreZ>
__device__ __forceinline__ void mlp_tile_k(const MlpDev& m, APair a_pair, Bias bias, StoreY store_y, StoreZ store_z,
                                           bool want_z, float (*part)[4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int r0 = (warp & 1) * 16;
    const int c0 = (warp >> 1) * 64;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    const uint32_t* W = reinterpret_cast<const uint32_t*>(m.W1);
#pragma unroll 2
    for (int kt = 0; kt < KT; ++kt) {
        const int k = kt * 16 + tq * 2;
        const uint32_t a0 = a_pair(r0 + gq, k), a1 = a_pair(r0 + gq + 8, k);
        const uint32_t a2 = a_pair(r0 + gq, k + 8), a3 = a_pair(r0 + gq + 8, k + 8);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n = c0 + nt * 8 + gq;
            const uint32_t b0 = __ldg(W + (n * kMlpIn + k) / 2);
            const uint32_t b1 = __ldg(W + (n * kMlpIn + k + 8) / 2);
            mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b1);
        }
    }
    // epilogue: bias, ReLU, dot with w2 (rows r0+gq and r0+gq+8)
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + nt * 8 + tq * 2 + h;
            const float ww = __ldg(m.w2 + c);
            const float z0 = acc[nt][h] + bias(r0 + gq, c), z1 = acc[nt][2 + h] + bias(r0 + gq + 8, c);
            if (want_z) {
                store_z(r0 + gq, c, z0);
                store_z(r0 + gq + 8, c, z1);
            }
            p0 += fmaxf(z0, 0.f) * ww;
            p1 += fmaxf(z1, 0.f) * ww;
        }
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    if (tq == 0) {
        part[r0 + gq][warp >> 1] = p0;
        part[r0 + gq + 8][warp >> 1] = p1;
    }
    __syncthreads();
    if (threadIdx.x < kMlpRows) {
        const float* pr = part[threadIdx.x];
        store_y(threadIdx.x, ((pr[0] + pr[1]) + (pr[2] + pr[3])) + __ldg(m.b2));
    }
    __syncthreads();
}

template <typename APair, typename StoreY, typename StoreZ>
__device__ __forceinline__ void mlp_tile(const MlpDev& m, APair a_pair, StoreY store_y, StoreZ store_z, bool want_z,
                                         float (*part)[4]) {
    mlp_tile_k<kMlpIn / 16>(m, a_pair, [&](int, int c) { return __ldg(m.b1 + c); }, store_y, store_z, want_z, part);
}

}  // namespace mhr
