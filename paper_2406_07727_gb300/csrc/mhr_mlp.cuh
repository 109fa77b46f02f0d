// Ordering MLP: y = w2 . relu(W1 x + b1) + b2, x = 256 bfloat16 features,
// 256 hidden units.  Shared definitions: the network's sizes and device view,
// the bf16 feature gather, and the warp-level bf16 mma used by the middle-edge
// screen of the search.  The first layer itself runs on tcgen05 (mhr_mlp_tc.cuh).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mhr_internal.cuh"

namespace mhr {

constexpr int kMlpIn = 256;
constexpr int kMlpHid = 256;

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

}  // namespace mhr
