// Ordering MLP: forward (tensor cores), backward and Adam kernels, feature
// gathering, and their C ABI.  The network orders intermediate vertices so
// the K-th-score threshold of a query tightens early; it never decides what is
// pruned (that is left to provable bounds), so it cannot change any result.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "mhr_internal.cuh"
#include "mhr_mlp.cuh"
#include "mhr_mlp_tc.cuh"

namespace mhr {

constexpr int kMlpParams = kMlpHid * kMlpIn + kMlpHid + kMlpHid + 1;  // W1, b1, w2, b2

// Dense forward on the tensor cores (tcgen05, accumulator in TMEM): one CTA
// per SM runs 128-row tiles of X; y, and z1 (pre-activations) when asked.
// With a tensor map (tmap_ok), each whole tile is staged by one TMA load: a
// 4-D view of X (8 columns, 8 rows, 32 column blocks, row groups) whose box
// {8, 8, 32, 16} lands in shared memory exactly in the K-major core-matrix
// layout the MMA descriptors describe; the ragged last tile, and every tile
// without a map, is staged by the threads.  A tile whose TMA or MMA does not
// complete within a second gets NaN outputs.
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_forward_tc(MlpDev m, const uint16_t* __restrict__ X,
                                                                  int64_t n, float* __restrict__ y,
                                                                  float* __restrict__ z1,
                                                                  const __grid_constant__ CUtensorMap tmap,
                                                                  int tmap_ok) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTcSmem<kMlpIn>& sm = *reinterpret_cast<MlpTcSmem<kMlpIn>*>(smem_raw);
    tc_setup(sm);
    tc_stage_w1(sm, m.W1);
    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    const int64_t tma_tiles = tmap_ok && (tc::smem_u32(sm.A) & 127u) == 0u ? (n / 8) / 16 : 0;  // whole tiles
    uint32_t phase = 0, tphase = 0;
    const uint4* Xv = reinterpret_cast<const uint4*>(X);
    const float b2 = __ldg(m.b2);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * kTcRows;
        bool staged = true;
        if (tile < tma_tiles) {
            __syncthreads();  // the set-up (barrier init) and the previous tile's reads are done
            if (threadIdx.x == 0) {
                tc::mbar_arrive_expect_tx(&sm.tma_bar, kTcRows * kMlpIn * 2);
                tc::tma_load_4d(sm.A, &tmap, 0, 0, 0, static_cast<int>(tile * (kTcRows / 8)), &sm.tma_bar);
            }
            staged = tc::mbar_wait(&sm.tma_bar, tphase, kTcWaitNs);
            tphase ^= 1u;
        } else {
            for (int i = threadIdx.x; i < kTcRows * (kMlpIn / 8); i += blockDim.x) {
                const int r = i >> 5, c = i & 31;
                const int64_t row = r0 + r;
                const uint4 v = row < n ? __ldg(Xv + row * (kMlpIn / 8) + c) : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(sm.A + tc::core_offset(r, c * 8, kMlpIn)) = v;
            }
        }
        if (__syncthreads_or(staged ? 0 : 1)) {
            const int64_t row = r0 + threadIdx.x;
            if (threadIdx.x < kTcRows && row < n) y[row] = __int_as_float(0x7fc00000);
            break;
        }
        const bool ok = tc_mma_tile(sm, phase);
        const int r = ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
        const int h = threadIdx.x >> 7;
        const int64_t row = r0 + r;
        if (!ok) {
            if (h == 0 && row < n) y[row] = __int_as_float(0x7fc00000);
            break;
        }
        float* zr = (z1 != nullptr && row < n) ? z1 + row * kMlpHid : nullptr;
        const float p = tc_row_half(
            sm.tmem, m.w2, [&](int c) { return __ldg(m.b1 + c); },
            [&](int c0, const float(&z)[32]) {
                if (zr) {
                    float4* d4 = reinterpret_cast<float4*>(zr + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d4[i] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
                }
            });
        sm.part[r][h] = p;
        __syncthreads();
        if (threadIdx.x < kTcRows && r0 + static_cast<int64_t>(threadIdx.x) < n)
            y[r0 + threadIdx.x] = (sm.part[threadIdx.x][0] + sm.part[threadIdx.x][1]) + b2;
    }
    tc_teardown(sm);
}

__global__ void k_mlp_features(DevGraph g, const uint32_t* __restrict__ va, const uint32_t* __restrict__ vb, int64_t n,
                               uint16_t* __restrict__ X) {
    uint32_t* Xw = reinterpret_cast<uint32_t*>(X);
    const int64_t total = n * (kMlpIn / 2);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total; i += stride) {
        const int64_t r = i / (kMlpIn / 2);
        const int k = static_cast<int>(i - r * (kMlpIn / 2)) * 2;
        Xw[i] = feature_pair(g, va[r], vb[r], k);
    }
}

// dZ[r][c] = (z[r][c] > 0) * dy[r] * w2[c],  dy[r] = 2 (y[r] - t[r]) / n
__global__ void k_mlp_bwd_rows(const float* __restrict__ w2, const float* __restrict__ y,
                               const float* __restrict__ tgt, const float* __restrict__ z1, int64_t n,
                               float* __restrict__ dz) {
    const int64_t total = n * kMlpHid;
    const float inv = 2.0f / static_cast<float>(n);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total; i += stride) {
        const int64_t r = i / kMlpHid;
        const int c = static_cast<int>(i - r * kMlpHid);
        const float dy = (y[r] - tgt[r]) * inv;
        dz[i] = z1[i] > 0.f ? dy * w2[c] : 0.f;
    }
}

// column sums in a fixed order: db1[c] = sum_r dZ[r][c], dw2[c] = sum_r
// relu(z[r][c]) dy[r]; block 0 also db2 = sum_r dy[r] and the loss
__global__ void __launch_bounds__(256) k_mlp_bwd_cols(const float* __restrict__ y, const float* __restrict__ tgt,
                                                      const float* __restrict__ z1, const float* __restrict__ dz,
                                                      int64_t n, float* __restrict__ grads,
                                                      float* __restrict__ loss) {
    __shared__ float s1[8][32], s2[8][32];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int grp = threadIdx.x >> 5;
    const float inv = 2.0f / static_cast<float>(n);
    float a = 0.f, b = 0.f;
    for (int64_t r = grp; r < n; r += 8) {
        const float dy = (y[r] - tgt[r]) * inv;
        a += dz[r * kMlpHid + c];
        b += fmaxf(z1[r * kMlpHid + c], 0.f) * dy;
    }
    s1[grp][threadIdx.x & 31] = a;
    s2[grp][threadIdx.x & 31] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        float sa = 0.f, sb = 0.f;
        for (int k = 0; k < 8; ++k) {
            sa += s1[k][threadIdx.x];
            sb += s2[k][threadIdx.x];
        }
        grads[kMlpHid * kMlpIn + c] = sa;            // db1
        grads[kMlpHid * kMlpIn + kMlpHid + c] = sb;  // dw2
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        // db2 and the loss, fixed order
        float d = 0.f, l = 0.f;
        for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
            const float e = y[r] - tgt[r];
            d += e * inv;
            l += e * e;
        }
        s1[threadIdx.x >> 5][threadIdx.x & 31] = d;
        s2[threadIdx.x >> 5][threadIdx.x & 31] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            float sd = 0.f, sl = 0.f;
            for (int k = 0; k < 256; ++k) {
                sd += s1[k >> 5][k & 31];
                sl += s2[k >> 5][k & 31];
            }
            grads[kMlpHid * kMlpIn + 2 * kMlpHid] = sd;  // db2
            if (loss) *loss = sl / static_cast<float>(n);
        }
    }
}

// dW1 = dZ^T X on the tensor cores (tcgen05).  CTA (bx, by) owns hidden units
// 128 by .. +127 and inputs 64 bx .. +63 (M = 128, N = 64, 64 TMEM columns) and
// runs over all rows in chunks of 64 (the contraction dimension): dZ^T is
// staged as bf16 hi + lo parts (dZ = hi + lo + r, |r| <= 2^-16 |dZ|; two MMAs
// per K step), X^T as bf16 (exact); both are transposed into K-major core
// matrices on the way into shared memory.  Each output element is summed by
// one CTA in a fixed order, so gradients are deterministic.  A chunk whose MMA
// does not complete within a second makes the CTA's gradients NaN.
constexpr int kDwRows = 64;  // rows of dZ / X per chunk
struct DwSmem {
    alignas(128) uint8_t Ahi[kTcRows * kDwRows * 2];
    alignas(128) uint8_t Alo[kTcRows * kDwRows * 2];
    alignas(128) uint8_t B[64 * kDwRows * 2];
    uint64_t bar;
    uint32_t tmem;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_dw1_tc(const float* __restrict__ dz, const uint16_t* __restrict__ X,
                                                              int64_t n, float* __restrict__ grads) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    DwSmem& sm = *reinterpret_cast<DwSmem*>(smem_raw);
    const int i0 = blockIdx.x * 64, o0 = blockIdx.y * kTcRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc::tmem_alloc(&sm.tmem, 64);
    if (threadIdx.x == 0) {
        tc::mbar_init(&sm.bar, 1);
        tc::mbar_fence_init();
    }
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t r0 = 0; r0 < n && ok; r0 += kDwRows) {
        // 128 core matrices of dZ^T (16 hidden blocks x 8 row blocks), 64 of X^T (8 x 8)
        for (int job = threadIdx.x; job < 192; job += blockDim.x) {
            if (job < 128) {
                const int og = job >> 3, rg = job & 7;
                float v[8][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t row = r0 + rg * 8 + j;
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                    if (row < n) {
                        const float4* src = reinterpret_cast<const float4*>(dz + row * kMlpHid + o0 + og * 8);
                        a = __ldg(src);
                        b = __ldg(src + 1);
                    }
                    v[j][0] = a.x; v[j][1] = a.y; v[j][2] = a.z; v[j][3] = a.w;
                    v[j][4] = b.x; v[j][5] = b.y; v[j][6] = b.z; v[j][7] = b.w;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float x0 = v[2 * m][k], x1 = v[2 * m + 1][k];
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                        hw[m] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) |
                                (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
                        lw[m] = pack_bf16x2(x0 - __bfloat162float(h0), x1 - __bfloat162float(h1));
                    }
                    const uint32_t off = tc::core_offset(og * 8 + k, rg * 8, kDwRows);
                    *reinterpret_cast<uint4*>(sm.Ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(sm.Alo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            } else {
                const int b = job - 128, ig = b >> 3, rg = b & 7;
                uint32_t w[8][4];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t row = r0 + rg * 8 + j;
                    uint4 t = make_uint4(0u, 0u, 0u, 0u);
                    if (row < n) t = __ldg(reinterpret_cast<const uint4*>(X + row * kMlpIn + i0 + ig * 8));
                    w[j][0] = t.x; w[j][1] = t.y; w[j][2] = t.z; w[j][3] = t.w;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const unsigned sel = (k & 1) ? 0x7632u : 0x5410u;  // high or low halves
                    uint32_t o[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) o[m] = __byte_perm(w[2 * m][k >> 1], w[2 * m + 1][k >> 1], sel);
                    *reinterpret_cast<uint4*>(sm.B + tc::core_offset(ig * 8 + k, rg * 8, kDwRows)) =
                        make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcRows, 64);
            constexpr uint32_t sbo = (kDwRows / 8) * 128;
            const uint32_t ah = tc::smem_u32(sm.Ahi), al = tc::smem_u32(sm.Alo), bb = tc::smem_u32(sm.B);
#pragma unroll
            for (int kk = 0; kk < kDwRows / 16; ++kk) {
                const uint64_t bd = tc::smem_desc(bb + kk * 256, 128, sbo);
                tc::mma_bf16(sm.tmem, tc::smem_desc(ah + kk * 256, 128, sbo), bd, idesc, (r0 > 0 || kk > 0) ? 1u : 0u);
                tc::mma_bf16(sm.tmem, tc::smem_desc(al + kk * 256, 128, sbo), bd, idesc, 1u);
            }
            tc::mma_commit(&sm.bar);
        }
        const bool done = tc::mbar_wait(&sm.bar, phase, kTcWaitNs);
        phase ^= 1u;
        tc::fence_after_sync();
        ok = !__syncthreads_or(done ? 0 : 1);
    }
    if (warp < 4) {
        const int o = o0 + warp * 32 + lane;
        float* dst = grads + static_cast<int64_t>(o) * kMlpIn + i0;
        for (int c0 = 0; c0 < 64; c0 += 32) {
            float v[32];
            tc::tmem_ld32(sm.tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) dst[c0 + i] = ok ? v[i] : __int_as_float(0x7fc00000);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sm.tmem, 64);
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const float g = gr[i];
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float b = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

__global__ void k_to_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst, int64_t n) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
        dst[i] = __bfloat16_as_ushort(__float2bfloat16_rn(src[i]));
}

// Tensor map of the feature matrix X [n x 256] bf16 viewed as 4-D: element
// (e, i, c, g) = X[8 g + i][8 c + e], strides 2 B (implicit), 512 B, 16 B,
// 4096 B; a box of {8, 8, 32, 16} is one 128-row tile in the K-major
// core-matrix layout.  Whole groups of 8 rows only (the kernel stages a
// ragged tail itself).  The driver's encoder is looked up once through the
// runtime; false (threads stage every tile) when it is missing, when X is
// not 16-byte aligned or when the encoder declines the view.
static bool encode_feature_map(const uint16_t* X, int64_t n, CUtensorMap* out) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    }
    const int64_t groups = n / 8;
    if (!enc || groups < 16 || (reinterpret_cast<uintptr_t>(X) & 15u)) return false;
    const cuuint64_t dims[4] = {8, 8, kMlpIn / 8, static_cast<cuuint64_t>(groups)};
    const cuuint64_t strides[3] = {kMlpIn * 2, 16, 8 * kMlpIn * 2};
    const cuuint32_t box[4] = {8, 8, kMlpIn / 8, kTcRows / 8};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static MlpDev to_dev(const mhr_mlp* m) {
    MlpDev d;
    d.W1 = m->W1;
    d.b1 = m->b1;
    d.w2 = m->w2;
    d.b2 = m->b2;
    return d;
}

static mhr_status check_mlp(const mhr_mlp* m) {
    if (!m || !m->W1 || !m->b1 || !m->w2 || !m->b2) return fail(MHR_EINVAL, "MLP weights are incomplete");
    return MHR_OK;
}

}  // namespace mhr

using namespace mhr;

extern "C" mhr_status mhr_mlp_features(const mhr_graph* g, const uint32_t* va, const uint32_t* vb, int64_t n,
                                       uint16_t* X, void* cuda_stream) {
    MHR_TRY(check_graph(g));
    if (n < 0 || (n && (!va || !vb || !X))) return fail(MHR_EINVAL, "bad feature arguments");
    if (!n) return MHR_OK;
    k_mlp_features<<<std::max(1, g->num_sms) * 4, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(g->dg, va, vb, n, X);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}

extern "C" mhr_status mhr_mlp_forward(const mhr_mlp* m, const uint16_t* X, int64_t n, float* y, float* z1,
                                      void* cuda_stream) {
    MHR_TRY(check_mlp(m));
    if (n < 0 || (n && (!X || !y))) return fail(MHR_EINVAL, "bad forward arguments");
    if (!n) return MHR_OK;
    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, std::max(1, device_sm_count())));
    const int sb = static_cast<int>(sizeof(MlpTcSmem<kMlpIn>));
    MHR_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sb));
    CUtensorMap tmap;
    const int tmap_ok = encode_feature_map(X, n, &tmap) ? 1 : 0;
    k_mlp_forward_tc<<<grid, kTcThreads, sb, static_cast<cudaStream_t>(cuda_stream)>>>(to_dev(m), X, n, y, z1, tmap,
                                                                                       tmap_ok);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}

extern "C" mhr_status mhr_mlp_backward(const mhr_mlp* m, const uint16_t* X, int64_t n, const float* target,
                                       const float* y, const float* z1, float* work, float* grads, float* loss,
                                       void* cuda_stream) {
    MHR_TRY(check_mlp(m));
    if (n < 1 || !X || !target || !y || !z1 || !work || !grads) return fail(MHR_EINVAL, "bad backward arguments");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int sms = std::max(1, device_sm_count());
    k_mlp_bwd_rows<<<sms * 4, 256, 0, st>>>(m->w2, y, target, z1, n, work);
    k_mlp_bwd_cols<<<kMlpHid / 32, 256, 0, st>>>(y, target, z1, work, n, grads, loss);
    MHR_CUDA_TRY(cudaFuncSetAttribute(k_mlp_dw1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(sizeof(DwSmem))));
    k_mlp_dw1_tc<<<dim3(kMlpIn / 64, kMlpHid / kTcRows), kTcThreads, sizeof(DwSmem), st>>>(work, X, n, grads);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}

extern "C" mhr_status mhr_mlp_adam(float* params, const float* grads, float* m1, float* m2, int64_t count, float lr,
                                   float beta1, float beta2, float eps, int32_t step, void* cuda_stream) {
    if (count < 0 || (count && (!params || !grads || !m1 || !m2)) || step < 1)
        return fail(MHR_EINVAL, "bad Adam arguments");
    if (!count) return MHR_OK;
    const float c1 = 1.f - powf(beta1, static_cast<float>(step));
    const float c2 = 1.f - powf(beta2, static_cast<float>(step));
    k_adam<<<std::max(1, device_sm_count()) * 4, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        params, grads, m1, m2, count, lr, beta1, beta2, eps, c1, c2);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}

extern "C" mhr_status mhr_mlp_to_bf16(const float* src, uint16_t* dst, int64_t count, void* cuda_stream) {
    if (count < 0 || (count && (!src || !dst))) return fail(MHR_EINVAL, "bad conversion arguments");
    if (!count) return MHR_OK;
    k_to_bf16<<<std::max(1, device_sm_count()) * 4, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(src, dst, count);
    MHR_CUDA_TRY(cudaGetLastError());
    return MHR_OK;
}
