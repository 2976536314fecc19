// train.cu -- learning the network heuristic on the GPU (the paper trains its heuristics
// from PDB values: Experimental Setup; Background, Heuristics) with BF16 tensor-core GEMMs,
// FP32 accumulation, an FP32 last layer and loss, and FP32 Adam on master weights.
//
// One step on a batch of B states (B padded to 128):
//   forward   layer 0..L-2: tcgen05 layers (one-hot A built from the packed states), ReLU,
//             activations A_l kept in BF16; last layer FP32: logits = A_{L-2} W_L^T + b_L
//   loss      cross-entropy over the classes (labels = class index) or MSE (one output);
//             dZ_L = dLoss/dlogits (mean over the batch)
//   backward  last layer, FP32-accurate on the tensor cores: dZ_L (FP32) as two BF16 parts and
//             W_L as three, every product exact and accumulated in FP32:
//             dW_L = dZ_L^T A_{L-2} (split-K over the batch), db_L = colsum(dZ_L),
//             dZ_{L-2} = (dZ_L W_L) * [A_{L-2} > 0] (BF16)
//             hidden l: dW_l = dZ_l^T A_{l-1} as a tcgen05 GEMM over the batch with both
//             operands MN-major as stored (A_{-1} is the one-hot, written transposed),
//             db_l = colsum(dZ_l), dZ_{l-1} = (dZ_l W_l) * [A_{l-1} > 0] as a tcgen05 GEMM
//             with the mask fused in the epilogue (W_l^T kept in BF16 beside W_l)
//   update    Adam (bias-corrected) on the FP32 masters of every tensor in one launch, adding
//             the gradient's split partials in order; BF16 copies W_l (K-padded, the
//             inference layout), W_l^T and the last layer's parts rewritten by the same kernel
// Every reduction has a fixed order, so a step is deterministic.
#include <algorithm>
#include <cerrno>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <thread>
#include <type_traits>

#include "chain.h"

namespace cbdfs {

uint64_t fnv1a64(const void *data, size_t n, uint64_t h);  // files.cpp
int tc_layer(bool first, int domain, bool fp8, bool out_fp8, int bn, const CUtensorMap &tmA,
             const CUtensorMap &tmB, const uint64_t *states, uint32_t n, uint32_t rows_pad, int K,
             int N, const float *bias, void *out, float acc_scale, float out_qscale, int *err,
             cudaStream_t st);
uint64_t npk(int n, int k);
// the forward pass through the fused chain, every hidden layer stored (api.cu)
int chain_forward_store(Ctx *c, Slot &s, const NetGPU &net, const uint64_t *d_states, uint32_t n,
                        void *const *outs, uint32_t out_rows, cudaStream_t st);

namespace {

using namespace dev;

constexpr int kThreads = 192;
constexpr int kSumRows = 64;   // rows of one chunk of a column sum
constexpr int kStageA = kBM * 128;

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle: 64-element (128-byte)
// rows along M (or N), one per k, eight k rows to a 1024-byte swizzle atom; `lbo` is the byte
// distance between 64-element blocks along M (N), the k atoms follow each other (1024 bytes).
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;  // leading byte offset: the next 64 along M (N)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: the next 8 k rows
    d |= (uint64_t)1 << 46;                     // descriptor version for sm_100 family
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}
constexpr int kMnBox = 64 * 128;  // one 64-element x 64-row TMA box of an MN-major operand

// ---------------------------------------------------------------------------------------
// TN GEMM on tcgen05: C[M][N] = A[M][K] B[N][K]^T, BF16, FP32 accumulate.
// Operands K-major ([M][K], [N][K]), or MN-major (MNA / MNB: stored [K][M], [K][N], as the
// backward has dZ and the activations, so dW = dZ^T A needs no transposes): an MN-major stage
// is loaded as 64 x 64 boxes, 8 KB apart along M (N).
// EPI 1: C FP32.  EPI 2: C BF16 = acc * (mask[m][n] > 0) (mask BF16 [M][N]).
// Split K (gridDim.z > 1, EPI 1): CTA z contracts k-blocks [z KB/S, (z+1) KB/S) into its own
// partial out + z M N; k_sum_splits then adds the partials in split order.
// ---------------------------------------------------------------------------------------
template <int BN, int EPI, bool MNA = false, bool MNB = false>
__global__ void __launch_bounds__(kThreads, 1)
k_gemm_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K, int N,
          void *__restrict__ out, const __nv_bfloat16 *__restrict__ mask, int stages, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int kStageB = BN * 128;
    const int kb0 = (int)((long long)(K / 64) * blockIdx.z / gridDim.z);
    const int KB = (int)((long long)(K / 64) * (blockIdx.z + 1) / gridDim.z) - kb0;
    if (EPI == 1) out = static_cast<float *>(out) + (size_t)blockIdx.z * gridDim.y * kBM * N;
    uint8_t *A = smem;
    uint8_t *B = smem + stages * kStageA;
    uint64_t *bars = reinterpret_cast<uint64_t *>(B + stages * kStageB);
    uint64_t *full = bars, *empty = bars + stages, *accum = bars + 2 * stages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accum), 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    uint32_t issued = 0;
    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % stages, u = kb / stages;
                if (kb >= stages && !mbar_wait(smem_u32(&empty[s]), (u - 1) & 1, err, DEVERR_STAGE_EMPTY)) break;
                mbar_arrive_expect_tx(smem_u32(&full[s]), kStageA + kStageB);
                const int k0 = (kb0 + kb) * 64;
                if (MNA) {
#pragma unroll
                    for (int h = 0; h < kBM / 64; ++h)
                        tma_load_2d(smem_u32(A + s * kStageA + h * kMnBox), &tmA, smem_u32(&full[s]), m0 + 64 * h, k0);
                } else {
                    tma_load_2d(smem_u32(A + s * kStageA), &tmA, smem_u32(&full[s]), k0, m0);
                }
                if (MNB) {
#pragma unroll
                    for (int h = 0; h < BN / 64; ++h)
                        tma_load_2d(smem_u32(B + s * kStageB + h * kMnBox), &tmB, smem_u32(&full[s]), n0 + 64 * h, k0);
                } else {
                    tma_load_2d(smem_u32(B + s * kStageB), &tmB, smem_u32(&full[s]), k0, n0);
                }
                ++issued;
            }
            // bounded drain of this thread's loads before the CTA can exit
            for (uint32_t j = issued > (uint32_t)stages ? issued - stages : 0; j < issued; ++j)
                mbar_wait_drain(smem_u32(&full[j % stages]), (j / stages) & 1, err, DEVERR_TMA_FULL, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // bits 15 / 16 of the instruction descriptor: A / B MN-major
            constexpr uint32_t idesc = make_idesc(kBM, BN, 1, 1) | (MNA ? 1u << 15 : 0u) | (MNB ? 1u << 16 : 0u);
            bool ok = true;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % stages, u = kb / stages;
                if (!mbar_wait(smem_u32(&full[s]), u & 1, err, DEVERR_TMA_FULL)) { ok = false; break; }
                tc_fence_after();
                // a 16-deep MMA step advances 32 bytes along a K-major row, or two 8-row k atoms
                // (2048 bytes) of an MN-major stage
                const uint64_t ad = MNA ? sw128_mn_desc(smem_u32(A + s * kStageA), kMnBox) : sw128_desc(smem_u32(A + s * kStageA));
                const uint64_t bd = MNB ? sw128_mn_desc(smem_u32(B + s * kStageB), kMnBox) : sw128_desc(smem_u32(B + s * kStageB));
                constexpr uint64_t da = MNA ? 2048 >> 4 : 2, db = MNB ? 2048 >> 4 : 2;
#pragma unroll
                for (int k = 0; k < 4; ++k) umma_bf16(tmem_d, ad + da * k, bd + db * k, idesc, (kb | k) != 0);
                umma_commit(smem_u32(&empty[s]));
            }
            umma_commit(smem_u32(accum));
            if (!ok) atomicCAS(err, 0, DEVERR_TMA_FULL);
        }
    } else {
        const int q = warp & 3;
        const uint32_t m = m0 + q * 32 + lane;
        const bool good = mbar_wait(smem_u32(accum), 0, err, DEVERR_ACCUM);
        tc_fence_after();
#pragma unroll 1
        for (int c = 0; c < BN / 32 && good; ++c) {
            uint32_t r[32];
            tmem_ld32(tmem_d + ((uint32_t)(q * 32) << 16) + c * 32, r);
            tmem_ld_wait();
            const size_t base = (size_t)m * N + n0 + c * 32;
            if (EPI == 1) {
                float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(out) + base);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                         __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            } else {
                const uint4 *mk = reinterpret_cast<const uint4 *>(mask + base);
                uint32_t pk[16];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint4 mm = __ldg(mk + j);
                    const __nv_bfloat162 *mh = reinterpret_cast<const __nv_bfloat162 *>(&mm);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float2 a = __bfloat1622float2(mh[t]);
                        const int e = 8 * j + 2 * t;
                        const float v0 = a.x > 0.f ? __uint_as_float(r[e]) : 0.f;
                        const float v1 = a.y > 0.f ? __uint_as_float(r[e + 1]) : 0.f;
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                        pk[4 * j + t] = *reinterpret_cast<uint32_t *>(&h2);
                    }
                }
                uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out) + base);
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_d, BN);
    }
}

__global__ void k_sum_splits(const float *__restrict__ part, int S, int len, float *__restrict__ out);

// splits > 1 (EPI 1 only): the partials go to `part` (splits x M x N floats), then (sum) their
// sum in split order to `out`
template <int BN, int EPI, bool MNA = false, bool MNB = false>
int gemm_tn(const CUtensorMap &tmA, const CUtensorMap &tmB, int M, int N, int K, void *out,
            const __nv_bfloat16 *mask, int *err, cudaStream_t st, int splits = 1, float *part = nullptr,
            bool sum = true) {
    constexpr int kStageB = BN * 128;
    const int stages = 4;
    const size_t smem = 1024 + 256 + (size_t)stages * (kStageA + kStageB);
    auto kern = k_gemm_tn<BN, EPI, MNA, MNB>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const bool split = EPI == 1 && splits > 1 && part;
    kern<<<dim3(N / BN, M / kBM, split ? splits : 1), kThreads, smem, st>>>(tmA, tmB, K, N, split ? part : out,
                                                                           mask, stages, err);
    CUDA_TRY(cudaGetLastError());
    if (split && sum) {
        const int len = M * N;
        k_sum_splits<<<(len + 255) / 256, 256, 0, st>>>(part, splits, len, static_cast<float *>(out));
        CUDA_TRY(cudaGetLastError());
    }
    return CBDFS_OK;
}

// ---------------------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------------------

// BF16 transpose: in [R][C] (row stride ldi) -> out [C][R] (row stride ldo; and out2 when
// given), R and C multiples of 64, 64 x 64 tiles through shared memory moved as 16-byte
// vectors: eight threads read one 128-byte tile row and eight write one 128-byte output row.
// The tile rows are 66 elements (33 words) apart, so the eight rows a column read gathers fall
// on distinct banks.  colsum (optional): the column sums of the tile's 64 rows, in row order,
// at colsum[tile row][C].  Block (32, 8).
constexpr int kTrPitch = 66;
__global__ void __launch_bounds__(256) k_transpose(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out,
                                                   int R, int C, int ldi, int ldo,
                                                   __nv_bfloat16 *__restrict__ out2, float *__restrict__ colsum) {
    __shared__ __align__(16) __nv_bfloat16 t[64 * kTrPitch];
    const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int v = tid & 7;  // the 16-byte vector of a 64-element row
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int r = (tid >> 3) + 32 * p;
        const uint4 x = *reinterpret_cast<const uint4 *>(in + (size_t)(r0 + r) * ldi + c0 + 8 * v);
        uint32_t *row = reinterpret_cast<uint32_t *>(t + r * kTrPitch + 8 * v);  // 4-byte aligned
        row[0] = x.x;
        row[1] = x.y;
        row[2] = x.z;
        row[3] = x.w;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int c = (tid >> 3) + 32 * p;  // input column = output row
        const unsigned short *ts = reinterpret_cast<const unsigned short *>(t);
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            w[i] = (uint32_t)ts[(8 * v + 2 * i) * kTrPitch + c] | ((uint32_t)ts[(8 * v + 2 * i + 1) * kTrPitch + c] << 16);
        const uint4 y = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(out + (size_t)(c0 + c) * ldo + r0 + 8 * v) = y;
        if (out2) *reinterpret_cast<uint4 *>(out2 + (size_t)(c0 + c) * ldo + r0 + 8 * v) = y;
    }
    // the tile's column sums over its 64 rows, in row order: the row-chunk partials of the
    // bias gradient (chunk r0 / 64)
    static_assert(kSumRows == 64, "a bias-gradient chunk is one transpose tile");
    if (colsum && tid < 64) {
        float sum = 0.f;
        for (int i = 0; i < 64; ++i) sum += __bfloat162float(t[i * kTrPitch + tid]);
        colsum[(size_t)blockIdx.y * C + c0 + tid] = sum;
    }
}

// transposed one-hot X^T [K1pad][Bp] (BF16) of the packed states; rows >= n are zero
template <int DOMAIN>
__global__ void k_onehot_t(const uint64_t *__restrict__ states, uint32_t n, int Bp, __nv_bfloat16 *__restrict__ xt) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (uint32_t)Bp) return;
    if (m >= n) return;  // the buffer was zeroed
    const __nv_bfloat16 one = __float2bfloat16(1.f);
    if (DOMAIN == CBDFS_DOM_RC3) {
        const uint64_t w0 = states[2 * m], w1 = states[2 * m + 1];
        for (int c = 0; c < 8; ++c) xt[(size_t)(c * 24 + ((w0 >> (5 * c)) & 31u)) * Bp + m] = one;
        for (int e = 0; e < 12; ++e) xt[(size_t)(192 + e * 24 + ((w1 >> (5 * e)) & 31u)) * Bp + m] = one;
    } else {
        constexpr int N = DOMAIN == CBDFS_DOM_STP3 ? 9 : 16;
        const uint64_t s = states[m];
        for (int p = 0; p < N; ++p) xt[(size_t)(((s >> (4 * p)) & 15u) * N + p) * Bp + m] = one;
    }
}


// loss and dZ = dLoss/dlogits (mean over n rows).  loss 0: softmax cross-entropy against
// the class index; loss 1: 0.5 (y - label)^2 on one output.  Per-row losses to row_loss.
constexpr int kExtParts = 5;
// BF16 parts of x: x ~ p[0] + p[1] + p[2], each the round-to-nearest-even of what is left
__device__ __forceinline__ void bf16_parts3(float r, __nv_bfloat16 (&p)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p[i] = __float2bfloat16_rn(r);
        r -= __bfloat162float(p[i]);
    }
}
// w_ext[k][s cs + c] for the last layer's weight w = W[c][k] (sections W1 W2 W3 W1 W2)
__device__ __forceinline__ void ext_store_w(float w, int c, int k, int cs, __nv_bfloat16 *__restrict__ w_ext) {
    __nv_bfloat16 p[3];
    bf16_parts3(w, p);
    __nv_bfloat16 *row = w_ext + (size_t)k * kExtParts * cs + c;
    row[0] = p[0];
    row[cs] = p[1];
    row[2 * cs] = p[2];
    row[3 * cs] = p[0];
    row[4 * cs] = p[1];
}
// dz_ext[m][s cs + c] for the loss gradient d = dZ[m][c] (sections D1 D1 D1 D2 D2)
__device__ __forceinline__ void ext_store_dz(float d, int c, __nv_bfloat16 *__restrict__ row, int cs) {
    const __nv_bfloat16 d1 = __float2bfloat16_rn(d);
    const __nv_bfloat16 d2 = __float2bfloat16_rn(d - __bfloat162float(d1));
    row[c] = d1;
    row[cs + c] = d1;
    row[2 * cs + c] = d1;
    row[3 * cs + c] = d2;
    row[4 * cs + c] = d2;
}
__global__ void k_write_ext(const float *__restrict__ w, int C, int K, int cs, __nv_bfloat16 *__restrict__ w_ext) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C * K) ext_store_w(w[i], i / K, i % K, cs, w_ext);
}

__global__ void k_loss(const float *__restrict__ logits, const uint8_t *__restrict__ labels, int n, int Bp,
                       int C, int loss, float *__restrict__ dz, float *__restrict__ row_loss,
                       __nv_bfloat16 *__restrict__ dz_ext, int cs) {
    // one warp per row: coalesced reads of the row's logits, butterfly reductions (every lane
    // ends with the same maximum and sum, in a fixed order).  Rows n..Bp-1 of dz_ext are zeroed.
    const int m = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (m >= Bp) return;  // warp-uniform
    __nv_bfloat16 *e = dz_ext + (size_t)m * kExtParts * cs;
    if (m >= n) {
        for (int c = lane; c < C; c += 32) ext_store_dz(0.f, c, e, cs);
        return;
    }
    const float *z = logits + (size_t)m * C;
    float *d = dz + (size_t)m * C;
    const float inv_n = 1.f / (float)n;
    if (loss == 1) {
        if (lane == 0) {
            const float r = z[0] - (float)labels[m];
            row_loss[m] = 0.5f * r * r;
            d[0] = r * inv_n;
            ext_store_dz(r * inv_n, 0, e, cs);
        }
        return;
    }
    float mx = -INFINITY;
    for (int c = lane; c < C; c += 32) mx = fmaxf(mx, z[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    float sum = 0.f;
    for (int c = lane; c < C; c += 32) sum += expf(z[c] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    const int y = labels[m];
    if (lane == 0) row_loss[m] = logf(sum) + mx - z[y];
    for (int c = lane; c < C; c += 32) {
        const float p = expf(z[c] - mx) / sum;
        const float g = (p - (c == y ? 1.f : 0.f)) * inv_n;
        d[c] = g;
        ext_store_dz(g, c, e, cs);
    }
}

// ---- FP32 GEMM on the CUDA cores (the logits of a network without split last-layer weights) --
// out[m][n] = sum over k of A(m,k) B(k,n) + bias[n], FP32: A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  64x64 tiles, k-steps of 16, 256 threads each owning a 4x4 block.
// AK: A is contiguous along k (else along m); BNC: B is contiguous along n (else along k).
constexpr int FG_T = 64, FG_BK = 16;
__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename TA, typename TB, bool AK, bool BNC>
__global__ void __launch_bounds__(256)
k_fgemm(const TA *__restrict__ A, long sam, long sak, const TB *__restrict__ B, long sbk, long sbn, int M,
        int N, int K, float *__restrict__ out, const float *__restrict__ bias) {
    __shared__ __align__(16) float As[FG_BK][FG_T];
    __shared__ __align__(16) float Bs[FG_BK][FG_T];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int m0 = blockIdx.y * FG_T, n0 = blockIdx.x * FG_T;
    const int kb = 0, ke = K;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += FG_BK) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            // A: 64 (m) x 16 (k), 4 values per thread along the contiguous index
            const int am = AK ? (tid >> 2) : ((tid & 15) * 4 + j), ak = AK ? ((tid & 3) * 4 + j) : (tid >> 4);
            const int gm = m0 + am, gk = k0 + ak;
            As[ak][am] = (gm < M && gk < ke) ? tof(A[(size_t)gm * sam + (size_t)gk * sak]) : 0.f;
            // B: 16 (k) x 64 (n)
            const int bn = BNC ? ((tid & 15) * 4 + j) : (tid >> 2), bk = BNC ? (tid >> 4) : ((tid & 3) * 4 + j);
            const int gn = n0 + bn, gk2 = k0 + bk;
            Bs[bk][bn] = (gn < N && gk2 < ke) ? tof(B[(size_t)gk2 * sbk + (size_t)gn * sbn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < FG_BK; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m >= M || n >= N) continue;
            out[(size_t)m * N + n] = acc[i][j] + bias[n];
        }
}

// the last layer's FP32 weights w[C][K] as three BF16 parts out[part][cpad][K] (W = W1 + W2 + W3,
// each part the round-to-nearest-even BF16 of what the previous parts leave), for the
// tensor-core head
__device__ __forceinline__ void split3_store(float r, int c, int k, int K, int cpad, __nv_bfloat16 *__restrict__ out) {
#pragma unroll
    for (int part = 0; part < 3; ++part) {
        const __nv_bfloat16 b = __float2bfloat16_rn(r);
        out[((size_t)part * cpad + c) * K + k] = b;
        r -= __bfloat162float(b);
    }
}

// out[i] = sum over z of part[z][i] (+ bias), in split order
__global__ void k_sum_splits(const float *__restrict__ part, int S, int len, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(size_t)z * len + i];
    out[i] = s;
}

// column sums by row chunks: part[r][j] = sum of X[m][j] over m in chunk r (fixed order);
// k_sum_splits then adds the chunks in order
template <typename T>
__global__ void k_colsum_part(const T *__restrict__ X, int n, int J, int chunk, float *__restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (j >= J) return;
    const int mb = r * chunk, me = min(n, mb + chunk);
    float s = 0.f;
    for (int m = mb; m < me; ++m) s += tof(X[(size_t)m * J + j]);
    part[(size_t)r * J + j] = s;
}
// the same for BF16 with J even: a thread sums a column pair (one 4-byte load per row), rows
// in the same order, so every column's sum is the scalar kernel's
__global__ void k_colsum_part2(const __nv_bfloat16 *__restrict__ X, int n, int J, int chunk, float *__restrict__ part) {
    const int j = 2 * (blockIdx.x * blockDim.x + threadIdx.x), r = blockIdx.y;
    if (j >= J) return;
    const int mb = r * chunk, me = min(n, mb + chunk);
    float s0 = 0.f, s1 = 0.f;
    if (me - mb == 64) {
        // a full chunk: all 64 rows' loads in flight, then the sums in row order
        uint32_t w[64];
#pragma unroll
        for (int q = 0; q < 64; ++q) w[q] = __ldg(reinterpret_cast<const unsigned int *>(X + (size_t)(mb + q) * J + j));
#pragma unroll
        for (int q = 0; q < 64; ++q) {
            const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[q]));
            s0 += v.x;
            s1 += v.y;
        }
    } else {
        for (int m = mb; m < me; ++m) {
            const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(X + (size_t)m * J + j));
            s0 += v.x;
            s1 += v.y;
        }
    }
    part[(size_t)r * J + j] = s0;
    part[(size_t)r * J + j + 1] = s1;
}

// sum of per-row losses (one block, fixed order), divided by n; ctr (a training run): the
// step and batch counters advance here, after this step's gather has read the batch counter
// and before its Adam reads the step counter (which then holds the step's number + 1)
__global__ void k_mean(const float *__restrict__ v, int n, float *__restrict__ out, int *ctr) {
    __shared__ float part[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += v[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < 256; ++i) t += part[i];
        *out = t / (float)n;
        if (ctr) {
            ctr[0]++;
            ctr[1]++;
        }
    }
}

// Adam on the FP32 masters of every tensor in one launch: segment s (a layer's weights [O][I]
// or biases [O]) owns blocks [block0, next block0).  Besides the master it writes the copies
// the other kernels read: the BF16 inference weights w_lp[o][Kp], their transpose wt[i][O] for
// the backward GEMM, an FP32 inference copy (the last layer, the biases) and the last layer's
// three BF16 parts for the tensor-core head.
struct AdamSeg {
    float *w;
    const float *g;  // parts x [O][I]: the gradient is the sum of the parts in order
    float *m, *v;
    int O, I, block0, Kp, cpad, parts, cs;
    size_t pstride;  // floats from one gradient part to the next
    __nv_bfloat16 *w_lp, *wt, *split, *w_ext;
    float *w_out;
};
struct AdamParams {
    AdamSeg seg[2 * kMaxLayers];
    int nseg;
    int copies_only;  // no update: only the copies of the masters as they are (a loaded checkpoint)
    float lr, b1, b2, eps, c1, c2;
    // optional: c1, c2 of step ctr[0] - 1 of a run from a table [2 x steps] (one captured step
    // serves every step of the run; k_mean has advanced the counter)
    const float *c12;
    const int *ctr;
};



__global__ void __launch_bounds__(256) k_adam_all(const __grid_constant__ AdamParams P) {
    int s = 0;
    while (s + 1 < P.nseg && (int)blockIdx.x >= P.seg[s + 1].block0) ++s;
    const AdamSeg &S = P.seg[s];
    const int idx = ((int)blockIdx.x - S.block0) * blockDim.x + threadIdx.x;
    if (idx >= S.O * S.I) return;
    float nw = S.w[idx];
    if (!P.copies_only) {
        float c1 = P.c1, c2 = P.c2;
        if (P.c12) {
            c1 = P.c12[2 * (P.ctr[0] - 1)];
            c2 = P.c12[2 * (P.ctr[0] - 1) + 1];
        }
        // the split partials added in split order; loaded four at a time, so that the loads are
        // in flight together instead of one after another
        float gg = 0.f;
        int z = 0;
        for (; z + 4 <= S.parts; z += 4) {
            const float g0 = __ldg(S.g + (size_t)z * S.pstride + idx), g1 = __ldg(S.g + (size_t)(z + 1) * S.pstride + idx);
            const float g2 = __ldg(S.g + (size_t)(z + 2) * S.pstride + idx), g3 = __ldg(S.g + (size_t)(z + 3) * S.pstride + idx);
            gg += g0;
            gg += g1;
            gg += g2;
            gg += g3;
        }
        for (; z < S.parts; ++z) gg += __ldg(S.g + (size_t)z * S.pstride + idx);
        const float m = P.b1 * S.m[idx] + (1.f - P.b1) * gg;
        const float v = P.b2 * S.v[idx] + (1.f - P.b2) * gg * gg;
        S.m[idx] = m;
        S.v[idx] = v;
        const float mh = m / c1, vh = v / c2;
        nw = S.w[idx] - P.lr * mh / (sqrtf(vh) + P.eps);
        S.w[idx] = nw;
    }
    const int o = idx / S.I, i = idx % S.I;
    if (S.w_lp) S.w_lp[(size_t)o * S.Kp + i] = __float2bfloat16(nw);
    if (S.wt) S.wt[(size_t)i * S.O + o] = __float2bfloat16(nw);
    if (S.w_out) S.w_out[idx] = nw;
    if (S.split) split3_store(nw, o, i, S.I, S.cpad, S.split);
    if (S.w_ext) ext_store_w(nw, o, i, S.cs, S.w_ext);
}

// wt[i][O] = BF16(w[o][i])
__global__ void k_write_t(const float *__restrict__ w, int O, int I, __nv_bfloat16 *__restrict__ wt) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= O * I) return;
    wt[(size_t)(idx % I) * O + idx / I] = __float2bfloat16(w[idx]);
}

// batch rows i < n from the epoch's permutation, starting at row ctr[1] * batch of it (the
// counter is the batch's index in the epoch, advanced on the device after each step, so that
// one captured step serves every full batch)
__global__ void k_gather(const uint64_t *__restrict__ src, const uint8_t *__restrict__ lab, const uint32_t *__restrict__ idx,
                         const int *__restrict__ ctr, uint32_t batch, int words, uint32_t n,
                         uint64_t *__restrict__ dst, uint8_t *__restrict__ dlab) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = idx[(size_t)ctr[1] * batch + i];
    for (int w = 0; w < words; ++w) dst[(size_t)i * words + w] = src[(size_t)j * words + w];
    dlab[i] = lab[j];
}

// Random walks of the blank from the goal (label generation): walk i draws from the
// splitmix64 stream seeded with seed_for(tag, i) = mix((tag << 32) | i); first its length
// 1 + (draw mod max_len), then each move uniformly (draw mod #choices) among the legal
// directions (up, left, right, down order) other than the reverse of the previous one.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <int SIDE>
__global__ void k_walks(uint32_t tag, uint64_t first, uint32_t n, int max_len, uint64_t *__restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t idx = first + i;
    uint64_t st = mix64(((uint64_t)tag << 32) | (idx & 0xFFFFFFFFull));
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        return mix64(st);
    };
    uint64_t s = 0;
    for (int t = 0; t < SIDE * SIDE; ++t) s |= (uint64_t)t << (4 * t);
    int r = 0, c = 0, prev = -1;
    const int len = 1 + (int)(next() % (uint64_t)max_len);
    for (int k = 0; k < len; ++k) {
        int cand[4], nc = 0;
        const int dr[4] = {-1, 0, 0, 1}, dcl[4] = {0, -1, 1, 0};
        for (int d = 0; d < 4; ++d) {
            if (prev >= 0 && d == 3 - prev) continue;
            const int nr = r + dr[d], ncl = c + dcl[d];
            if (nr >= 0 && nr < SIDE && ncl >= 0 && ncl < SIDE) cand[nc++] = d;
        }
        const int d = cand[next() % (uint64_t)nc];
        const int b = r * SIDE + c, nr = r + dr[d], ncl = c + dcl[d], q = nr * SIDE + ncl;
        const uint64_t tile = (s >> (4 * q)) & 15u;
        s = (s & ~((uint64_t)15 << (4 * q))) | (tile << (4 * b));
        r = nr;
        c = ncl;
        prev = d;
    }
    out[i] = s;
}

}  // namespace

// =========================================================================================
// host side
// =========================================================================================

struct TrainState {
    int L = 0, B = 0, Bp = 0;
    int dims[kMaxLayers + 1] = {};
    float *w[kMaxLayers] = {}, *b[kMaxLayers] = {};        // FP32 masters
    float *mw[kMaxLayers] = {}, *vw[kMaxLayers] = {}, *mb[kMaxLayers] = {}, *vb[kMaxLayers] = {};
    float *gw[kMaxLayers] = {}, *gb[kMaxLayers] = {};      // gradients
    __nv_bfloat16 *wt[kMaxLayers] = {};                    // W_l^T BF16 (hidden layers >= 1)
    __nv_bfloat16 *act[kMaxLayers] = {};                   // A_l, l = 0..L-2, [Bp][dims[l+1]]
    __nv_bfloat16 *dz[kMaxLayers] = {};                    // dZ_l BF16 [Bp][dims[l+1]]
    __nv_bfloat16 *t_a = nullptr;                          // the transposed one-hot of the batch
    float *logits = nullptr, *dzl = nullptr, *row_loss = nullptr, *loss = nullptr;
    // partial sums of every gradient tensor: the weights' row (split-K) partials and the
    // biases' row-chunk partials, [parts][len] each; the gradient is their sum in part order
    float *gw_buf[kMaxLayers] = {}, *gb_buf[kMaxLayers] = {};
    size_t gw_buf_floats[kMaxLayers] = {}, gb_buf_floats[kMaxLayers] = {};
    // where the last backward left each gradient: `parts` partials at gw_src (1: the sum itself)
    const float *gw_src[kMaxLayers] = {}, *gb_src[kMaxLayers] = {};
    int gw_parts[kMaxLayers] = {}, gb_parts[kMaxLayers] = {};
    size_t gw_pstride[kMaxLayers] = {};  // floats from one weight-gradient part to the next
    // the last layer's dX on the tensor cores: dZ_L (FP32) as BF16 parts D1 + D2 and W_L as
    // W1 + W2 + W3, stacked along K in kExtParts sections of `cs` columns (C padded to 64):
    // dz_ext[m] = [D1 D1 D1 D2 D2], w_ext[k] = [W1 W2 W3 W1 W2] (columns c of each section), so
    // one K = 5 cs GEMM adds D1 W1 + D1 W2 + D1 W3 + D2 W1 + D2 W2
    __nv_bfloat16 *dz_ext = nullptr, *w_ext = nullptr;
    int cs = 0;
    // the last layer's dW = dZ^T A on the tensor cores: K-major operands over 2 Bp batch
    // columns, t_dz_ext = [D1^T | D2^T] ([Mp][2 Bp], rows >= C zero) and t_a_ext = [A^T | A^T]
    // ([KL][2 Bp]); the product rows are Mp = C rounded up to the 128-row tile
    __nv_bfloat16 *t_dz_ext = nullptr, *t_a_ext = nullptr;
    int Mp = 0;
    uint64_t *states = nullptr;
    uint8_t *labels = nullptr;
    int64_t step = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    std::map<long long, CUtensorMap> maps;
};

// Row splits of a hidden layer's dW = dZ^T A (O x I outputs, Bp rows contracted): enough
// that the output tiles times the splits come near the SM count, at most one k-block each.
static int dw_splits(const Ctx *c, int O, int I, int Bp) {
    const int tiles = (I / (I % 256 == 0 ? 256 : 128)) * (O / kBM);
    return std::max(1, std::min(Bp / 64, c->num_sms / std::max(tiles, 1)));
}

static int talloc(Ctx *c, TrainState &T, void **p, size_t bytes) {
    int rc = dev_alloc(c, p, bytes);
    if (rc) return rc;
    T.allocs.emplace_back(*p, bytes);
    return cudaMemset(*p, 0, bytes) == cudaSuccess ? CBDFS_OK : fail(CBDFS_EDEVICE, "memset");
}

static const CUtensorMap *bmap(TrainState &T, const void *base, int inner, int outer, int box_outer) {
    long long key = (long long)(uintptr_t)base;
    key = key * 1000003LL + inner;
    key = key * 1000003LL + outer;
    key = key * 1000003LL + box_outer;
    auto it = T.maps.find(key);
    if (it != T.maps.end()) return &it->second;
    CUtensorMap m;
    if (make_tmap_2d(&m, const_cast<void *>(base), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)inner,
                     (uint64_t)outer, 64, box_outer))
        return nullptr;
    return &T.maps.emplace(key, m).first->second;
}

void train_free(Ctx *c, TrainState *T) {
    if (!T) return;
    for (auto &a : T->allocs) dev_free(c, a.first, a.second);
    delete T;
}

// set up (or resize) the training state of a BF16 network for batches of up to B states
static int train_setup(Ctx *c, NetGPU &net, int B, const float *const *host_w, const float *const *host_b) {
    if (net.prec != CBDFS_PREC_BF16) return fail(CBDFS_EINVAL, "training needs a BF16 network");
    if (!net.train || net.train->B < B) {
        if (!net.train && (!host_w || !host_b)) return fail(CBDFS_EINVAL, "no master weights to train from");
        TrainState *old = net.train;
        TrainState *T = new TrainState();
        T->L = net.L;
        for (int l = 0; l <= net.L; ++l) T->dims[l] = net.dims[l];
        T->B = B;
        T->Bp = (B + kBM - 1) / kBM * kBM;
        const int L = net.L, Bp = T->Bp;
        int rc = CBDFS_OK;
        const size_t k1 = (size_t)net.k1pad;
        for (int l = 0; l < L && !rc; ++l) {
            const size_t O = net.dims[l + 1], I = l == 0 ? k1 : (size_t)net.dims[l];
            rc = talloc(c, *T, (void **)&T->w[l], O * I * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->b[l], O * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->mw[l], O * I * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->vw[l], O * I * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->mb[l], O * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->vb[l], O * 4);
            // the last layer's gradient has C rounded up to 128 rows (its GEMM's row tile)
            if (!rc) rc = talloc(c, *T, (void **)&T->gw[l], (l == L - 1 ? (O + 127) / 128 * 128 : O) * I * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->gb[l], O * 4);
            if (!rc && l >= 1 && l < L - 1) rc = talloc(c, *T, (void **)&T->wt[l], O * I * 2);
            if (!rc && l < L - 1) rc = talloc(c, *T, (void **)&T->act[l], (size_t)Bp * O * 2);
            if (!rc && l < L - 1) rc = talloc(c, *T, (void **)&T->dz[l], (size_t)Bp * O * 2);
        }
        if (!rc) rc = talloc(c, *T, (void **)&T->t_a, (size_t)Bp * k1 * 2);
        const int C = net.dims[L];
        if (!rc) rc = talloc(c, *T, (void **)&T->logits, (size_t)Bp * C * 4);
        if (!rc) rc = talloc(c, *T, (void **)&T->dzl, (size_t)Bp * C * 4);
        if (!rc) rc = talloc(c, *T, (void **)&T->row_loss, (size_t)Bp * 4);
        T->cs = (C + 63) / 64 * 64;
        if (!rc) rc = talloc(c, *T, (void **)&T->dz_ext, (size_t)Bp * kExtParts * T->cs * 2);
        if (!rc) rc = talloc(c, *T, (void **)&T->w_ext, (size_t)net.dims[L - 1] * kExtParts * T->cs * 2);
        T->Mp = (C + 127) / 128 * 128;
        if (!rc) rc = talloc(c, *T, (void **)&T->t_dz_ext, (size_t)T->Mp * 2 * Bp * 2);
        if (!rc) rc = talloc(c, *T, (void **)&T->t_a_ext, (size_t)net.dims[L - 1] * 2 * Bp * 2);
        // partials of every gradient tensor: each layer's dW in row splits (dw_splits; the last
        // layer's over its 2 Bp stacked columns, Mp rows), the biases' column sums in row chunks
        // of kSumRows
        for (int l = 0; l < L && !rc; ++l) {
            const size_t O = net.dims[l + 1], I = l == 0 ? k1 : (size_t)net.dims[l];
            const size_t Op = l < L - 1 ? O : (O + 127) / 128 * 128;
            const size_t parts = (size_t)dw_splits(c, (int)Op, (int)I, l < L - 1 ? Bp : 2 * Bp);
            T->gw_buf_floats[l] = parts * Op * I;
            T->gb_buf_floats[l] = (size_t)((Bp + kSumRows - 1) / kSumRows) * O;
            rc = talloc(c, *T, (void **)&T->gw_buf[l], T->gw_buf_floats[l] * 4);
            if (!rc) rc = talloc(c, *T, (void **)&T->gb_buf[l], T->gb_buf_floats[l] * 4);
        }
        if (!rc) rc = talloc(c, *T, (void **)&T->loss, 4);
        if (!rc) rc = talloc(c, *T, (void **)&T->states, (size_t)Bp * 16);
        if (!rc) rc = talloc(c, *T, (void **)&T->labels, (size_t)Bp);
        if (rc) {
            train_free(c, T);
            return rc;
        }
        // masters: from the old state (resize) or from the host copies (layer 0 padded to
        // the one-hot K block with zero columns, which stay zero: their gradient is zero)
        for (int l = 0; l < L; ++l) {
            const size_t O = net.dims[l + 1], I = l == 0 ? k1 : (size_t)net.dims[l];
            if (old) {
                CUDA_TRY(cudaMemcpy(T->w[l], old->w[l], O * I * 4, cudaMemcpyDeviceToDevice));
                CUDA_TRY(cudaMemcpy(T->b[l], old->b[l], O * 4, cudaMemcpyDeviceToDevice));
                CUDA_TRY(cudaMemcpy(T->mw[l], old->mw[l], O * I * 4, cudaMemcpyDeviceToDevice));
                CUDA_TRY(cudaMemcpy(T->vw[l], old->vw[l], O * I * 4, cudaMemcpyDeviceToDevice));
                CUDA_TRY(cudaMemcpy(T->mb[l], old->mb[l], O * 4, cudaMemcpyDeviceToDevice));
                CUDA_TRY(cudaMemcpy(T->vb[l], old->vb[l], O * 4, cudaMemcpyDeviceToDevice));
            } else {
                const size_t Iu = net.dims[l];
                CUDA_TRY(cudaMemcpy2D(T->w[l], I * 4, host_w[l], Iu * 4, Iu * 4, O, cudaMemcpyHostToDevice));
                CUDA_TRY(cudaMemcpy(T->b[l], host_b[l], O * 4, cudaMemcpyHostToDevice));
            }
        }
        if (old) {
            T->step = old->step;
            train_free(c, old);
        }
        net.train = T;
        // W^T copies of the hidden layers >= 1, the last layer's stacked parts
        for (int l = 1; l < L - 1; ++l) {
            const int O = net.dims[l + 1], I = net.dims[l];
            k_write_t<<<(O * I + 255) / 256, 256>>>(T->w[l], O, I, T->wt[l]);
        }
        k_write_ext<<<(C * net.dims[L - 1] + 255) / 256, 256>>>(T->w[L - 1], C, net.dims[L - 1], T->cs, T->w_ext);
        CUDA_TRY(cudaDeviceSynchronize());
    }
    return CBDFS_OK;
}

// forward + loss + backward on the batch already in T.states / T.labels (n rows)
// column sums of X[m][j] over m < n by row chunks (fixed order) into part[R][J]; with sum,
// the chunks then added in order into out (deterministic).  Returns R through *parts.
template <typename T>
static int colsum(const T *X, int n, int J, float *part, size_t part_floats, float *out, bool sum, int *parts,
                  cudaStream_t st) {
    const int R = (n + kSumRows - 1) / kSumRows;
    if ((size_t)R * J > part_floats) return fail(CBDFS_EINVAL, "column-sum scratch");
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if (J % 2 == 0) k_colsum_part2<<<dim3((J / 2 + 255) / 256, R), 256, 0, st>>>(X, n, J, kSumRows, part);
        else k_colsum_part<T><<<dim3((J + 255) / 256, R), 256, 0, st>>>(X, n, J, kSumRows, part);
    } else {
        k_colsum_part<T><<<dim3((J + 255) / 256, R), 256, 0, st>>>(X, n, J, kSumRows, part);
    }
    if (sum) k_sum_splits<<<(J + 255) / 256, 256, 0, st>>>(part, R, J, out);
    *parts = R;
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

// forward + loss + backward on the batch already in T.states / T.labels (n rows).  sum: every
// gradient summed into gw / gb; otherwise the partials stay where gw_src / gb_src say (the
// training step's Adam adds them)
static int train_fwd_bwd(Ctx *c, NetGPU &net, int n, int loss_kind, cudaStream_t st, bool sum, int *ctr = nullptr) {
    TrainState &T = *net.train;
    const int L = net.L, C = net.dims[L];
    const int Bp = (n + kBM - 1) / kBM * kBM;
    int rc;
    // forward through the tensor-core layers: one fused-chain launch storing every hidden layer
    // where the chain takes the network, else layer by layer
    void *outs[kMaxLayers];
    for (int l = 0; l < L - 1; ++l) outs[l] = T.act[l];
    rc = chain_forward_store(c, c->slots[0], net, T.states, (uint32_t)n, outs, (uint32_t)T.Bp, st);
    if (rc != CBDFS_OK && rc != CBDFS_ENOTFOUND) return rc;
    const bool per_layer = rc == CBDFS_ENOTFOUND;
    for (int l = 0; per_layer && l < L - 1; ++l) {
        const bool first = l == 0;
        const int K = first ? net.k1pad : net.dims[l];
        const CUtensorMap *tmA = first ? &net.tm_w[0] : bmap(T, T.act[l - 1], K, T.Bp, kBM);
        if (!tmA) return CBDFS_EDEVICE;
        rc = tc_layer(first, net.domain, false, false, net.bn[l], *tmA, net.tm_w[l], T.states, n, Bp, K,
                      net.dims[l + 1], T.b[l], T.act[l], 1.f, 1.f, c->d_err, st);
        if (rc) return rc;
    }
    const int KL = net.dims[L - 1];
    const dim3 blk(256);
    // logits[m][c] = sum_k A[m][k] W[c][k] + b[c]
    if (net.w_split) {
        // the logits on the tensor cores: the masters' three BF16 parts (re-split after every
        // update) and biases, as the inference head computes them
        const CUtensorMap *ma = bmap(T, T.act[L - 2], KL, Bp, kBM);
        if (!ma) return CBDFS_EDEVICE;
        HeadTcParams H{};
        H.K = KL;
        H.C = C;
        H.cpad = net.head_cpad;
        H.head_kind = net.head;
        H.n = n;
        H.b_last = net.b32[L - 1];
        H.y = T.logits;
        H.err = c->d_err;
        H.groups = 1;
        if (int r = head_tc(net.domain, *ma, net.tm_wsplit, H, Bp, st)) return r;
    } else {
        k_fgemm<__nv_bfloat16, float, true, false><<<dim3((C + FG_T - 1) / FG_T, (n + FG_T - 1) / FG_T, 1), blk, 0, st>>>(
            T.act[L - 2], KL, 1, T.w[L - 1], 1, KL, n, C, KL, T.logits, T.b[L - 1]);
    }
    k_loss<<<(Bp + 7) / 8, 256, 0, st>>>(T.logits, T.labels, n, Bp, C, loss_kind, T.dzl, T.row_loss, T.dz_ext, T.cs);
    k_mean<<<1, 256, 0, st>>>(T.row_loss, n, T.loss, ctr);
    // last layer backward: dW[c][k] = sum_m dZ[m][c] A[m][k] with dZ = D1 + D2 (BF16 parts, the
    // products exact, FP32 accumulation) as one split-K tensor-core GEMM over 2 Bp columns;
    // db = column sums of dZ; dZ_prev = (dZ W) * [A > 0] in BF16
    {
        const int Kd = 2 * Bp;
        k_transpose<<<dim3(T.cs / 64, Bp / 64), dim3(32, 8), 0, st>>>(T.dz_ext, T.t_dz_ext, Bp, T.cs,
                                                                      kExtParts * T.cs, Kd, nullptr, nullptr);
        k_transpose<<<dim3(T.cs / 64, Bp / 64), dim3(32, 8), 0, st>>>(T.dz_ext + 3 * T.cs, T.t_dz_ext + Bp, Bp, T.cs,
                                                                      kExtParts * T.cs, Kd, nullptr, nullptr);
        k_transpose<<<dim3(KL / 64, Bp / 64), dim3(32, 8), 0, st>>>(T.act[L - 2], T.t_a_ext, Bp, KL, KL, Kd,
                                                                    T.t_a_ext + Bp, nullptr);
        const CUtensorMap *ma = bmap(T, T.t_dz_ext, Kd, T.Mp, kBM);
        const CUtensorMap *mb = bmap(T, T.t_a_ext, Kd, KL, KL % 256 == 0 ? 256 : 128);
        if (!ma || !mb) return CBDFS_EDEVICE;
        const int S = dw_splits(c, T.Mp, KL, Kd);
        if ((size_t)S * T.Mp * KL > T.gw_buf_floats[L - 1]) return fail(CBDFS_EINVAL, "dW scratch");
        rc = KL % 256 == 0 ? gemm_tn<256, 1>(*ma, *mb, T.Mp, KL, Kd, T.gw[L - 1], nullptr, c->d_err, st, S, T.gw_buf[L - 1], sum)
                           : gemm_tn<128, 1>(*ma, *mb, T.Mp, KL, Kd, T.gw[L - 1], nullptr, c->d_err, st, S, T.gw_buf[L - 1], sum);
        if (rc) return rc;
        T.gw_src[L - 1] = S > 1 && !sum ? T.gw_buf[L - 1] : T.gw[L - 1];
        T.gw_parts[L - 1] = S > 1 && !sum ? S : 1;
        T.gw_pstride[L - 1] = (size_t)T.Mp * KL;
    }
    {
        int parts = 0;
        if (int r = colsum(T.dzl, n, C, T.gb_buf[L - 1], T.gb_buf_floats[L - 1], T.gb[L - 1], sum, &parts, st)) return r;
        T.gb_src[L - 1] = sum ? T.gb[L - 1] : T.gb_buf[L - 1];
        T.gb_parts[L - 1] = sum ? 1 : parts;
    }
    {
        // dZ_{L-2} = (dZ_L W_L) * [A_{L-2} > 0]: the split parts on the tensor cores (rows n..Bp-1
        // of dz_ext are zero, so those rows of the product are zero)
        const int Ke = kExtParts * T.cs;
        const CUtensorMap *mz = bmap(T, T.dz_ext, Ke, T.Bp, kBM);
        const CUtensorMap *mw = bmap(T, T.w_ext, Ke, KL, KL % 256 == 0 ? 256 : 128);
        if (!mz || !mw) return CBDFS_EDEVICE;
        rc = KL % 256 == 0 ? gemm_tn<256, 2>(*mz, *mw, Bp, KL, Ke, T.dz[L - 2], T.act[L - 2], c->d_err, st)
                           : gemm_tn<128, 2>(*mz, *mw, Bp, KL, Ke, T.dz[L - 2], T.act[L - 2], c->d_err, st);
        if (rc) return rc;
    }
    // hidden layers, last to first
    for (int l = L - 2; l >= 0; --l) {
        const int O = net.dims[l + 1], I = l == 0 ? net.k1pad : net.dims[l];
        // dW_l = dZ_l^T A_{l-1}, both operands MN-major as the backward stores them ([batch][O],
        // [batch][I]); layer 0's A is the one-hot, written transposed (K-major over the batch)
        if (l == 0) {
            CUDA_TRY(cudaMemsetAsync(T.t_a, 0, (size_t)I * Bp * 2, st));
            if (net.domain == CBDFS_DOM_STP3) k_onehot_t<CBDFS_DOM_STP3><<<(Bp + 255) / 256, 256, 0, st>>>(T.states, n, Bp, T.t_a);
            else if (net.domain == CBDFS_DOM_STP4) k_onehot_t<CBDFS_DOM_STP4><<<(Bp + 255) / 256, 256, 0, st>>>(T.states, n, Bp, T.t_a);
            else k_onehot_t<CBDFS_DOM_RC3><<<(Bp + 255) / 256, 256, 0, st>>>(T.states, n, Bp, T.t_a);
        }
        // the output width is the (padded) input width; padding columns of the one-hot are
        // zero, so their gradient is exactly zero
        const CUtensorMap *ma = bmap(T, T.dz[l], O, T.Bp, 64);
        const CUtensorMap *mb = l == 0 ? bmap(T, T.t_a, Bp, I, I % 256 == 0 ? 256 : 128) : bmap(T, T.act[l - 1], I, T.Bp, 64);
        if (!ma || !mb) return CBDFS_EDEVICE;
        const int S = dw_splits(c, O, I, Bp);
        if ((size_t)S * O * I > T.gw_buf_floats[l]) return fail(CBDFS_EINVAL, "dW scratch");
        if (l == 0)
            rc = (I % 256 == 0) ? gemm_tn<256, 1, true, false>(*ma, *mb, O, I, Bp, T.gw[l], nullptr, c->d_err, st, S, T.gw_buf[l], sum)
                                : gemm_tn<128, 1, true, false>(*ma, *mb, O, I, Bp, T.gw[l], nullptr, c->d_err, st, S, T.gw_buf[l], sum);
        else
            rc = (I % 256 == 0) ? gemm_tn<256, 1, true, true>(*ma, *mb, O, I, Bp, T.gw[l], nullptr, c->d_err, st, S, T.gw_buf[l], sum)
                                : gemm_tn<128, 1, true, true>(*ma, *mb, O, I, Bp, T.gw[l], nullptr, c->d_err, st, S, T.gw_buf[l], sum);
        if (rc) return rc;
        T.gw_src[l] = S > 1 && !sum ? T.gw_buf[l] : T.gw[l];
        T.gw_parts[l] = S > 1 && !sum ? S : 1;
        T.gw_pstride[l] = (size_t)O * I;
        {
            // db_l: the column sums of dZ_l per 64-row chunk, rows in order (rows n..Bp-1 are zero)
            int parts = 0;
            if (int r = colsum(T.dz[l], n, O, T.gb_buf[l], T.gb_buf_floats[l], T.gb[l], sum, &parts, st)) return r;
            T.gb_src[l] = sum ? T.gb[l] : T.gb_buf[l];
            T.gb_parts[l] = sum ? 1 : parts;
        }
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l) * [A_{l-1} > 0]
            const CUtensorMap *mz = bmap(T, T.dz[l], O, T.Bp, kBM);
            const CUtensorMap *mw = bmap(T, T.wt[l], O, I, I % 256 == 0 ? 256 : 128);
            if (!mz || !mw) return CBDFS_EDEVICE;
            rc = (I % 256 == 0) ? gemm_tn<256, 2>(*mz, *mw, Bp, I, O, T.dz[l - 1], T.act[l - 1], c->d_err, st)
                                : gemm_tn<128, 2>(*mz, *mw, Bp, I, O, T.dz[l - 1], T.act[l - 1], c->d_err, st);
            if (rc) return rc;
        }
    }
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

// one Adam launch over every tensor (copies_only: no update, the copies of the masters)
// c12/ctr: the bias corrections from a table at the device step counter (see AdamParams)
static int launch_adam(NetGPU &net, const cbdfs_train_cfg *tc, bool copies_only, cudaStream_t st,
                       const float *c12 = nullptr, const int *ctr = nullptr) {
    TrainState &T = *net.train;
    AdamParams A{};
    A.copies_only = copies_only ? 1 : 0;
    A.c12 = c12;
    A.ctr = ctr;
    if (tc) {
        A.lr = tc->lr;
        A.b1 = tc->beta1;
        A.b2 = tc->beta2;
        A.eps = tc->eps;
        A.c1 = 1.f - powf(tc->beta1, (float)T.step);
        A.c2 = 1.f - powf(tc->beta2, (float)T.step);
    }
    int blocks = 0;
    auto add = [&](const AdamSeg &g) {
        A.seg[A.nseg] = g;
        A.seg[A.nseg].block0 = blocks;
        blocks += (g.O * g.I + 255) / 256;
        ++A.nseg;
    };
    for (int l = 0; l < net.L; ++l) {
        const int O = net.dims[l + 1], I = l == 0 ? net.k1pad : net.dims[l];
        const bool last = l == net.L - 1;
        AdamSeg w{};
        w.w = T.w[l];
        w.g = T.gw_src[l];
        w.parts = T.gw_parts[l];
        w.pstride = T.gw_pstride[l];
        w.m = T.mw[l];
        w.v = T.vw[l];
        w.O = O;
        w.I = I;
        w.w_lp = last ? nullptr : static_cast<__nv_bfloat16 *>(net.w_lp[l]);
        w.Kp = I;
        w.wt = (l >= 1 && !last) ? T.wt[l] : nullptr;
        w.w_out = last ? net.w32[l] : nullptr;  // the inference head reads the FP32 last layer
        w.split = last ? static_cast<__nv_bfloat16 *>(net.w_split) : nullptr;  // and the tensor-core head its parts
        w.cpad = net.head_cpad;
        w.w_ext = last ? T.w_ext : nullptr;  // and the backward its stacked parts
        w.cs = T.cs;
        add(w);
        AdamSeg b{};
        b.w = T.b[l];
        b.g = T.gb_src[l];
        b.parts = T.gb_parts[l];
        b.pstride = O;
        b.m = T.mb[l];
        b.v = T.vb[l];
        b.O = O;
        b.I = 1;
        b.w_out = net.b32[l];
        add(b);
    }
    k_adam_all<<<blocks, 256, 0, st>>>(A);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}



// ---- training checkpoints ---------------------------------------------------------------
namespace {

struct TrainFileHeader {
    char magic[8];
    uint32_t version, L;
    uint32_t dims[kMaxLayers + 1];
    uint32_t k1pad;
    int64_t step;
    uint64_t payload, hash;
};
constexpr char kTrainMagic[8] = {'C', 'B', 'D', 'F', 'S', 'T', 'R', 'N'};
constexpr uint64_t kFnvBasis = 14695981039346656037ull;

// layer l's six FP32 tensors in file order: W, b, m(W), v(W), m(b), v(b)
void layer_tensors(TrainState &T, const NetGPU &net, int l, float *(&p)[6], size_t (&cnt)[6]) {
    const size_t O = net.dims[l + 1], I = l == 0 ? (size_t)net.k1pad : (size_t)net.dims[l];
    float *pp[6] = {T.w[l], T.b[l], T.mw[l], T.vw[l], T.mb[l], T.vb[l]};
    const size_t cc[6] = {O * I, O, O * I, O * I, O, O};
    for (int i = 0; i < 6; ++i) {
        p[i] = pp[i];
        cnt[i] = cc[i];
    }
}

// the training state, created from the loaded weights if the network has not been trained
int ensure_train_state(Ctx *c, NetGPU &net) {
    if (net.train) return CBDFS_OK;
    std::vector<const float *> hw, hb;
    for (int l = 0; l < net.L; ++l) {
        hw.push_back(net.host_w[l].data());
        hb.push_back(net.host_b[l].data());
    }
    return train_setup(c, net, (int)std::min<uint32_t>(c->max_batch, 8192), hw.data(), hb.data());
}

struct FileCloser {
    FILE *f = nullptr;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

}  // namespace

}  // namespace cbdfs

using namespace cbdfs;

static int get_train_net(cbdfs_ctx *ctx, int net_id, NetGPU **out) {
    if (!ctx) return fail(CBDFS_EINVAL, "null context");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (net_id < 0 || net_id >= (int)c->heur_kind.size() || c->heur_kind[net_id] != 0)
        return fail(CBDFS_EINVAL, "heuristic %d is not a network", net_id);
    *out = c->nets[c->heur_index[net_id]].get();
    return CBDFS_OK;
}

static int upload_batch(Ctx *c, NetGPU &net, const uint64_t *states, const uint8_t *labels, uint32_t n, cudaStream_t st) {
    TrainState &T = *net.train;
    const int w = dom_words(net.domain);
    CUDA_TRY(cudaMemcpyAsync(T.states, states, (size_t)n * 8 * w, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(T.labels, labels, n, cudaMemcpyHostToDevice, st));
    return CBDFS_OK;
}

static int check_labels(const NetGPU &net, const uint8_t *labels, uint64_t n, int loss) {
    if (loss == CBDFS_LOSS_CE) {
        for (uint64_t i = 0; i < n; ++i)
            if (labels[i] >= net.dims[net.L]) return fail(CBDFS_EINVAL, "label %d of state %llu outside the %d classes", labels[i], (unsigned long long)i, net.dims[net.L]);
    } else if (net.dims[net.L] != 1) {
        return fail(CBDFS_EINVAL, "the squared-error loss needs one output");
    }
    return CBDFS_OK;
}

extern "C" {

int cbdfs_train_grad(cbdfs_ctx *ctx, int net_id, const uint64_t *states, const uint8_t *labels, uint32_t n,
                     int loss, float *loss_out, float *const *gw_out, float *const *gb_out) {
    NetGPU *net;
    int rc = get_train_net(ctx, net_id, &net);
    if (rc) return rc;
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!states || !labels || !loss_out || !gw_out || !gb_out || n == 0) return fail(CBDFS_EINVAL, "null argument");
    if (loss != CBDFS_LOSS_CE && loss != CBDFS_LOSS_MSE) return fail(CBDFS_EINVAL, "loss %d", loss);
    if ((rc = check_labels(*net, labels, n, loss))) return rc;
    CUDA_TRY(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    const float *const *hw = nullptr;
    std::vector<const float *> hwv, hbv;
    for (int l = 0; l < net->L; ++l) {
        hwv.push_back(net->host_w[l].data());
        hbv.push_back(net->host_b[l].data());
    }
    hw = hwv.data();
    if ((rc = train_setup(c, *net, (int)n, hw, hbv.data()))) return rc;
    cudaStream_t st = c->slots[0].stream;
    if ((rc = upload_batch(c, *net, states, labels, n, st))) return rc;
    if ((rc = train_fwd_bwd(c, *net, (int)n, loss, st, true))) return rc;
    TrainState &T = *net->train;
    CUDA_TRY(cudaMemcpyAsync(loss_out, T.loss, 4, cudaMemcpyDeviceToHost, st));
    for (int l = 0; l < net->L; ++l) {
        const size_t O = net->dims[l + 1], Iu = net->dims[l], I = l == 0 ? (size_t)net->k1pad : Iu;
        if (gw_out[l])
            CUDA_TRY(cudaMemcpy2DAsync(gw_out[l], Iu * 4, T.gw[l], I * 4, Iu * 4, O, cudaMemcpyDeviceToHost, st));
        if (gb_out[l]) CUDA_TRY(cudaMemcpyAsync(gb_out[l], T.gb[l], O * 4, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    int flag = 0;
    CUDA_TRY(cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(CBDFS_ETIMEDOUT, "a device wait ran out (code %d)", flag);
    return CBDFS_OK;
}

int net_train(cbdfs_ctx *ctx, int net_id, const uint64_t *states, const uint8_t *labels, uint64_t n,
              const cbdfs_train_cfg *cfg, cbdfs_train_report *rep) {
    NetGPU *net;
    int rc = get_train_net(ctx, net_id, &net);
    if (rc) return rc;
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!states || !labels || !cfg || !rep || n == 0) return fail(CBDFS_EINVAL, "null argument");
    // the server's launches read the weights the optimizer rewrites
    if (c->server) return fail(CBDFS_EINVAL, "stop the server before training");
    cbdfs_train_cfg tc = *cfg;
    if (tc.batch == 0 || tc.batch > c->max_batch) return fail(CBDFS_EINVAL, "batch %u outside 1..max_batch", tc.batch);
    if (tc.epochs < 1) return fail(CBDFS_EINVAL, "epochs %d", tc.epochs);
    if (tc.loss != CBDFS_LOSS_CE && tc.loss != CBDFS_LOSS_MSE) return fail(CBDFS_EINVAL, "loss %d", tc.loss);
    if (n > 0xFFFFFFFFull) return fail(CBDFS_EINVAL, "too many states");
    if ((rc = check_labels(*net, labels, n, tc.loss))) return rc;
    memset(rep, 0, sizeof(*rep));
    CUDA_TRY(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    std::vector<const float *> hwv, hbv;
    for (int l = 0; l < net->L; ++l) {
        hwv.push_back(net->host_w[l].data());
        hbv.push_back(net->host_b[l].data());
    }
    if ((rc = train_setup(c, *net, (int)tc.batch, hwv.data(), hbv.data()))) return rc;
    TrainState &T = *net->train;
    cudaStream_t st = c->slots[0].stream;
    const int w = dom_words(net->domain);
    // the whole training set on the device
    uint64_t *d_states = nullptr;
    uint8_t *d_labels = nullptr;
    uint32_t *d_idx = nullptr;
    const uint64_t per_epoch = (n + tc.batch - 1) / tc.batch;
    int64_t total = (int64_t)tc.epochs * (int64_t)per_epoch;
    if (tc.max_steps > 0) total = std::min<int64_t>(total, tc.max_steps);
    // the run's device counters (step in the run, batch in the epoch) and every step's Adam bias
    // corrections, computed here as a single step computes them, so that one captured step
    // (a CUDA graph: gather, forward, backward, update) replays for every full batch
    int *d_ctr = nullptr;
    float *d_c12 = nullptr;
    cudaGraphExec_t step_graph = nullptr;
    auto cleanup = [&]() {
        if (step_graph) cudaGraphExecDestroy(step_graph);
        dev_free(c, d_states, n * 8 * w);
        dev_free(c, d_labels, n);
        dev_free(c, d_idx, n * 4);
        dev_free(c, d_ctr, 2 * sizeof(int));
        dev_free(c, d_c12, 2 * sizeof(float) * (size_t)total);
    };
    if ((rc = dev_alloc(c, (void **)&d_states, n * 8 * w)) || (rc = dev_alloc(c, (void **)&d_labels, n)) ||
        (rc = dev_alloc(c, (void **)&d_idx, n * 4)) || (rc = dev_alloc(c, (void **)&d_ctr, 2 * sizeof(int))) ||
        (rc = dev_alloc(c, (void **)&d_c12, 2 * sizeof(float) * (size_t)total))) {
        cleanup();
        return rc;
    }
    {
        std::vector<float> c12(2 * (size_t)total);
        for (int64_t j = 0; j < total; ++j) {
            const float t = (float)(T.step + 1 + j);
            c12[2 * j] = 1.f - powf(tc.beta1, t);
            c12[2 * j + 1] = 1.f - powf(tc.beta2, t);
        }
        if (cudaMemcpy(d_c12, c12.data(), c12.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(d_ctr, 0, 2 * sizeof(int)) != cudaSuccess) {
            cleanup();
            return fail(CBDFS_EDEVICE, "training counters");
        }
    }
    // one step on the stream: rows from the permutation at the batch counter, forward, loss
    // (whose mean kernel advances both counters), backward, Adam at the step counter
    auto enqueue_step = [&](uint32_t bn) -> int {
        k_gather<<<(bn + 255) / 256, 256, 0, st>>>(d_states, d_labels, d_idx, d_ctr, tc.batch, w, bn, T.states, T.labels);
        int r = train_fwd_bwd(c, *net, (int)bn, tc.loss, st, false, d_ctr);
        if (!r) r = launch_adam(*net, &tc, false, st, d_c12, d_ctr);
        return r;
    };
    if (cudaMemcpy(d_states, states, n * 8 * w, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_labels, labels, n, cudaMemcpyHostToDevice) != cudaSuccess) {
        cleanup();
        return fail(CBDFS_EDEVICE, "training set upload");
    }
    // epoch order: Fisher-Yates driven by splitmix64(seed + epoch), j = draw mod (i+1).  The next
    // epoch's order is drawn on a host thread while this epoch's steps run, into the other of
    // two page-locked buffers (a buffer is rewritten once its previous upload has completed)
    auto make_perm = [n, seed = tc.seed](int ep, uint32_t *perm) {
        for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
        uint64_t sm = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(ep + 1);
        for (uint64_t i = n - 1; i > 0; --i) {
            sm += 0x9E3779B97F4A7C15ull;
            uint64_t z = sm;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            std::swap(perm[i], perm[z % (i + 1)]);
        }
    };
    uint32_t *hperm[2] = {nullptr, nullptr};
    cudaEvent_t up_ev[2] = {nullptr, nullptr};
    std::thread drawer;
    auto perm_cleanup = [&]() {
        if (drawer.joinable()) drawer.join();
        cudaStreamSynchronize(st);  // no upload still reads the buffers
        for (int b = 0; b < 2; ++b) {
            if (up_ev[b]) cudaEventDestroy(up_ev[b]);
            if (hperm[b]) cudaFreeHost(hperm[b]);
        }
    };
    for (int b = 0; b < 2; ++b)
        if (cudaHostAlloc((void **)&hperm[b], n * 4, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&up_ev[b], cudaEventDisableTiming) != cudaSuccess) {
            perm_cleanup();
            cleanup();
            return fail(CBDFS_ENOMEM, "page-locked permutation buffers");
        }
    const auto t0 = std::chrono::steady_clock::now();
    make_perm(0, hperm[0]);
    float loss = 0.f;
    int64_t steps = 0;
    for (int ep = 0; ep < tc.epochs && !rc; ++ep) {
        if (drawer.joinable()) drawer.join();  // this epoch's order is in hperm[ep & 1]
        if (cudaMemcpyAsync(d_idx, hperm[ep & 1], n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaEventRecord(up_ev[ep & 1], st) != cudaSuccess ||
            cudaMemsetAsync(d_ctr + 1, 0, sizeof(int), st) != cudaSuccess) {
            rc = fail(CBDFS_EDEVICE, "permutation upload");
            break;
        }
        const bool more = ep + 1 < tc.epochs && !(tc.max_steps > 0 && steps + (int64_t)per_epoch >= tc.max_steps);
        if (more) {
            // the other buffer was last read by the previous epoch's upload
            if (ep >= 1 && cudaEventSynchronize(up_ev[(ep + 1) & 1]) != cudaSuccess) {
                rc = fail(CBDFS_EDEVICE, "permutation upload");
                break;
            }
            drawer = std::thread(make_perm, ep + 1, hperm[(ep + 1) & 1]);
        }
        for (uint64_t k = 0; k < per_epoch && !rc; ++k) {
            if (tc.max_steps > 0 && steps >= tc.max_steps) break;
            const uint32_t off = (uint32_t)(k * tc.batch);
            const uint32_t bn = (uint32_t)std::min<uint64_t>(tc.batch, n - off);
            if (bn == tc.batch) {
                if (!step_graph) {
                    cudaGraph_t g = nullptr;
                    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                        rc = fail(CBDFS_EDEVICE, "step capture");
                        break;
                    }
                    rc = enqueue_step(bn);
                    const cudaError_t e = cudaStreamEndCapture(st, &g);
                    if (!rc && e != cudaSuccess) rc = fail(CBDFS_EDEVICE, "step capture: %s", cudaGetErrorString(e));
                    if (!rc && cudaGraphInstantiate(&step_graph, g, 0) != cudaSuccess) {
                        step_graph = nullptr;
                        rc = fail(CBDFS_EDEVICE, "step graph instantiate");
                    }
                    if (g) cudaGraphDestroy(g);
                    if (rc) break;
                }
                if (cudaGraphLaunch(step_graph, st) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "step graph launch");
            } else {
                rc = enqueue_step(bn);  // the epoch's last, partial batch
            }
            T.step++;
            if (!rc && (steps == 0 || (steps & 255) == 255)) {
                if (cudaMemcpyAsync(&loss, T.loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = fail(CBDFS_EDEVICE, "training step");
                    break;
                }
                if (steps == 0) rep->first_loss = loss;
            }
            ++steps;
        }
        if (tc.max_steps > 0 && steps >= tc.max_steps) break;
    }
    if (!rc) {
        if (cudaMemcpyAsync(&loss, T.loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = fail(CBDFS_EDEVICE, "training: %s", cudaGetErrorString(cudaGetLastError()));
        rep->last_loss = loss;
    }
    rep->steps = steps;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->samples = 0;
    for (int64_t i = 0; i < steps; ++i) rep->samples += std::min<uint64_t>(tc.batch, n);
    perm_cleanup();
    cleanup();
    if (!rc) {
        int flag = 0;
        if (cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && flag)
            rc = fail(CBDFS_ETIMEDOUT, "a device wait ran out (code %d)", flag);
    }
    return rc;
}

int cbdfs_net_read(cbdfs_ctx *ctx, int net_id, float *const *w_out, float *const *b_out) {
    NetGPU *net;
    int rc = get_train_net(ctx, net_id, &net);
    if (rc) return rc;
    if (!w_out || !b_out) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    CUDA_TRY(cudaSetDevice(c->device));
    for (int l = 0; l < net->L; ++l) {
        const size_t O = net->dims[l + 1], Iu = net->dims[l];
        if (net->train) {
            const size_t I = l == 0 ? (size_t)net->k1pad : Iu;
            if (w_out[l]) CUDA_TRY(cudaMemcpy2D(w_out[l], Iu * 4, net->train->w[l], I * 4, Iu * 4, O, cudaMemcpyDeviceToHost));
            if (b_out[l]) CUDA_TRY(cudaMemcpy(b_out[l], net->train->b[l], O * 4, cudaMemcpyDeviceToHost));
        } else {
            if (w_out[l]) memcpy(w_out[l], net->host_w[l].data(), O * Iu * 4);
            if (b_out[l]) memcpy(b_out[l], net->host_b[l].data(), O * 4);
        }
    }
    return CBDFS_OK;
}

int cbdfs_gen_walk_states(cbdfs_ctx *ctx, int domain, uint32_t tag, uint64_t first, uint64_t n, int max_len,
                          uint64_t *states_out) {
    if (!ctx || !states_out) return fail(CBDFS_EINVAL, "null argument");
    if (domain != CBDFS_DOM_STP3 && domain != CBDFS_DOM_STP4) return fail(CBDFS_EINVAL, "walks are for sliding-tile domains");
    if (max_len < 1) return fail(CBDFS_EINVAL, "max_len %d", max_len);
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = c->slots[0].stream;
    const uint64_t chunk = 1ull << 22;
    uint64_t *d = nullptr;
    int rc = dev_alloc(c, (void **)&d, std::min(n, chunk) * 8);
    if (rc) return rc;
    for (uint64_t o = 0; o < n && !rc; o += chunk) {
        const uint32_t m = (uint32_t)std::min(chunk, n - o);
        if (domain == CBDFS_DOM_STP3) k_walks<3><<<(m + 255) / 256, 256, 0, st>>>(tag, first + o, m, max_len, d);
        else k_walks<4><<<(m + 255) / 256, 256, 0, st>>>(tag, first + o, m, max_len, d);
        if (cudaMemcpyAsync(states_out + o, d, (size_t)m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = fail(CBDFS_EDEVICE, "walk generation");
    }
    dev_free(c, d, std::min(n, chunk) * 8);
    return rc;
}


int cbdfs_train_save(cbdfs_ctx *ctx, int net_id, const char *path) {
    NetGPU *net;
    int rc = get_train_net(ctx, net_id, &net);
    if (rc) return rc;
    if (!path) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    CUDA_TRY(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    if ((rc = ensure_train_state(c, *net))) return rc;
    CUDA_TRY(cudaDeviceSynchronize());
    TrainState &T = *net->train;
    std::vector<unsigned char> payload;
    for (int l = 0; l < net->L; ++l) {
        float *p[6];
        size_t cnt[6];
        layer_tensors(T, *net, l, p, cnt);
        for (int i = 0; i < 6; ++i) {
            const size_t off = payload.size();
            payload.resize(off + cnt[i] * 4);
            CUDA_TRY(cudaMemcpy(payload.data() + off, p[i], cnt[i] * 4, cudaMemcpyDeviceToHost));
        }
    }
    TrainFileHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kTrainMagic, 8);
    hd.version = 1;
    hd.L = (uint32_t)net->L;
    for (int l = 0; l <= net->L; ++l) hd.dims[l] = (uint32_t)net->dims[l];
    hd.k1pad = (uint32_t)net->k1pad;
    hd.step = T.step;
    hd.payload = payload.size();
    hd.hash = fnv1a64(payload.data(), payload.size(), kFnvBasis);
    FileCloser out;
    out.f = fopen(path, "wb");
    if (!out.f) return fail(CBDFS_EDEVICE, "%s: %s", path, strerror(errno));
    if (fwrite(&hd, sizeof hd, 1, out.f) != 1 || fwrite(payload.data(), 1, payload.size(), out.f) != payload.size())
        return fail(CBDFS_EDEVICE, "%s: short write", path);
    const int closed = fclose(out.f);
    out.f = nullptr;
    return closed == 0 ? CBDFS_OK : fail(CBDFS_EDEVICE, "%s: close", path);
}

int cbdfs_train_load(cbdfs_ctx *ctx, int net_id, const char *path) {
    NetGPU *net;
    int rc = get_train_net(ctx, net_id, &net);
    if (rc) return rc;
    if (!path) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    // the server's launches read the weights this rewrites
    if (c->server) return fail(CBDFS_EINVAL, "stop the server before loading a checkpoint");
    if (net->prec != CBDFS_PREC_BF16) return fail(CBDFS_EINVAL, "training needs a BF16 network");
    FileCloser in;
    in.f = fopen(path, "rb");
    if (!in.f) return fail(CBDFS_ENOTFOUND, "%s: %s", path, strerror(errno));
    TrainFileHeader hd;
    if (fread(&hd, sizeof hd, 1, in.f) != 1 || std::memcmp(hd.magic, kTrainMagic, 8) != 0)
        return fail(CBDFS_EINVAL, "%s is not a training checkpoint", path);
    if (hd.version != 1) return fail(CBDFS_EINVAL, "%s: format version %u", path, hd.version);
    bool same = hd.L == (uint32_t)net->L && hd.k1pad == (uint32_t)net->k1pad;
    for (int l = 0; l <= net->L && same; ++l) same = hd.dims[l] == (uint32_t)net->dims[l];
    if (!same) return fail(CBDFS_EINVAL, "%s holds another network shape", path);
    size_t want = 0;
    for (int l = 0; l < net->L; ++l) {
        const size_t O = net->dims[l + 1], I = l == 0 ? (size_t)net->k1pad : (size_t)net->dims[l];
        want += (3 * O * I + 3 * O) * 4;
    }
    if (hd.payload != want) return fail(CBDFS_EINVAL, "%s: payload of %llu bytes, %zu expected", path,
                                        (unsigned long long)hd.payload, want);
    std::vector<unsigned char> payload(want);
    if (fread(payload.data(), 1, want, in.f) != want) return fail(CBDFS_EINVAL, "%s: short file", path);
    if (fnv1a64(payload.data(), want, kFnvBasis) != hd.hash) return fail(CBDFS_EINVAL, "%s: hash mismatch", path);
    CUDA_TRY(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    if ((rc = ensure_train_state(c, *net))) return rc;
    CUDA_TRY(cudaDeviceSynchronize());
    TrainState &T = *net->train;
    size_t off = 0;
    for (int l = 0; l < net->L; ++l) {
        float *p[6];
        size_t cnt[6];
        layer_tensors(T, *net, l, p, cnt);
        for (int i = 0; i < 6; ++i) {
            CUDA_TRY(cudaMemcpy(p[i], payload.data() + off, cnt[i] * 4, cudaMemcpyHostToDevice));
            off += cnt[i] * 4;
        }
    }
    T.step = hd.step;
    // the copies the heuristic and the backward read: BF16 weights, transposes, FP32 head, parts
    cudaStream_t st = c->slots[0].stream;
    if ((rc = launch_adam(*net, nullptr, true, st))) return rc;
    CUDA_TRY(cudaStreamSynchronize(st));
    return CBDFS_OK;
}

}  // extern "C"
