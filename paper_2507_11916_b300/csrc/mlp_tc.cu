// mlp_tc.cu -- the network heuristic's hidden layers on the 5th-generation tensor cores.
//
// One launch computes one layer for a batch of states:  out = ReLU(A W^T + b), A the
// previous layer's activations (or, for the first layer, the one-hot encoding of the
// packed states, built here in shared memory), W the layer's weights, K-major.
//
// CTA tile: 128 states x BN outputs, K in blocks of 128 bytes (64 BF16 or 128 E4M3).
//   warp 0      TMA producer: weight tiles (and activation tiles) into a ring of stages
//   warp 1      owns the TMEM accumulator; one lane issues tcgen05.mma, commits each
//               stage back to the producer and the finished tile to the epilogue
//   warps 2..5  epilogue: tcgen05.ld the FP32 accumulator, add bias, ReLU, convert to
//               BF16 (or scale to E4M3) and store the activation row
// For the first layer all six warps first decode their states (one coalesced 8- or
// 16-byte load per state) into the one-hot A tile (the paper's TensorRepresentation of
// Algorithm 3, moved from the CPU to the GPU), which stays resident for every K block.
// Every mbarrier wait is bounded (common.cuh) and reports through the error flag.
#include <cuda_fp8.h>

#include "common.cuh"

namespace cbdfs {
namespace {

using namespace dev;

constexpr int kThreads = 192;
constexpr int kStageA = kBM * 128;  // bytes of one A k-block (128 rows x 128 B)

template <int DOMAIN, bool FP8>
__device__ __forceinline__ void put_one(uint8_t *A, int r, int j) {
    // (row r, k-index j) -> byte offset in the 128B-swizzled K-major layout
    if (FP8) {
        int kb = j >> 7, w = j & 127;
        uint32_t off = kb * kStageA + r * 128 + ((((w >> 4) ^ (r & 7)) << 4) | (w & 15));
        A[off] = 0x38;  // E4M3 1.0
    } else {
        int kb = j >> 6, w = j & 63;
        uint32_t off = kb * kStageA + r * 128 + ((((w >> 3) ^ (r & 7)) << 4) | ((w & 7) << 1));
        *reinterpret_cast<uint16_t *>(A + off) = 0x3F80;  // BF16 1.0
    }
}

template <int DOMAIN, bool FP8>
__device__ __forceinline__ void encode_row(uint8_t *A, int r, const uint64_t *__restrict__ states,
                                           uint32_t m) {
    if (DOMAIN == CBDFS_DOM_RC3) {
        const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(states) + m);
#pragma unroll
        for (int c = 0; c < 8; ++c) put_one<DOMAIN, FP8>(A, r, c * 24 + (int)((w.x >> (5 * c)) & 31u));
#pragma unroll
        for (int e = 0; e < 12; ++e)
            put_one<DOMAIN, FP8>(A, r, 192 + e * 24 + (int)((w.y >> (5 * e)) & 31u));
    } else {
        constexpr int N = DOMAIN == CBDFS_DOM_STP3 ? 9 : 16;
        const uint64_t s = __ldg(states + m);
#pragma unroll
        for (int p = 0; p < N; ++p) put_one<DOMAIN, FP8>(A, r, (int)((s >> (4 * p)) & 15u) * N + p);
    }
}

// FIRST: A = one-hot(states) built in smem.  DOMAIN only matters when FIRST.
// OUT_FP8: store E4M3 activations scaled by out_qscale (= 1 / activation scale).
template <int BN, bool FIRST, int DOMAIN, bool FP8, bool OUT_FP8>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_layer(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const uint64_t *__restrict__ states, uint32_t n, int K, int N,
           const float *__restrict__ bias, void *__restrict__ out, float acc_scale,
           float out_qscale, int stages, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    constexpr int kStageB = BN * 128;
    const int KB = K / (FP8 ? 128 : 64);                 // k-blocks
    const int a_bytes = FIRST ? KB * kStageA : stages * kStageA;
    uint8_t *A = smem;
    uint8_t *B = smem + a_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(B + stages * kStageB);
    uint64_t *full = bars, *empty = bars + stages, *accum = bars + 2 * stages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN;
    const int m0 = blockIdx.y * kBM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accum), 1);
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        if (!FIRST) tma_prefetch_map(&tmA);
        tma_prefetch_map(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), BN);
        tmem_relinquish();
    }
    if (FIRST) {
        // one-hot A: zero the tile, then one thread per row sets its 1s
        uint4 *A4 = reinterpret_cast<uint4 *>(A);
        const int nvec = KB * kStageA / 16;
        for (int i = threadIdx.x; i < nvec; i += kThreads) A4[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        if (threadIdx.x < kBM && m0 + threadIdx.x < n)
            encode_row<DOMAIN, FP8>(A, threadIdx.x, states, m0 + threadIdx.x);
        fence_proxy_async();  // make the generic-proxy writes visible to the tensor cores
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t tx = kStageB + (FIRST ? 0 : kStageA);
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % stages, u = kb / stages;
                if (kb >= stages && !mbar_wait(smem_u32(&empty[s]), (u - 1) & 1, err, DEVERR_STAGE_EMPTY))
                    break;
                mbar_arrive_expect_tx(smem_u32(&full[s]), tx);
                const int kx = kb * (FP8 ? 128 : 64);
                if (!FIRST) tma_load_2d(smem_u32(A + s * kStageA), &tmA, smem_u32(&full[s]), kx, m0);
                tma_load_2d(smem_u32(B + s * kStageB), &tmB, smem_u32(&full[s]), kx, n0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = FP8 ? make_idesc(kBM, BN, 0, 0) : make_idesc(kBM, BN, 1, 1);
            bool ok = true;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % stages, u = kb / stages;
                if (!mbar_wait(smem_u32(&full[s]), u & 1, err, DEVERR_TMA_FULL)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(FIRST ? A + kb * kStageA : A + s * kStageA);
                const uint64_t ad = sw128_desc(a_addr), bd = sw128_desc(smem_u32(B + s * kStageB));
#pragma unroll
                for (int k = 0; k < 4; ++k) {  // 4 MMAs of 32 bytes of K each
                    if (FP8) umma_fp8(tmem_d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                    else umma_bf16(tmem_d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                }
                umma_commit(smem_u32(&empty[s]));
            }
            if (ok) umma_commit(smem_u32(accum));
            else atomicCAS(err, 0, DEVERR_TMA_FULL);
        }
    } else {
        // epilogue: warps 2..5 cover TMEM lane quarters (warp % 4)
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const uint32_t m = m0 + row;
        if (mbar_wait(smem_u32(accum), 0, err, DEVERR_ACCUM)) {
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(tmem_d + ((uint32_t)(q * 32) << 16) + c * 32, r);
                tmem_ld_wait();
                const float4 *b4 = reinterpret_cast<const float4 *>(bias + n0 + c * 32);
                float v[32];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 bb = __ldg(b4 + j);
                    v[4 * j + 0] = fmaxf(fmaf(__uint_as_float(r[4 * j + 0]), acc_scale, bb.x), 0.f);
                    v[4 * j + 1] = fmaxf(fmaf(__uint_as_float(r[4 * j + 1]), acc_scale, bb.y), 0.f);
                    v[4 * j + 2] = fmaxf(fmaf(__uint_as_float(r[4 * j + 2]), acc_scale, bb.z), 0.f);
                    v[4 * j + 3] = fmaxf(fmaf(__uint_as_float(r[4 * j + 3]), acc_scale, bb.w), 0.f);
                }
                if (OUT_FP8) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        __nv_fp8x4_e4m3 q4(make_float4(v[4 * j] * out_qscale, v[4 * j + 1] * out_qscale,
                                                       v[4 * j + 2] * out_qscale, v[4 * j + 3] * out_qscale));
                        pk[j] = *reinterpret_cast<uint32_t *>(&q4);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(out) +
                                                           (size_t)m * N + n0 + c * 32);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else {
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        pk[j] = *reinterpret_cast<uint32_t *>(&h2);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(out) +
                                                           (size_t)m * N + n0 + c * 32);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                }
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

template <int BN, bool FIRST, int DOMAIN, bool FP8, bool OUT_FP8>
int launch_layer(const CUtensorMap &tmA, const CUtensorMap &tmB, const uint64_t *states, uint32_t n,
                 uint32_t rows_pad, int K, int N, const float *bias, void *out, float acc_scale,
                 float out_qscale, int *err, cudaStream_t st) {
    constexpr int kStageB = BN * 128;
    const int KB = K / (FP8 ? 128 : 64);
    const int budget = 225 * 1024;  // dynamic smem we allow ourselves (227 KB max per CTA)
    const int fixed = 1024 + 256;   // alignment slack + barriers
    int stages;
    if (FIRST) stages = (budget - fixed - KB * kStageA) / kStageB;
    else stages = (budget - fixed) / (kStageA + kStageB);
    if (stages > 4) stages = 4;
    if (stages < 1) return fail(CBDFS_EINVAL, "layer K=%d too wide for shared memory", K);
    const int a_bytes = FIRST ? KB * kStageA : stages * kStageA;
    const size_t smem = fixed + a_bytes + (size_t)stages * kStageB;
    auto kern = k_tc_layer<BN, FIRST, DOMAIN, FP8, OUT_FP8>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(N / BN, rows_pad / kBM);
    kern<<<grid, kThreads, smem, st>>>(tmA, tmB, states, n, K, N, bias, out, acc_scale, out_qscale,
                                       stages, err);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

struct LayerArgs {
    const CUtensorMap *tmA, *tmB;
    const uint64_t *states;
    uint32_t n, rows_pad;
    int K, N;
    const float *bias;
    void *out;
    float acc_scale, out_qscale;
    int *err;
    cudaStream_t st;
};

template <bool F, int D, bool P, bool O>
int go(int bn, const LayerArgs &a) {
    if (bn == 256)
        return launch_layer<256, F, D, P, O>(*a.tmA, *a.tmB, a.states, a.n, a.rows_pad, a.K, a.N,
                                             a.bias, a.out, a.acc_scale, a.out_qscale, a.err, a.st);
    return launch_layer<128, F, D, P, O>(*a.tmA, *a.tmB, a.states, a.n, a.rows_pad, a.K, a.N,
                                         a.bias, a.out, a.acc_scale, a.out_qscale, a.err, a.st);
}

template <bool F, int D>
int go_prec(bool fp8, bool out_fp8, int bn, const LayerArgs &a) {
    if (!fp8) return go<F, D, false, false>(bn, a);
    return out_fp8 ? go<F, D, true, true>(bn, a) : go<F, D, true, false>(bn, a);
}

}  // namespace

// Dispatch one tensor-core layer.  `first` builds A from `states` (of `domain`); otherwise
// A comes from tmA.  The output is BF16, or E4M3 (scaled by out_qscale) when out_fp8.
int tc_layer(bool first, int domain, bool fp8, bool out_fp8, int bn, const CUtensorMap &tmA,
             const CUtensorMap &tmB, const uint64_t *states, uint32_t n, uint32_t rows_pad, int K,
             int N, const float *bias, void *out, float acc_scale, float out_qscale, int *err,
             cudaStream_t st) {
    if (bn != 128 && bn != 256) return fail(CBDFS_EINVAL, "tile width %d", bn);
    LayerArgs a{&tmA, &tmB, states, n, rows_pad, K, N, bias, out, acc_scale, out_qscale, err, st};
    if (!first) return go_prec<false, 0>(fp8, out_fp8, bn, a);
    switch (domain) {
    case CBDFS_DOM_STP3: return go_prec<true, CBDFS_DOM_STP3>(fp8, out_fp8, bn, a);
    case CBDFS_DOM_STP4: return go_prec<true, CBDFS_DOM_STP4>(fp8, out_fp8, bn, a);
    default: return go_prec<true, CBDFS_DOM_RC3>(fp8, out_fp8, bn, a);
    }
}

}  // namespace cbdfs
