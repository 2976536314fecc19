// head_tc.cu -- the last layer of a classifier network on the tensor cores (17..128 outputs),
// after the fused chain has stored the last hidden layer in BF16.
//
// Y[128 rows][C] = A[128][K] W^T + b.  W (FP32, the last layer) is split on the host into three
// BF16 parts, W = W1 + W2 + W3 to 24 bits of mantissa (each part the BF16 rounding of what the
// previous parts leave), stacked as [3][cpad][K].  Every k-block issues the three tcgen05 MMAs
// (A x W1, A x W2, A x W3) into one FP32 TMEM accumulator: each BF16 x BF16 product is exact,
// so FP32 accumulation is the only rounding, as in an FP32 GEMM.  (Paper, Experimental Setup:
// the classifier heuristic h_M; Background, Heuristics: classes are h values.)
//
// One CTA per 128-row block, 192 threads: warp 0 feeds a 3-stage TMA ring (A: 128 x 64 BF16;
// W: three boxes of cpad x 64), warp 1 issues the MMAs, warps 2-5 run the epilogue: per row the
// logits from TMEM in 32-column chunks, + bias, the head rule (argmax with the lowest index on
// ties; or the quantile, computed in the same order as quantile_class), max with Manhattan
// distance, goal = 0, the bound test (ballot mask word, warp minimum + atomicMin).
#include "chain.h"

namespace cbdfs {

namespace {

using namespace dev;

constexpr int kHtThreads = 192, kHtStages = 3, kHtStageA = kBM * 128;

__device__ __forceinline__ float head_logit(const uint32_t (&r)[32], int j, const float *bsm, int c) {
    return __uint_as_float(r[j]) + bsm[c];
}

template <int DOMAIN>
__global__ void __launch_bounds__(kHtThreads, 1)
k_head_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, const HeadTcParams P,
          uint32_t tmem_cols) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t stageW = 3u * P.cpad * 128u, stage = kHtStageA + stageW;
    float *bsm = reinterpret_cast<float *>(smem + kHtStages * stage);  // [128] biases
    uint64_t *bars = reinterpret_cast<uint64_t *>(bsm + 128);
    uint64_t *full = bars, *empty = bars + kHtStages, *accf = bars + 2 * kHtStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accf + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t m0 = blockIdx.x * kBM;
    const int KB = P.K / 64;
    const int e = blockIdx.y;                 // ensemble member (0 for one network)
    const int ax0 = e * P.K, wy0 = e * 3 * P.cpad;
    const float *b_last = P.b_last + e * P.C;
    uint8_t *h_out = P.h ? P.h + e * P.h_stride : nullptr;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kHtStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accf), 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), tmem_cols);
        tmem_relinquish();
    }
    for (int c = threadIdx.x; c < 128; c += kHtThreads) bsm[c] = c < P.C ? __ldg(b_last + c) : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // launched as a programmatic dependent of the kernel that stores the activations (the fused
    // chain): the set-up above overlaps that kernel's end; nothing it writes is read before
    // here, where the whole grid before this one has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            uint32_t issued = 0;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % kHtStages, u = kb / kHtStages;
                if (kb >= kHtStages && !mbar_wait(smem_u32(&empty[s]), (u - 1) & 1, P.err, DEVERR_STAGE_EMPTY)) break;
                uint8_t *A = smem + s * stage;
                mbar_arrive_expect_tx(smem_u32(&full[s]), stage);
                tma_load_2d(smem_u32(A), &tmA, smem_u32(&full[s]), ax0 + kb * 64, m0);
                for (int sp = 0; sp < 3; ++sp)
                    tma_load_2d(smem_u32(A + kHtStageA + sp * P.cpad * 128), &tmW, smem_u32(&full[s]), kb * 64,
                                wy0 + sp * P.cpad);
                ++issued;
            }
            // every load issued has landed before the CTA can exit (bounded)
            for (uint32_t j = issued > (uint32_t)kHtStages ? issued - kHtStages : 0; j < issued; ++j)
                mbar_wait_drain(smem_u32(&full[j % kHtStages]), (j / kHtStages) & 1, P.err, DEVERR_TMA_FULL, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(kBM, P.cpad, 1, 1);
            bool ok = true;
            for (int kb = 0; kb < KB && ok; ++kb) {
                const int s = kb % kHtStages, u = kb / kHtStages;
                if (!mbar_wait(smem_u32(&full[s]), u & 1, P.err, DEVERR_TMA_FULL)) { ok = false; break; }
                tc_fence_after();
                uint8_t *A = smem + s * stage;
                const uint64_t ad = sw128_desc(smem_u32(A));
                for (int sp = 0; sp < 3; ++sp) {
                    const uint64_t bd = sw128_desc(smem_u32(A + kHtStageA + sp * P.cpad * 128));
#pragma unroll
                    for (int k = 0; k < 4; ++k) umma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | sp | k) != 0);
                }
                umma_commit(smem_u32(&empty[s]));
            }
            umma_commit(smem_u32(accf));
        }
    } else {
        const int q = warp & 3;
        const uint32_t m = m0 + q * 32 + lane;
        const bool valid = m < P.n;
        const bool good = mbar_wait(smem_u32(accf), 0, P.err, DEVERR_ACCUM);
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        const int nch = (P.C + 31) / 32;
        // pass 1: the logits (written out when asked), their argmax and their largest value
        float best = -INFINITY, mx = -INFINITY;
        int bi = 0;
#pragma unroll 1
        for (int ch = 0; ch < nch && good; ++ch) {
            uint32_t r[32];
            tmem_ld32(taddr + ch * 32, r);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = ch * 32 + j;
                if (c < P.C) {
                    const float v = head_logit(r, j, bsm, c);
                    if (P.y && valid && P.groups <= 1) P.y[(size_t)m * P.C + c] = v;
                    if (v > best) { best = v; bi = c; }
                    mx = fmaxf(mx, v);
                }
            }
        }
        int hv = bi;
        if (P.h) {  // (no h: the logits alone, for the training forward)
        if (P.head_kind == CBDFS_HEAD_QUANTILE && good) {
            // the smallest class whose softmax cumulative sum reaches q (quantile_class's order)
            float S = 0.f;
#pragma unroll 1
            for (int ch = 0; ch < nch; ++ch) {
                uint32_t r[32];
                tmem_ld32(taddr + ch * 32, r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (ch * 32 + j < P.C) S += expf(head_logit(r, j, bsm, ch * 32 + j) - mx);
            }
            const float T = P.quantile * S;
            float acc = 0.f;
            hv = P.C - 1;
            bool hit = false;
            // every lane takes every chunk: tcgen05.ld is a warp-collective load
#pragma unroll 1
            for (int ch = 0; ch < nch; ++ch) {
                uint32_t r[32];
                tmem_ld32(taddr + ch * 32, r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = ch * 32 + j;
                    if (c < P.C && !hit) {
                        acc += expf(head_logit(r, j, bsm, c) - mx);
                        if (acc >= T) { hv = c; hit = true; }
                    }
                }
            }
        }
        uint32_t f = 0xFFFFFFFFu;
        bool pass = false;
        if (valid && good) {
            bool goal;
            int md = -1;
            if (DOMAIN == CBDFS_DOM_RC3) {
                goal = rc_is_goal(P.states[2 * m], P.states[2 * m + 1]);
            } else {
                constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
                const uint64_t s = P.states[m];
                if (P.max_with_md) md = manhattan<SIDE>(s);
                goal = stp_is_goal<SIDE>(s);
            }
            hv = goal ? 0 : min(max(hv, md), 255);
            h_out[m] = (uint8_t)hv;
            f = (uint32_t)P.g[m] + (uint32_t)hv;
            pass = f <= P.bound;
        }
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
        const uint32_t word = (m0 >> 5) + q;
        if (lane == 0 && P.groups <= 1 && word < (P.n + 31) / 32) {
            P.mask[word] = bits;
            if (mn != 0xFFFFFFFFu) atomicMin(P.minf, mn);
        }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

template <int DOMAIN>
int launch(const CUtensorMap &tmA, const CUtensorMap &tmW, const HeadTcParams &P, uint32_t rows_pad,
           cudaStream_t st) {
    const size_t smem = 1024 + (size_t)kHtStages * (kHtStageA + 3 * P.cpad * 128) + 128 * 4 + 256;
    CUDA_TRY(cudaFuncSetAttribute(k_head_tc<DOMAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    uint32_t cols = 32;
    while ((int)cols < P.cpad) cols <<= 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(rows_pad / kBM, P.groups > 1 ? P.groups : 1);
    cfg.blockDim = dim3(kHtThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // programmatic dependent launch: the CTAs may start (and set up) while the previous kernel
    // on the stream ends; they wait for it (griddepcontrol.wait) before reading its output
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_head_tc<DOMAIN>, tmA, tmW, P, cols);
    if (e != cudaSuccess) return fail(CBDFS_EDEVICE, "head launch: %s", cudaGetErrorString(e));
    return CBDFS_OK;
}

}  // namespace

int head_tc(int domain, const CUtensorMap &tmA, const CUtensorMap &tmW, const HeadTcParams &P, uint32_t rows_pad,
            cudaStream_t st) {
    if (domain == CBDFS_DOM_STP3) return launch<CBDFS_DOM_STP3>(tmA, tmW, P, rows_pad, st);
    if (domain == CBDFS_DOM_STP4) return launch<CBDFS_DOM_STP4>(tmA, tmW, P, rows_pad, st);
    return launch<CBDFS_DOM_RC3>(tmA, tmW, P, rows_pad, st);
}

}  // namespace cbdfs
