// mlp_chain.cu -- the whole network heuristic in one persistent launch.
//
// Every hidden layer is cut into 128-state x 256-output tiles; the tiles of all layers form
// one sequence, layer by layer and, inside a layer, row block by row block.  Each CTA (one
// per SM, all resident: a cooperative launch, of single CTAs or of CTA pairs) takes tiles
// i, i+G, i+2G, ... (CTA pairs: pair tiles, see k_chain).  A tile
// of layer l+1 for row block m starts as soon as every tile of layer l for that row block is
// stored: the epilogue counts finished tiles per (layer, row block) with a release atomic and
// the producer waits for the count with a bounded acquire poll.  Dependencies only point to
// earlier tiles of the sequence, and all CTAs are resident, so the earliest unfinished tile
// can always proceed.  Activations of a row block stay in L2 between layers.
//
// Before the tiles, every warp of the grid decodes packed states into the one-hot input rows
// (units of 16 or 8 rows, about 8 KB each, one coalesced state load per unit, 16-byte
// coalesced stores, every chunk computed branch-free) and counts finished units per row
// block, so that layer 0 waits only for its own 128 rows.  The launch leaves every count zero
// for the next one: a count is zeroed once nothing reads it any more (by the next layer's
// producer, the row block's head finisher, or a stored last layer's final warp).
//
// Per CTA (192 threads):
//   warp 0      producer: TMA loads the A k-block (the one-hot rows for layer 0, the stored
//               activations of layer l-1 otherwise) and the weight k-block into a 4-stage
//               ring, once the rows it reads are published
//   warp 1      owns 512 TMEM columns (two 256-column FP32 accumulators); one lane issues
//               tcgen05.mma and commits stages back to the producer and finished
//               accumulators to the epilogue, so one tile's epilogue overlaps the next main loop
//   warps 2..5  epilogue: bias + ReLU + BF16 (or scaled E4M3) store of the activation tile,
//               or, for the last hidden layer, the FP32 last layer as per-tile partial dot
//               products; the CTA that stores the last partial of a row block adds the
//               partials in tile order (deterministic), applies the integer-h rule (rint or
//               argmax, max with Manhattan distance, goal = 0) and the bound test (mask bits
//               by ballot, least f above the bound by warp minimum + atomicMin).
// Every wait is bounded (ChainParams::wait_ns of %globaltimer, 2 s unless the context sets
// another bound) and reports through the error flag.
#include <cuda_fp8.h>

#include <cstdlib>

#include <map>
#include <mutex>
#include <set>

#include "chain.h"

namespace cbdfs {

namespace {

using namespace dev;

constexpr int kStageA = kBM * 128;
constexpr int kStagingWarp = 2 * 32 * 64;   // two 32-row x 64-byte boxes per epilogue warp
constexpr int kStaging = 4 * kStagingWarp;
constexpr int kBiasSmem = 2 * kChainBN * 4;  // the tile's biases, double-buffered

__device__ __forceinline__ uint32_t ld_acquire(const int *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// count += v with release semantics at GPU scope (this thread's prior writes become visible first)
__device__ __forceinline__ void red_release_add(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void epi_bar() {  // the 128 epilogue threads
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// bounded wait until *p >= want (acquire)
__device__ __forceinline__ bool wait_count(const int *p, int want, int *err, unsigned long long limit_ns) {
    if ((int)ld_acquire(p) >= want) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1; i < (1u << 28); ++i) {
        if ((int)ld_acquire(p) >= want) return true;
        __nanosleep(64);
        if ((i & 63) == 0) {
            if (*reinterpret_cast<volatile int *>(err) != 0) return false;
            if (globaltimer() - t0 > limit_ns) break;
        }
    }
    atomicCAS(err, 0, DEVERR_DEPENDENCY);
    return false;
}

__device__ __forceinline__ void stamp(const ChainParams &P, uint32_t i, int k) {
    if (P.trace && (int)i < P.trace_tiles)
        P.trace[((size_t)blockIdx.x * P.trace_tiles + i) * 8 + k] = globaltimer();
}

struct Tile {
    int l, m, n;
};
// tile t of the sequence as this CTA sees it: with CTA pairs, the sequence counts pair tiles
// (two row blocks, 2p and 2p+1) and the CTA of rank r works on row block 2p + r
template <bool PAIR>
__device__ __forceinline__ Tile tile_of(const ChainParams &P, int t, uint32_t rank) {
    int l = 0;
    while (l + 1 < P.nh && t >= P.tile_start[l + 1]) ++l;
    const int local = t - P.tile_start[l];
    const int m = local / P.nt[l];
    return Tile{l, PAIR ? 2 * m + (int)rank : m, local % P.nt[l]};
}

// The one-hot encoding (the network's input): slot j of the state (STP: tile j, whose value
// is its cell; cube: cubie j, corners then edges, whose value is pos*k + ori in 0..23) sets
// element j * W + value, W = cells (STP) or 24 (cube).
template <int DOMAIN>
struct OneHot {
    static constexpr int W = DOMAIN == CBDFS_DOM_RC3 ? 24 : (DOMAIN == CBDFS_DOM_STP3 ? 9 : 16);
    static constexpr int slots = DOMAIN == CBDFS_DOM_RC3 ? 20 : W;
    // the per-row words: STP the inverse permutation (nibble j = cell of tile j), cube the
    // two packed words
    __device__ __forceinline__ static void prepare(uint64_t s0, uint64_t s1, uint64_t &a, uint64_t &b) {
        if (DOMAIN == CBDFS_DOM_RC3) {
            a = s0;
            b = s1;
        } else {
            uint64_t where = 0;
#pragma unroll
            for (int p = 0; p < W; ++p) where |= (uint64_t)p << (4 * ((s0 >> (4 * p)) & 15u));
            a = where;
            b = 0;
        }
    }
    // the value of slot j (0 for j >= slots, where no shift may reach 64 bits)
    __device__ __forceinline__ static int value(uint64_t a, uint64_t b, int j) {
        if (DOMAIN == CBDFS_DOM_RC3)
            return j < 8 ? (int)((a >> (5 * j)) & 31u) : j < 20 ? (int)((b >> (5 * (j - 8))) & 31u) : 0;
        return j < 16 ? (int)((a >> (4 * j)) & 15u) : 0;
    }
};

// 16-byte chunk k of a row's one-hot encoding (elements k*E .. k*E+E-1, E = 8 BF16 or 16
// E4M3): the ones of the slots whose columns the chunk covers.  Branch-free: a lane-dependent
// branch per chunk would cost a reconvergence each.
template <int DOMAIN, bool FP8>
__device__ __forceinline__ uint4 onehot_chunk(uint64_t a, uint64_t b, bool live, int k) {
    using OH = OneHot<DOMAIN>;
    constexpr int E = FP8 ? 16 : 8;
    constexpr int NS = OH::W % E == 0 ? 1 : (E + OH::W - 1) / OH::W + 1;  // slots a chunk can meet
    constexpr uint32_t ONE = FP8 ? 0x38u : 0x3F80u;                       // E4M3 / BF16 1.0
    const int e0 = k * E;
    const int s0 = e0 / OH::W;
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) {
        const int sl = s0 + kk;
        const int e = sl * OH::W + OH::value(a, b, sl) - e0;
        const bool in = live && sl < OH::slots && (unsigned)e < (unsigned)E;
        const int wi = FP8 ? (e >> 2) : (e >> 1);
        const uint32_t bits = in ? (FP8 ? (ONE << (8 * (e & 3))) : (ONE << (16 * (e & 1)))) : 0u;
        w0 |= wi == 0 ? bits : 0u;
        w1 |= wi == 1 ? bits : 0u;
        w2 |= wi == 2 ? bits : 0u;
        w3 |= wi == 3 ? bits : 0u;
    }
    return make_uint4(w0, w1, w2, w3);
}

template <int DOMAIN, int CMAX>
__device__ __forceinline__ void finish_row(const ChainParams &P, uint32_t row_g, const float (&yv)[CMAX],
                                           bool valid, int lane, int wq, int m) {
    uint32_t f = 0xFFFFFFFFu;
    bool pass = false;
    if (valid) {
        bool goal;
        int md = -1;
        if (DOMAIN == CBDFS_DOM_RC3) {
            const ulonglong2 w = reinterpret_cast<const ulonglong2 *>(P.states)[row_g];
            goal = rc_is_goal(w.x, w.y);
        } else {
            constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
            const uint64_t s = P.states[row_g];
            if (P.max_with_md) md = manhattan<SIDE>(s);
            goal = stp_is_goal<SIDE>(s);
        }
        if (P.head_kind == CBDFS_HEAD_REAL) {
            const float hr = real_h(yv[0], P.head_param, md, goal);
            if (P.h) P.h[row_g] = real_h_u8(hr);
            if (P.y) P.y[row_g] = hr;
            f = real_f_key(P.g[row_g], hr);
        } else {
            int hv;
            if (P.head_kind == CBDFS_HEAD_REGRESSION) {
                hv = (int)fminf(fmaxf(rintf(yv[0]), 0.f), 255.f);
            } else if (P.head_kind == CBDFS_HEAD_QUANTILE) {
                // quantile_class's arithmetic, in the same order, over the register array
                float mx = yv[0];
#pragma unroll
                for (int c = 1; c < CMAX; ++c)
                    if (c < P.C) mx = fmaxf(mx, yv[c]);
                float S = 0.f;
#pragma unroll
                for (int c = 0; c < CMAX; ++c)
                    if (c < P.C) S += expf(yv[c] - mx);
                const float T = P.head_param * S;
                float acc = 0.f;
                bool hit = false;
                hv = P.C - 1;
#pragma unroll
                for (int c = 0; c < CMAX; ++c)
                    if (c < P.C && !hit) {
                        acc += expf(yv[c] - mx);
                        if (acc >= T) { hv = c; hit = true; }
                    }
            } else {
                int best = 0;
                float bv = yv[0];
#pragma unroll
                for (int c = 1; c < CMAX; ++c)
                    if (c < P.C && yv[c] > bv) { bv = yv[c]; best = c; }
                hv = best;
            }
            hv = goal ? 0 : min(max(hv, md), 255);
            P.h[row_g] = (uint8_t)hv;
            f = (uint32_t)P.g[row_g] + (uint32_t)hv;
            if (P.y)
#pragma unroll
                for (int c = 0; c < CMAX; ++c)
                    if (c < P.C) P.y[(size_t)row_g * P.C + c] = yv[c];
        }
        pass = f <= P.bound;
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
    const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
    const uint32_t word = (uint32_t)m * 4 + wq;
    if (lane == 0 && word < (P.n + 31) / 32) {
        P.mask[word] = bits;
        if (mn != 0xFFFFFFFFu) atomicMin(P.minf, mn);
    }
}

// BN: outputs of a tile (one TMEM accumulator); STAGES: depth of the (A, B) k-block ring.
// PAIR: a cluster of two CTAs computes each 256-row x BN tile with tcgen05 cta_group::2 MMAs
// issued by the even CTA; each CTA loads its own 128 rows of A and half of the BN weight rows,
// so a k-block stage is 32 KB per SM instead of 48 KB and the ring holds more stages.
template <int DOMAIN, bool FP8, int CMAX, int BN, int STAGES, bool PAIR>
__global__ void __launch_bounds__(kChainThreads, 1)
k_chain(const __grid_constant__ ChainMaps maps, const __grid_constant__ ChainParams P) {
    constexpr int kStageB = (PAIR ? BN / 2 : BN) * 128;
    constexpr int HS = BN < 128 ? BN : 128;  // columns of a last-layer slice in shared memory
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *A = smem;
    uint8_t *B = smem + STAGES * kStageA;
    uint8_t *stg = B + STAGES * kStageB;  // epilogue staging: 4 warps x 2 x 2 KB
    float *bsm = reinterpret_cast<float *>(stg + kStaging);  // [2][256] tile biases
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + kStaging + kBiasSmem);
    uint64_t *full = bars, *empty = bars + STAGES;
    uint64_t *acc_full = bars + 2 * STAGES, *acc_empty = acc_full + 2;
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    int *flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = P.tile_start[P.nh];
    const uint32_t rank = PAIR ? cluster_ctarank() : 0;
    const bool leader = rank == 0;
    const int t0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;    // this CTA's first tile
    const int tstride = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    // stage and accumulator waits wait on work that itself waits on row-block counts: their
    // bound is twice the count wait's, so that a count that never comes is the wait that runs
    // out first and names the cause
    const unsigned long long stage_ns = 2 * P.wait_ns;
    const int last_l = P.fused_head ? P.nh - 1 : P.nh;  // the layer whose epilogue runs the head

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), PAIR ? 8 : 4);  // the epilogue warps of both CTAs
        }
        mbar_init(smem_u32(drain), 1);
        fence_mbar_init();
        if (PAIR) fence_mbar_init_cluster();
    }
    if (warp == 0 && lane == 0) {
        for (int l = 0; l < P.nh; ++l) {
            tma_prefetch_map(&maps.w[l]);
            tma_prefetch_map(&maps.a[l]);
        }
    }
    if (warp == 1) {
        if (PAIR) {
            tmem_alloc_pair(smem_u32(tmem_slot), 2 * BN);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(smem_u32(tmem_slot), 2 * BN);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync_all();  // the peer's barriers are initialised before any signal
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr int KBLK = FP8 ? 128 : 64;

    {
        // one-hot pre-pass by every warp of the grid: unit v = rows [R v, R v + R) goes to warp
        // v mod (warps in the grid), R = P.unit_rows (16 for one-hot rows of up to 512 bytes,
        // else 8: about 8 KB per unit); a row block counts its kBM / R units.  The next unit's
        // states are loaded while this one is written and published.
        constexpr int EB = FP8 ? 1 : 2;
        constexpr int nwarps = kChainThreads / 32;
        const int R = P.unit_rows;
        const int units = P.mblocks * (kBM / R);
        const int nchunk = P.kdim[0] * EB / 16;
        const int vstride = gridDim.x * nwarps;
        uint64_t n0 = 0, n1 = 0;
        bool nlv = false;
        auto load_unit = [&](int v) {
            const uint32_t my = v * R + (lane & (R - 1));
            n0 = n1 = 0;
            nlv = lane < R && my < P.n;
            if (nlv) {
                if (DOMAIN == CBDFS_DOM_RC3) {
                    const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(P.states) + my);
                    n0 = w.x;
                    n1 = w.y;
                } else {
                    n0 = __ldg(P.states + my);
                }
            }
        };
        if (blockIdx.x * nwarps + warp < units) load_unit(blockIdx.x * nwarps + warp);
        for (int v = blockIdx.x * nwarps + warp; v < units; v += vstride) {
            const uint64_t s0 = n0, s1 = n1;
            const bool lv = nlv;
            if (v + vstride < units) load_unit(v + vstride);
            uint64_t wa, wb;
            OneHot<DOMAIN>::prepare(s0, s1, wa, wb);
            // eight rows at a time, unrolled, so that their shuffles and stores overlap; a lane
            // writes chunks lane and lane + 32 of each row (rows of up to 1 KB; wider rows go on
            // in the loop after)
#pragma unroll 1
            for (int r0 = 0; r0 < R; r0 += 8) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int r = r0 + j;
                    const uint64_t ar = __shfl_sync(0xFFFFFFFFu, wa, r);
                    const uint64_t br = DOMAIN == CBDFS_DOM_RC3 ? __shfl_sync(0xFFFFFFFFu, wb, r) : 0ull;
                    const bool lr = __shfl_sync(0xFFFFFFFFu, lv, r);
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(P.onehot) +
                                                           (size_t)(v * R + r) * P.kdim[0] * EB);
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        if (lane + 32 * q < nchunk) dst[lane + 32 * q] = onehot_chunk<DOMAIN, FP8>(ar, br, lr, lane + 32 * q);
                    for (int k = lane + 64; k < nchunk; k += 32) dst[k] = onehot_chunk<DOMAIN, FP8>(ar, br, lr, k);
                }
            }
            fence_proxy_async_global();  // the rows are read by TMA (the async proxy)
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(P.counters + v / (kBM / R), 1);
        }
    }

    if (warp == 0) {
        // ------------------------------------------------------------- producer
        uint32_t it = 0, pi = 0;
        bool ok = true;
        for (int t = t0; t < total && ok; t += tstride, ++pi) {
            const Tile T = tile_of<PAIR>(P, t, rank);
            const int KB = P.kdim[T.l] / KBLK;
            const int kb0 = P.group_nt[T.l] ? (T.n / P.group_nt[T.l]) * KB : 0;  // member's K block
            if (lane == 0) stamp(P, pi, 0);
            // layer 0 reads the one-hot rows (kBM / R units), layer l the stored tiles of
            // layer l-1 (4 warps per tile)
            const int *cnt = P.counters + T.l * P.mblocks + T.m;
            const int want = T.l == 0 ? kBM / P.unit_rows : 4 * P.nt[T.l - 1];
            if (lane == 0) ok = wait_count(cnt, want, P.err, P.wait_ns);
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) break;
            fence_proxy_async_global();
            // this layer's inputs are complete, so every tile of the previous layer in this row
            // block has read its own input count: that count is left zero for the next launch
            if (lane == 0 && T.l > 0) P.counters[(T.l - 1) * P.mblocks + T.m] = 0;
            if (lane == 0) stamp(P, pi, 1);
            for (int kb = 0; kb < KB; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t u = it / STAGES;
                if (it >= STAGES) {
                    bool w = true;
                    if (lane == 0) w = mbar_wait(smem_u32(&empty[s]), (u - 1) & 1, P.err, DEVERR_STAGE_EMPTY, stage_ns);
                    w = __shfl_sync(0xFFFFFFFFu, w, 0);
                    if (!w) { ok = false; break; }
                }
                if (lane == 0) {
                    if (PAIR) {
                        // both CTAs' loads count on the leader's stage barrier, which the leader
                        // arms for the pair's bytes; each CTA loads its rows and its half of B
                        const uint32_t fb = mapa_shared(smem_u32(&full[s]), 0);
                        if (leader) mbar_arrive_expect_tx(smem_u32(&full[s]), 2 * (kStageA + kStageB));
                        tma_load_2d_pair(smem_u32(A + s * kStageA), &maps.a[T.l], fb, (kb + kb0) * KBLK, T.m * kBM);
                        tma_load_2d_pair(smem_u32(B + s * kStageB), &maps.w[T.l], fb, kb * KBLK,
                                         T.n * BN + (int)rank * (BN / 2));
                    } else {
                        mbar_arrive_expect_tx(smem_u32(&full[s]), kStageA + kStageB);
                        tma_load_2d(smem_u32(A + s * kStageA), &maps.a[T.l], smem_u32(&full[s]), (kb + kb0) * KBLK,
                                    T.m * kBM);
                        tma_load_2d(smem_u32(B + s * kStageB), &maps.w[T.l], smem_u32(&full[s]), kb * KBLK,
                                    T.n * BN);
                    }
                }
                __syncwarp();
            }
            if (lane == 0) stamp(P, pi, 2);
        }
        // every TMA load this CTA issued has landed before the CTA can exit (bounded); with
        // pairs the leader's barriers count both CTAs' loads, and the peer's loads have all been
        // consumed by the leader's MMAs unless a wait ran out (see the end of the kernel)
        if (lane == 0 && leader) {
            const uint32_t first = it > STAGES ? it - STAGES : 0;
            for (uint32_t j = first; j < it; ++j)
                mbar_wait_drain(smem_u32(&full[j % STAGES]), (j / STAGES) & 1, P.err, DEVERR_TMA_FULL, 100000000ull);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0 && leader) {
            constexpr int MM = PAIR ? 2 * kBM : kBM;  // the pair's MMA covers both CTAs' rows
            constexpr uint32_t idesc = FP8 ? make_idesc(MM, BN, 0, 0) : make_idesc(MM, BN, 1, 1);
            uint32_t it = 0, i = 0;
            bool ok = true;
            for (int t = t0; t < total && ok; t += tstride, ++i) {
                const Tile T = tile_of<PAIR>(P, t, rank);
                const int KB = P.kdim[T.l] / KBLK;
                const uint32_t b = i & 1, u = i >> 1;
                if (i >= 2 && !mbar_wait(smem_u32(&acc_empty[b]), (u - 1) & 1, P.err, DEVERR_ACCUM, stage_ns)) break;
                tc_fence_after();
                stamp(P, i, 3);
                const uint32_t d = tmem + b * BN;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(smem_u32(&full[s]), (it / STAGES) & 1, P.err, DEVERR_TMA_FULL, stage_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = sw128_desc(smem_u32(A + s * kStageA));
                    const uint64_t bd = sw128_desc(smem_u32(B + s * kStageB));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (PAIR) {
                            if (FP8) umma_fp8_pair(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                            else umma_bf16_pair(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                        } else {
                            if (FP8) umma_fp8(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                            else umma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                        }
                    }
                    if (PAIR) umma_commit_pair(smem_u32(&empty[s]));  // both CTAs' stage is free
                    else umma_commit(smem_u32(&empty[s]));
                }
                if (ok) {
                    if (PAIR) umma_commit_pair(smem_u32(&acc_full[b]));
                    else umma_commit(smem_u32(&acc_full[b]));
                }
                stamp(P, i, 4);
            }
            // all MMAs this thread issued have completed before TMEM is released (bounded); the
            // pair's drain arrives in both CTAs
            if (PAIR) umma_commit_pair(smem_u32(drain));
            else umma_commit(smem_u32(drain));
            mbar_wait_drain(smem_u32(drain), 0, P.err, DEVERR_ACCUM, 100000000ull);
        } else if (PAIR && lane == 0) {
            // the peer's TMEM is written by the leader's MMAs: wait for the leader's drain, which
            // comes after the leader's whole tile loop
            mbar_wait_drain(smem_u32(drain), 0, P.err, DEVERR_ACCUM, stage_ns + 100000000ull);
        }
    } else {
        // ------------------------------------------------------------- epilogue
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int ep_tid = threadIdx.x - 64;
        uint32_t i = 0;
        // an accumulator is released to the (leader's) MMA issuer once this warp has read it
        auto release_acc = [&](uint32_t b) {
            if (PAIR && !leader) mbar_arrive_cluster(mapa_shared(smem_u32(&acc_empty[b]), 0));
            else mbar_arrive(smem_u32(&acc_empty[b]));
        };
        for (int t = t0; t < total; t += tstride, ++i) {
            const Tile T = tile_of<PAIR>(P, t, rank);
            const uint32_t b = i & 1, u = i >> 1;
            // the tile's biases into shared memory while the MMAs run (buffer i & 1 was last
            // read two tiles ago, before everyone passed the previous tile's barrier)
            float *bt = bsm + (i & 1) * kChainBN;
            for (int j = ep_tid; j < BN; j += 128) bt[j] = __ldg(P.bias[T.l] + T.n * BN + j);
            epi_bar();
            // after a failed wait the warps skip the work but keep every barrier, so that
            // the four epilogue warps stay in step
            const bool good = mbar_wait(smem_u32(&acc_full[b]), u & 1, P.err, DEVERR_ACCUM, stage_ns);
            tc_fence_after();
            if (ep_tid == 0) stamp(P, i, 5);
            const uint32_t taddr = tmem + b * BN + ((uint32_t)(q * 32) << 16);
            const uint32_t rg = T.m * kBM + row;
            const int n0 = T.n * BN;
            const float *bias = bt;  // shared memory
            const float sc = P.acc_scale[T.l];
            if (T.l < last_l) {
                const bool out8 = FP8 && T.l != P.bf16_store_layer;  // E4M3 unless the BF16 head reads it
                const float oq = P.out_qscale[T.l];
                uint8_t *wstg = stg + q * kStagingWarp;
#pragma unroll 1
                for (int c2 = 0; c2 < BN / 32 && good; c2 += 2) {
                    uint32_t ra[2][32];
                    tmem_ld32(taddr + c2 * 32, ra[0]);
                    tmem_ld32(taddr + (c2 + 1) * 32, ra[1]);
                    tmem_ld_wait();
#pragma unroll
                    for (int hb = 0; hb < 2; ++hb) {
                        const int c = c2 + hb;
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            const float4 bb = *reinterpret_cast<const float4 *>(bias + c * 32 + j);
                            v[j + 0] = fmaxf(fmaf(__uint_as_float(ra[hb][j + 0]), sc, bb.x), 0.f);
                            v[j + 1] = fmaxf(fmaf(__uint_as_float(ra[hb][j + 1]), sc, bb.y), 0.f);
                            v[j + 2] = fmaxf(fmaf(__uint_as_float(ra[hb][j + 2]), sc, bb.z), 0.f);
                            v[j + 3] = fmaxf(fmaf(__uint_as_float(ra[hb][j + 3]), sc, bb.w), 0.f);
                        }
                        uint8_t *sb = wstg + hb * (32 * 64);
                        // both boxes of the previous pair must have been read out
                        if (hb == 0 && c >= 2) {
                            if (lane == 0) bulk_wait_read<0>();
                            __syncwarp();
                        }
                        if (out8) {
                            uint32_t pk[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                __nv_fp8x4_e4m3 q4(make_float4(v[4 * j] * oq, v[4 * j + 1] * oq, v[4 * j + 2] * oq,
                                                               v[4 * j + 3] * oq));
                                pk[j] = *reinterpret_cast<uint32_t *>(&q4);
                            }
                            // 32-byte row, 32-byte swizzle: chunk k of row r at k ^ ((r >> 2) & 1)
                            uint8_t *rowp = sb + lane * 32;
                            const int sw = (lane >> 2) & 1;
                            *reinterpret_cast<uint4 *>(rowp + ((0 ^ sw) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                            *reinterpret_cast<uint4 *>(rowp + ((1 ^ sw) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        } else {
                            uint32_t pk[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                                pk[j] = *reinterpret_cast<uint32_t *>(&h2);
                            }
                            // 64-byte row, 64-byte swizzle: chunk k of row r at k ^ ((r >> 1) & 3)
                            uint8_t *rowp = sb + lane * 64;
                            const int sw = (lane >> 1) & 3;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                *reinterpret_cast<uint4 *>(rowp + ((k ^ sw) << 4)) =
                                    make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
                        }
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&maps.o[T.l], smem_u32(wstg), n0 + c2 * 32, T.m * kBM + q * 32);
                        tma_store_2d(&maps.o[T.l], smem_u32(wstg + 32 * 64), n0 + (c2 + 1) * 32,
                                     T.m * kBM + q * 32);
                        bulk_commit();
                    }
                }
                if (ep_tid == 0) stamp(P, i, 7);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    release_acc(b);
                    // publish this warp's 32 rows: stores complete, then the count (4 per tile)
                    bulk_wait_all();
                    fence_proxy_async_global();
                    int *oc = P.counters + (1 + T.l) * P.mblocks + T.m;
                    if (good && T.l + 1 < P.nh) {
                        if (!(T.l == 0 && T.m == P.hold_mblock)) red_release_add(oc, 1);
                    } else if (good && atomicAdd(oc, 1) == 4 * P.nt[T.l] - 1) {
                        // the last hidden layer, stored for a separate head kernel: the row block's
                        // last warp leaves its own count and the layer's input count zero
                        atomicExch(oc, 0);
                        atomicExch(P.counters + T.l * P.mblocks + T.m, 0);
                    }
                }
                __syncwarp();
            } else {
                // last hidden layer: partial dot products with the FP32 last layer
                float acc[CMAX];
#pragma unroll
                for (int c = 0; c < CMAX; ++c) acc[c] = 0.f;
                const int K = P.dims[T.l + 1];
                float *wsm = reinterpret_cast<float *>(stg);  // [C][HS] slice of the last layer
#pragma unroll 1
                for (int half = 0; half < BN / HS; ++half) {
                    epi_bar();  // the previous slice has been read
#pragma unroll 8
                    for (int idx = ep_tid; idx < P.C * HS; idx += 128)
                        wsm[idx] = __ldg(P.w_last + (size_t)(idx / HS) * K + n0 + half * HS + idx % HS);
                    epi_bar();
#pragma unroll 1
                    for (int c = half * (HS / 32); c < (half + 1) * (HS / 32) && good; ++c) {
                        uint32_t r[32];
                        tmem_ld32(taddr + c * 32, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float v[4];
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj)
                                v[jj] = fmaxf(fmaf(__uint_as_float(r[j + jj]), sc, bias[c * 32 + j + jj]), 0.f);
                            const float *wj = wsm + (c - half * (HS / 32)) * 32 + j;
#pragma unroll
                            for (int o = 0; o < CMAX; ++o) {
                                if (o < P.C) {  // predicated: the loop stays unrolled, acc in registers
                                    const float4 w4 = *reinterpret_cast<const float4 *>(wj + o * HS);
                                    acc[o] = fmaf(v[0], w4.x, fmaf(v[1], w4.y, fmaf(v[2], w4.z, fmaf(v[3], w4.w, acc[o]))));
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) release_acc(b);
                float *pp = P.partial + ((size_t)T.n * P.rows_pad + rg) * P.C;
#pragma unroll
                for (int o = 0; o < CMAX; ++o)
                    if (o < P.C) pp[o] = acc[o];
                __threadfence();
                epi_bar();
                if (ep_tid == 0) {
                    int *hc = P.counters + (1 + P.nh) * P.mblocks + T.m;
                    const int old = good ? atomicAdd(hc, 1) : -1;
                    *flag = old == P.nt[T.l] - 1;
                    if (*flag) {  // the row block's last partial: its counts are left zero for the next launch
                        atomicExch(hc, 0);
                        atomicExch(P.counters + T.l * P.mblocks + T.m, 0);
                    }
                }
                epi_bar();
                if (*flag) {
                    __threadfence();
                    // y = b + partial[0] + partial[1] + ... in tile order (deterministic); all of a
                    // tile's C loads are issued together
                    float yv[CMAX];
#pragma unroll
                    for (int o = 0; o < CMAX; ++o) yv[o] = o < P.C ? __ldg(P.b_last + o) : 0.f;
                    for (int nt = 0; nt < P.nt[T.l]; ++nt) {
                        const float *pp = P.partial + ((size_t)nt * P.rows_pad + rg) * P.C;
#pragma unroll
                        for (int o = 0; o < CMAX; ++o)
                            if (o < P.C) yv[o] += __ldcg(pp + o);
                    }
                    finish_row<DOMAIN, CMAX>(P, rg, yv, rg < P.n, lane, q, T.m);
                }
                epi_bar();
            }
            if (ep_tid == 0) stamp(P, i, 6);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) {
        // after a wait ran out, loads the peer issued may not have been consumed: give them
        // time to land (they always complete) before the CTA's shared memory goes away
        if (threadIdx.x == 0 && *reinterpret_cast<volatile int *>(P.err) != 0) {
            const uint64_t t_end = globaltimer() + 200000ull;
            while (globaltimer() < t_end) __nanosleep(1000);
        }
        __syncthreads();
        cluster_sync_all();  // neither CTA frees the pair's TMEM while the other still reads it
    }
    if (warp == 1) {
        tc_fence_after();
        if (PAIR) tmem_dealloc_pair(tmem, 2 * BN);
        else tmem_dealloc(tmem, 2 * BN);
    }
    // a programmatic dependent (the separate head kernel) may be scheduled once every CTA has
    // got here; it still waits for this grid's completion before reading what it stored
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace

template <int BN, int STAGES, bool PAIR>
static size_t chain_smem_bytes() {
    return 1024 + STAGES * (kStageA + (PAIR ? BN / 2 : BN) * 128) + kStaging + kBiasSmem + 256;
}

// the kernel's dynamic shared-memory limit, raised once per kernel and device
static int allow_smem(const void *kern, size_t smem) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({kern, dev})) return CBDFS_OK;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done.insert({kern, dev});
    return CBDFS_OK;
}

// Launch the chain for one batch.  P.counters must be zero (they are after the previous
// launch on the same counters, and after allocation).
template <int D, bool F, int BN, int STAGES, bool PAIR>
static int launch_t(const ChainMaps &maps, const ChainParams &P, int grid, cudaStream_t st) {
    const size_t smem = chain_smem_bytes<BN, STAGES, PAIR>();
    void (*kern)(const ChainMaps, const ChainParams) =
        P.C == 1 || !P.fused_head ? k_chain<D, F, 1, BN, STAGES, PAIR>
        : P.C <= 24              ? k_chain<D, F, 24, BN, STAGES, PAIR>
                                 : k_chain<D, F, kMaxHeadC, BN, STAGES, PAIR>;
    if (int rc = allow_smem(reinterpret_cast<const void *>(kern), smem)) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kChainThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // one CTA per SM, all resident at once: a cooperative launch (CTA pairs: with a cluster
    // dimension of 2; chain_pairs_fit has checked that the device holds every pair).  A plain
    // cluster launch can start only some of its pairs while other work holds SMs; its CTAs
    // then wait on tiles of pairs not yet started, and a full-device cooperative launch queued
    // on another stream waits for those SMs: neither proceeds until the bounded waits run out.
    // CBDFS_PLAIN_CLUSTER_LAUNCH=1 (read once) launches pairs without the cooperative attribute
    // for profilers that cannot replay a cooperative cluster launch; only for runs with one
    // launch in flight at a time
    static const bool plain_pairs = [] {
        const char *v = getenv("CBDFS_PLAIN_CLUSTER_LAUNCH");
        return v && v[0] == '1';
    }();
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (PAIR) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = 2;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (!PAIR || !plain_pairs) {
        attr[na].id = cudaLaunchAttributeCooperative;
        attr[na].val.cooperative = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, P);
    if (e != cudaSuccess) return fail(CBDFS_EDEVICE, "chain launch: %s", cudaGetErrorString(e));
    return CBDFS_OK;
}

template <int BN, int STAGES, bool PAIR>
static int launch_bn(int domain, bool fp8, const ChainMaps &maps, const ChainParams &P, int grid, cudaStream_t st) {
    if (fp8) {
        if (domain == CBDFS_DOM_STP3) return launch_t<CBDFS_DOM_STP3, true, BN, STAGES, PAIR>(maps, P, grid, st);
        if (domain == CBDFS_DOM_STP4) return launch_t<CBDFS_DOM_STP4, true, BN, STAGES, PAIR>(maps, P, grid, st);
        return launch_t<CBDFS_DOM_RC3, true, BN, STAGES, PAIR>(maps, P, grid, st);
    }
    if (domain == CBDFS_DOM_STP3) return launch_t<CBDFS_DOM_STP3, false, BN, STAGES, PAIR>(maps, P, grid, st);
    if (domain == CBDFS_DOM_STP4) return launch_t<CBDFS_DOM_STP4, false, BN, STAGES, PAIR>(maps, P, grid, st);
    return launch_t<CBDFS_DOM_RC3, false, BN, STAGES, PAIR>(maps, P, grid, st);
}

int chain_launch(int domain, bool fp8, int bn, bool pair, const ChainMaps &maps, const ChainParams &P, int grid,
                 cudaStream_t st) {
    if (P.fused_head && (P.C < 1 || P.C > kMaxHeadC)) return fail(CBDFS_EINVAL, "fused head width %d", P.C);
    if (pair) {
        if (bn != kChainBN || (grid & 1) || (P.mblocks & 1)) return fail(CBDFS_EINVAL, "CTA-pair chain shape");
        return launch_bn<kChainBN, kChainPairStages, true>(domain, fp8, maps, P, grid, st);
    }
    if (bn == kChainBNSmall) return launch_bn<kChainBNSmall, 8, false>(domain, fp8, maps, P, grid, st);
    if (bn == kChainBN) return launch_bn<kChainBN, kChainStages, false>(domain, fp8, maps, P, grid, st);
    return fail(CBDFS_EINVAL, "chain tile width %d", bn);
}

// whether this device can hold every CTA pair of a one-CTA-per-SM chain launch at once
bool chain_pairs_fit(int num_sms) {
    static std::mutex mu;
    static std::map<int, bool> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find(dev);
    if (it != known.end()) return it->second;
    void (*kern)(const ChainMaps, const ChainParams) = k_chain<CBDFS_DOM_STP4, false, 1, kChainBN, kChainPairStages, true>;
    const size_t smem = chain_smem_bytes<kChainBN, kChainPairStages, true>();
    bool ok = allow_smem(reinterpret_cast<const void *>(kern), smem) == CBDFS_OK;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(num_sms & ~1);
        cfg.blockDim = dim3(kChainThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= num_sms / 2;
        cudaGetLastError();
    }
    known[dev] = ok;
    return ok;
}

}  // namespace cbdfs
