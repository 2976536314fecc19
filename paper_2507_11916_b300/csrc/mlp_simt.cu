// mlp_simt.cu -- the FP32 forms of the network heuristic and the fused head.
//
//   k_first_gather  FP32 first layer as what it is algorithmically: a sum of the weight
//                   columns picked by the one-hot input (16 / 9 / 20 of them), + bias, ReLU.
//   k_sgemm_relu    FP32 hidden layer, C = ReLU(A W^T + b), 128x128 tiles on the CUDA cores.
//   k_head_tiled    the last layer in FP32 fused with the integer-h rule and the bound test
//                   (Algorithm 3's expansion test g + h <= bound; the smallest f above the
//                   bound feeds UpdateThreshold, Algorithm 1), for up to 128 outputs: a block
//                   computes 64 states x all outputs as a register-tiled FP32 GEMM over
//                   k-chunks staged in shared memory.  Reads BF16 or FP32 activations.
//   k_head          the same for wider last layers: one warp per state and output.
#include "common.cuh"

namespace cbdfs {
namespace {

using namespace dev;

// ---- first layer, FP32: W1T is the first layer's weight transposed, [K1][H] ----------
template <int DOMAIN>
__global__ void __launch_bounds__(256)
k_first_gather(const uint64_t *__restrict__ states, uint32_t n, const float *__restrict__ W1T,
               const float *__restrict__ b1, int H, float *__restrict__ out) {
    constexpr int NIDX = DOMAIN == CBDFS_DOM_RC3 ? 20 : (DOMAIN == CBDFS_DOM_STP3 ? 9 : 16);
    __shared__ int idx[8][NIDX];
    const int r0 = blockIdx.x * 8;
    if (threadIdx.x < 8 && r0 + threadIdx.x < n) {
        const uint32_t m = r0 + threadIdx.x;
        if (DOMAIN == CBDFS_DOM_RC3) {
            const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(states) + m);
            for (int c = 0; c < 8; ++c) idx[threadIdx.x][c] = c * 24 + (int)((w.x >> (5 * c)) & 31u);
            for (int e = 0; e < 12; ++e)
                idx[threadIdx.x][8 + e] = 192 + e * 24 + (int)((w.y >> (5 * e)) & 31u);
        } else {
            constexpr int N = DOMAIN == CBDFS_DOM_STP3 ? 9 : 16;
            const uint64_t s = __ldg(states + m);
            for (int p = 0; p < N; ++p) idx[threadIdx.x][p] = (int)((s >> (4 * p)) & 15u) * N + p;
        }
    }
    __syncthreads();
    const int rows = min(8, (int)n - r0);
    for (int r = 0; r < rows; ++r)
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < NIDX; ++i) acc += __ldg(W1T + (size_t)idx[r][i] * H + j);
            out[(size_t)(r0 + r) * H + j] = fmaxf(acc + __ldg(b1 + j), 0.f);
        }
}

// ---- FP32 hidden layer: C[M][N] = ReLU(A[M][K] W[N][K]^T + b) --------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

__global__ void __launch_bounds__(256)
k_sgemm_relu(const float *__restrict__ A, const float *__restrict__ W, const float *__restrict__ b,
             float *__restrict__ C, int M, int N, int K, int relu) {
    __shared__ __align__(16) float As[2][SG_BK][SG_BM];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;
    const int lr = tid >> 1, lk = (tid & 1) * 4;  // loader: row, k offset (float4)
    const int tr = (tid >> 4) * 8, tc = (tid & 15) * 8;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    auto load = [&](int buf, int k0) {
        const float4 a = *reinterpret_cast<const float4 *>(A + (size_t)(m0 + lr) * K + k0 + lk);
        const float4 w = *reinterpret_cast<const float4 *>(W + (size_t)(n0 + lr) * K + k0 + lk);
        As[buf][lk + 0][lr] = a.x; As[buf][lk + 1][lr] = a.y;
        As[buf][lk + 2][lr] = a.z; As[buf][lk + 3][lr] = a.w;
        Bs[buf][lk + 0][lr] = w.x; Bs[buf][lk + 1][lr] = w.y;
        Bs[buf][lk + 2][lr] = w.z; Bs[buf][lk + 3][lr] = w.w;
    };
    load(0, 0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += SG_BK) {
        if (k0 + SG_BK < K) load(buf ^ 1, k0 + SG_BK);
#pragma unroll
        for (int k = 0; k < SG_BK; ++k) {
            float a[8], w[8];
            *reinterpret_cast<float4 *>(a) = *reinterpret_cast<const float4 *>(&As[buf][k][tr]);
            *reinterpret_cast<float4 *>(a + 4) = *reinterpret_cast<const float4 *>(&As[buf][k][tr + 4]);
            *reinterpret_cast<float4 *>(w) = *reinterpret_cast<const float4 *>(&Bs[buf][k][tc]);
            *reinterpret_cast<float4 *>(w + 4) = *reinterpret_cast<const float4 *>(&Bs[buf][k][tc + 4]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
        }
        __syncthreads();
        buf ^= 1;
    }
    float bb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) bb[j] = __ldg(b + n0 + tc + j);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v = acc[i][j] + bb[j];
            o[j] = relu ? fmaxf(v, 0.f) : v;
        }
        float4 *dst = reinterpret_cast<float4 *>(C + (size_t)(m0 + tr + i) * N + n0 + tc);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
}

// ---- head: y = W_L a + b_L (FP32), integer h, mask, minf --------------------------------
__device__ __forceinline__ void load8(const float *p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16 *p, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

template <typename TIn, int DOMAIN, int HEAD>
__global__ void __launch_bounds__(128)
k_head(const TIn *__restrict__ act, int K, int C, const float *__restrict__ W,
       const float *__restrict__ bL, const uint64_t *__restrict__ states,
       const uint8_t *__restrict__ g, uint32_t bound, uint32_t n, int max_with_md, float hparam,
       uint8_t *__restrict__ h_out, uint32_t *__restrict__ mask, uint32_t *__restrict__ minf,
       float *__restrict__ y_out) {
    extern __shared__ float ylog[];  // [4 warps][C]
    __shared__ uint32_t fval[32];
    __shared__ uint8_t pass[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t s0 = blockIdx.x * 32;
    float *yw = ylog + warp * C;
    for (int i = 0; i < 8; ++i) {
        const int loc = warp * 8 + i;
        const uint32_t m = s0 + loc;
        if (m >= n) {  // warp-uniform
            if (lane == 0) { pass[loc] = 0; fval[loc] = 0xFFFFFFFFu; }
            continue;
        }
        const TIn *a = act + (size_t)m * K;
        for (int c = 0; c < C; ++c) {
            const float *w = W + (size_t)c * K;
            float part = 0.f;
            for (int k = lane * 8; k < K; k += 256) {
                float av[8], wv[8];
                load8(a + k, av);
                load8(w + k, wv);
#pragma unroll
                for (int j = 0; j < 8; ++j) part = fmaf(av[j], wv[j], part);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            if (lane == 0) yw[c] = part + __ldg(bL + c);
        }
        __syncwarp();
        if (y_out && HEAD != CBDFS_HEAD_REAL)
            for (int c = lane; c < C; c += 32) y_out[(size_t)m * C + c] = yw[c];
        if (lane == 0) {
            bool goal;
            int md = -1;
            if (DOMAIN == CBDFS_DOM_RC3) {
                goal = rc_is_goal(states[2 * m], states[2 * m + 1]);
            } else {
                constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
                const uint64_t s = states[m];
                if (max_with_md) md = manhattan<SIDE>(s);
                goal = stp_is_goal<SIDE>(s);
            }
            uint32_t f;
            if (HEAD == CBDFS_HEAD_REAL) {
                const float hr = real_h(yw[0], hparam, md, goal);
                if (h_out) h_out[m] = real_h_u8(hr);
                if (y_out) y_out[m] = hr;
                f = real_f_key(g[m], hr);
            } else {
                int hv;
                if (HEAD == CBDFS_HEAD_REGRESSION) {
                    hv = (int)fminf(fmaxf(rintf(yw[0]), 0.f), 255.f);
                } else if (HEAD == CBDFS_HEAD_QUANTILE) {
                    hv = quantile_class([&](int c) { return yw[c]; }, C, hparam);
                } else {
                    int best = 0;
                    float bv = yw[0];
                    for (int c = 1; c < C; ++c)
                        if (yw[c] > bv) { bv = yw[c]; best = c; }
                    hv = best;
                }
                hv = goal ? 0 : min(max(hv, md), 255);
                h_out[m] = (uint8_t)hv;
                f = (uint32_t)g[m] + (uint32_t)hv;
            }
            pass[loc] = f <= bound;
            fval[loc] = f <= bound ? 0xFFFFFFFFu : f;
        }
        __syncwarp();
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass[lane] != 0);
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, fval[lane]);
        if (lane == 0) {
            mask[blockIdx.x] = bits;
            if (mn != 0xFFFFFFFFu) atomicMin(minf, mn);
        }
    }
}

// ---- the last layer, register-tiled: Y[64][CPAD] = A[64][K] W^T + b ------------------
// 256 threads, 64 states; thread (ty, tx) = (tid / 16, tid % 16) owns rows 4ty..4ty+3 and
// columns CPT*tx..CPT*tx+CPT-1 (CPAD = 16 CPT).  K is walked in chunks of 32, the next
// chunk's activations and weights loaded into registers while the current one is used: A
// transposed into As[k][row] (a thread's four rows are one float4), W as Ws[col][k] padded to
// 33 floats a row.  Then the logits go to shared memory and each warp finishes eight rows.
constexpr int HT_BM = 64, HT_BK = 32, HT_THREADS = 256;
static_assert(HT_BM * HT_BK == 8 * HT_THREADS && HT_BM == 8 * (HT_THREADS / 32), "head tile shape");

template <typename TIn, int DOMAIN, int HEAD, int CPT>
__global__ void __launch_bounds__(HT_THREADS)
k_head_tiled(const TIn *__restrict__ act, int K, int C, const float *__restrict__ W,
             const float *__restrict__ bL, const uint64_t *__restrict__ states,
             const uint8_t *__restrict__ g, uint32_t bound, uint32_t n, int max_with_md, float hparam,
             uint8_t *__restrict__ h_out, uint32_t *__restrict__ mask, uint32_t *__restrict__ minf,
             float *__restrict__ y_out) {
    constexpr int CPAD = 16 * CPT;
    constexpr int NW4 = (CPAD * HT_BK / 4 + HT_THREADS - 1) / HT_THREADS;  // float4 of W per thread
    // As + Ws while the K loop runs, then the logits Ys in the same memory
    constexpr int kLoop = HT_BK * HT_BM + CPAD * (HT_BK + 1), kOut = HT_BM * (CPAD + 1);
    __shared__ __align__(16) float buf[kLoop > kOut ? kLoop : kOut];
    float (*As)[HT_BM] = reinterpret_cast<float (*)[HT_BM]>(buf);
    float (*Ws)[HT_BK + 1] = reinterpret_cast<float (*)[HT_BK + 1]>(buf + HT_BK * HT_BM);
    float (*Ys)[CPAD + 1] = reinterpret_cast<float (*)[CPAD + 1]>(buf);
    __shared__ uint32_t fval[HT_BM];
    __shared__ uint8_t pass[HT_BM];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ty = tid >> 4, tx = tid & 15;
    const uint32_t r0 = blockIdx.x * HT_BM;
    float acc[4][CPT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
    // loaders: A row lr, k offset lk (8 elements); W float4 number tid + q * HT_THREADS
    const int lr = tid >> 2, lk = (tid & 3) * 8;
    float av[8];
    float4 wv[NW4];
    auto load = [&](int k0) {
        if (r0 + lr < n) load8(act + (size_t)(r0 + lr) * K + k0 + lk, av);
        else
#pragma unroll
            for (int j = 0; j < 8; ++j) av[j] = 0.f;
#pragma unroll
        for (int q = 0; q < NW4; ++q) {
            const int idx = tid + q * HT_THREADS;  // column idx / 8, k idx % 8 * 4
            const int c = idx >> 3;
            wv[q] = (idx < CPAD * HT_BK / 4 && c < C)
                        ? __ldg(reinterpret_cast<const float4 *>(W + (size_t)c * K + k0) + (idx & 7))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    load(0);
    for (int k0 = 0; k0 < K; k0 += HT_BK) {
#pragma unroll
        for (int j = 0; j < 8; ++j) As[lk + j][lr] = av[j];
#pragma unroll
        for (int q = 0; q < NW4; ++q) {
            const int idx = tid + q * HT_THREADS;
            if (idx < CPAD * HT_BK / 4) {
                float *w = &Ws[idx >> 3][(idx & 7) * 4];
                w[0] = wv[q].x;
                w[1] = wv[q].y;
                w[2] = wv[q].z;
                w[3] = wv[q].w;
            }
        }
        __syncthreads();
        if (k0 + HT_BK < K) load(k0 + HT_BK);  // in flight while this chunk is used
#pragma unroll 8
        for (int k = 0; k < HT_BK; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const float w = Ws[tx * CPT + j][k];
                acc[0][j] = fmaf(a.x, w, acc[0][j]);
                acc[1][j] = fmaf(a.y, w, acc[1][j]);
                acc[2][j] = fmaf(a.z, w, acc[2][j]);
                acc[3][j] = fmaf(a.w, w, acc[3][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = tx * CPT + j;
            Ys[ty * 4 + i][c] = acc[i][j] + (c < C ? __ldg(bL + c) : 0.f);
        }
    __syncthreads();
    // warp w finishes rows 8w .. 8w+7
    for (int i = 0; i < 8; ++i) {
        const int loc = warp * 8 + i;
        const uint32_t m = r0 + loc;
        if (m >= n) {  // warp-uniform
            if (lane == 0) { pass[loc] = 0; fval[loc] = 0xFFFFFFFFu; }
            continue;
        }
        if (y_out && HEAD != CBDFS_HEAD_REAL)
            for (int c = lane; c < C; c += 32) y_out[(size_t)m * C + c] = Ys[loc][c];
        int hv = 0;
        if (HEAD == CBDFS_HEAD_REGRESSION) {
            hv = (int)fminf(fmaxf(rintf(Ys[loc][0]), 0.f), 255.f);
        } else if (HEAD == CBDFS_HEAD_CLASSIFIER) {
            // argmax, lowest index on ties
            float bv = -INFINITY;
            int bi = 0x7FFFFFFF;
            for (int c = lane; c < C; c += 32)
                if (Ys[loc][c] > bv) { bv = Ys[loc][c]; bi = c; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
                const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            hv = bi;
        }
        if (lane == 0) {
            if (HEAD == CBDFS_HEAD_QUANTILE) hv = quantile_class([&](int c) { return Ys[loc][c]; }, C, hparam);
            bool goal;
            int md = -1;
            if (DOMAIN == CBDFS_DOM_RC3) {
                goal = rc_is_goal(states[2 * m], states[2 * m + 1]);
            } else {
                constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
                const uint64_t s = states[m];
                if (max_with_md) md = manhattan<SIDE>(s);
                goal = stp_is_goal<SIDE>(s);
            }
            uint32_t f;
            if (HEAD == CBDFS_HEAD_REAL) {
                const float hr = real_h(Ys[loc][0], hparam, md, goal);
                if (h_out) h_out[m] = real_h_u8(hr);
                if (y_out) y_out[m] = hr;
                f = real_f_key(g[m], hr);
            } else {
                hv = goal ? 0 : min(max(hv, md), 255);
                h_out[m] = (uint8_t)hv;
                f = (uint32_t)g[m] + (uint32_t)hv;
            }
            pass[loc] = f <= bound;
            fval[loc] = f <= bound ? 0xFFFFFFFFu : f;
        }
    }
    __syncthreads();
    if (warp < HT_BM / 32) {
        const int loc = warp * 32 + lane;
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass[loc] != 0);
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, fval[loc]);
        if (lane == 0 && r0 + warp * 32 < n) {
            mask[(r0 >> 5) + warp] = bits;
            if (mn != 0xFFFFFFFFu) atomicMin(minf, mn);
        }
    }
}

template <typename TIn, int DOMAIN, int HEAD>
int head_tiled(const TIn *act, int K, int C, const float *W, const float *b, const uint64_t *states,
               const uint8_t *g, uint32_t bound, uint32_t n, int md, float off, uint8_t *h,
               uint32_t *mask, uint32_t *minf, float *y, cudaStream_t st) {
    const unsigned blocks = (n + HT_BM - 1) / HT_BM;
#define HT_LAUNCH(CPT) k_head_tiled<TIn, DOMAIN, HEAD, CPT><<<blocks, HT_THREADS, 0, st>>>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y)
    if (HEAD == CBDFS_HEAD_REAL || C <= 16) {  // a real-valued head has one output
        HT_LAUNCH(1);
    } else if constexpr (HEAD != CBDFS_HEAD_REAL) {
        if (C <= 32) HT_LAUNCH(2);
        else if (C <= 64) HT_LAUNCH(4);
        else if (C <= 96) HT_LAUNCH(6);
        else HT_LAUNCH(8);
    }
#undef HT_LAUNCH
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

template <typename TIn, int DOMAIN, int HEAD>
int head_any(const TIn *act, int K, int C, const float *W, const float *b, const uint64_t *states,
             const uint8_t *g, uint32_t bound, uint32_t n, int md, float off, uint8_t *h,
             uint32_t *mask, uint32_t *minf, float *y, cudaStream_t st) {
    if (C <= 128 && K % HT_BK == 0 && (size_t)act % 16 == 0 && (size_t)W % 16 == 0)
        return head_tiled<TIn, DOMAIN, HEAD>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y, st);
    const unsigned blocks = (n + 31) / 32;
    const size_t sm = 4 * C * sizeof(float);
    k_head<TIn, DOMAIN, HEAD><<<blocks, 128, sm, st>>>(act, K, C, W, b, states, g, bound, n, md, off, h,
                                                       mask, minf, y);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

template <typename TIn, int DOMAIN>
int head_dom(int head, const TIn *act, int K, int C, const float *W, const float *b,
             const uint64_t *states, const uint8_t *g, uint32_t bound, uint32_t n, int md, float off,
             uint8_t *h, uint32_t *mask, uint32_t *minf, float *y, cudaStream_t st) {
    if (head == CBDFS_HEAD_REGRESSION)
        return head_any<TIn, DOMAIN, CBDFS_HEAD_REGRESSION>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y, st);
    if (head == CBDFS_HEAD_CLASSIFIER)
        return head_any<TIn, DOMAIN, CBDFS_HEAD_CLASSIFIER>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y, st);
    if (head == CBDFS_HEAD_QUANTILE)
        return head_any<TIn, DOMAIN, CBDFS_HEAD_QUANTILE>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y, st);
    return head_any<TIn, DOMAIN, CBDFS_HEAD_REAL>(act, K, C, W, b, states, g, bound, n, md, off, h, mask, minf, y, st);
}

}  // namespace

int first_gather(int domain, const uint64_t *states, uint32_t n, const float *W1T, const float *b1,
                 int H, float *out, cudaStream_t st) {
    const unsigned blocks = (n + 7) / 8;
    if (domain == CBDFS_DOM_STP3) k_first_gather<CBDFS_DOM_STP3><<<blocks, 256, 0, st>>>(states, n, W1T, b1, H, out);
    else if (domain == CBDFS_DOM_STP4) k_first_gather<CBDFS_DOM_STP4><<<blocks, 256, 0, st>>>(states, n, W1T, b1, H, out);
    else k_first_gather<CBDFS_DOM_RC3><<<blocks, 256, 0, st>>>(states, n, W1T, b1, H, out);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

int sgemm_relu(const float *A, const float *W, const float *b, float *C, int M, int N, int K,
               int relu, cudaStream_t st) {
    if (M % SG_BM || N % SG_BN || K % SG_BK)
        return fail(CBDFS_EINVAL, "sgemm shape %dx%dx%d not tile-aligned", M, N, K);
    dim3 grid(N / SG_BN, M / SG_BM);
    k_sgemm_relu<<<grid, 256, 0, st>>>(A, W, b, C, M, N, K, relu);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

int head(bool bf16_in, int domain, int head_kind, const void *act, int K, int C, const float *W,
         const float *b, const uint64_t *states, const uint8_t *g, uint32_t bound, uint32_t n,
         int max_with_md, float hparam, uint8_t *h, uint32_t *mask, uint32_t *minf, float *y,
         cudaStream_t st) {
    if (bf16_in) {
        auto a = static_cast<const __nv_bfloat16 *>(act);
        if (domain == CBDFS_DOM_STP3) return head_dom<__nv_bfloat16, CBDFS_DOM_STP3>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
        if (domain == CBDFS_DOM_STP4) return head_dom<__nv_bfloat16, CBDFS_DOM_STP4>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
        return head_dom<__nv_bfloat16, CBDFS_DOM_RC3>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
    }
    auto a = static_cast<const float *>(act);
    if (domain == CBDFS_DOM_STP3) return head_dom<float, CBDFS_DOM_STP3>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
    if (domain == CBDFS_DOM_STP4) return head_dom<float, CBDFS_DOM_STP4>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
    return head_dom<float, CBDFS_DOM_RC3>(head_kind, a, K, C, W, b, states, g, bound, n, max_with_md, hparam, h, mask, minf, y, st);
}

}  // namespace cbdfs
