// api.cu -- the C entry points around the heuristic kernels: context and slots, loading of
// networks and pattern databases (with the precision conversion), the evaluation
// pipeline, and the host-buffer / device-buffer evaluation calls.
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <thread>

#include "chain.h"

namespace cbdfs {

// kernels defined in the other translation units
int tc_layer(bool first, int domain, bool fp8, bool out_fp8, int bn, const CUtensorMap &tmA,
             const CUtensorMap &tmB, const uint64_t *states, uint32_t n, uint32_t rows_pad, int K,
             int N, const float *bias, void *out, float acc_scale, float out_qscale, int *err,
             cudaStream_t st);
int first_gather(int domain, const uint64_t *states, uint32_t n, const float *W1T, const float *b1,
                 int H, float *out, cudaStream_t st);
int sgemm_relu(const float *A, const float *W, const float *b, float *C, int M, int N, int K,
               int relu, cudaStream_t st);
int head(bool bf16_in, int domain, int head_kind, const void *act, int K, int C, const float *W,
         const float *b, const uint64_t *states, const uint8_t *g, uint32_t bound, uint32_t n,
         int max_with_md, float offset, uint8_t *h, uint32_t *mask, uint32_t *minf, float *y,
         cudaStream_t st);
int pdb_gather(int domain, const PdbParams &P, const uint64_t *states, uint32_t n, const uint8_t *g,
               uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf, cudaStream_t st);
int pdb_build_device(Ctx *c, int side, const int *tiles, int k, uint8_t *table, cudaStream_t st);
size_t rc_corner_entries();
int rc_corner_gather(const uint8_t *table, uint32_t div, const uint64_t *states, uint32_t n, const uint8_t *g,
                     uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf, cudaStream_t st);
int pdb_div_compress(const uint8_t *src, uint64_t n, uint32_t k, uint8_t *dst, cudaStream_t st);
int rc_corner_build_device(Ctx *c, uint8_t *table, cudaStream_t st);
int combine(int domain, const ComboParams &C, const uint64_t *states, uint32_t n, const uint8_t *member_h,
            size_t member_stride, const uint8_t *g, uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf,
            cudaStream_t st);
uint64_t npk(int n, int k);



// the fused chain runs low-precision networks whose hidden widths are multiples of 256; a last
// layer of at most 32 outputs runs in its epilogue, a wider one in a separate kernel after it
// ints of a slot's chain counters: (layers + 2) per row block.  A launch leaves them zero (after a
// device error, cbdfs_device_status does)
static int chain_counter_ints(const Ctx *c) { return (kMaxLayers + 2) * (c->max_batch_pad / kBM); }

// a network's device buffers (at context teardown)
static void free_net_buffers(NetGPU &n) {
    for (int l = 0; l < kMaxLayers; ++l) {
        if (n.w_lp[l]) cudaFree(n.w_lp[l]);
        if (n.w32[l]) cudaFree(n.w32[l]);
        if (n.b32[l]) cudaFree(n.b32[l]);
    }
    if (n.w_split) cudaFree(n.w_split);
}

// tables of an additive PDB that together fit in this many bytes are kept in L2 (half of
// the B300's 126 MB)
constexpr size_t kL2KeepBytes = 64ull << 20;

static bool chain_ok(const NetGPU &net) {
    if (net.prec == CBDFS_PREC_FP32) return false;
    for (int l = 1; l < net.L; ++l)
        if (net.dims[l] % kChainBN) return false;
    return true;
}
static size_t chain_partial_floats(const NetGPU &net) {
    if (net.dims[net.L] > kMaxHeadC) return 0;  // a separate kernel runs the last layer
    return (size_t)(net.dims[net.L - 1] / kChainBN) * net.dims[net.L];
}

// ------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------
static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

// ------------------------------------------------------------------------------------
// memory
// ------------------------------------------------------------------------------------
int dev_alloc(Ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return CBDFS_OK;
    if (c->mem_budget && c->mem_used + bytes > c->mem_budget)
        return fail(CBDFS_ENOMEM, "device memory budget of %zu bytes exceeded (%zu in use, %zu asked)",
                    c->mem_budget, c->mem_used, bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(CBDFS_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->mem_used += bytes;
    return CBDFS_OK;
}
void dev_free(Ctx *c, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->mem_used -= bytes;
}

// ------------------------------------------------------------------------------------
// TMA descriptors
// ------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int make_tmap_2d(CUtensorMap *map, void *base, CUtensorMapDataType dt, int elem_bytes,
                 uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer,
                 CUtensorMapSwizzle swizzle) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(CBDFS_EDEVICE, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * elem_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CBDFS_EDEVICE, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CBDFS_OK;
}

// ------------------------------------------------------------------------------------
// built-in heuristics: zero and Manhattan distance, with the bound test
// ------------------------------------------------------------------------------------
namespace {
template <int DOMAIN, bool MD>
__global__ void k_builtin(const uint64_t *__restrict__ states, uint32_t n, const uint8_t *__restrict__ g,
                          uint32_t bound, uint8_t *__restrict__ h, uint32_t *__restrict__ mask,
                          uint32_t *__restrict__ minf) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t f = 0xFFFFFFFFu;
    bool pass = false;
    if (i < n) {
        uint32_t hv = 0;
        if (MD && DOMAIN != CBDFS_DOM_RC3) {
            constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
            hv = dev::manhattan<SIDE>(states[i]);
        }
        h[i] = (uint8_t)hv;
        f = (uint32_t)g[i] + hv;
        pass = f <= bound;
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
    const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
    if (lane == 0 && i < n) {
        mask[i >> 5] = bits;
        if (mn != 0xFFFFFFFFu) atomicMin(minf, mn);
    }
}

int builtin(int heur, int domain, const uint64_t *s, uint32_t n, const uint8_t *g, uint32_t bound,
            uint8_t *h, uint32_t *mask, uint32_t *minf, cudaStream_t st) {
    const unsigned b = (n + 255) / 256;
    if (heur == CBDFS_HEUR_MD) {
        if (domain == CBDFS_DOM_STP3) k_builtin<CBDFS_DOM_STP3, true><<<b, 256, 0, st>>>(s, n, g, bound, h, mask, minf);
        else if (domain == CBDFS_DOM_STP4) k_builtin<CBDFS_DOM_STP4, true><<<b, 256, 0, st>>>(s, n, g, bound, h, mask, minf);
        else return fail(CBDFS_EINVAL, "Manhattan distance is defined for sliding-tile domains only");
    } else {
        if (domain == CBDFS_DOM_RC3) k_builtin<CBDFS_DOM_RC3, false><<<b, 256, 0, st>>>(s, n, g, bound, h, mask, minf);
        else k_builtin<CBDFS_DOM_STP4, false><<<b, 256, 0, st>>>(s, n, g, bound, h, mask, minf);
    }
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

uint16_t f32_to_bf16_rne(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

int ensure_act(Ctx *c, size_t width) {
    if (width <= c->max_width) return CBDFS_OK;
    const size_t bytes = (size_t)c->max_batch_pad * width * 4;
    for (auto &s : c->slots) {
        for (int i = 0; i < 2; ++i) {
            dev_free(c, s.act[i], c->act_bytes);
            s.act[i] = nullptr;
        }
        s.tm_act.clear();
    }
    c->act_bytes = 0;
    for (auto &s : c->slots)
        for (int i = 0; i < 2; ++i) {
            int rc = dev_alloc(c, &s.act[i], bytes);
            if (rc) return rc;
        }
    c->act_bytes = bytes;
    c->max_width = width;
    ++c->buf_gen;
    return CBDFS_OK;
}

// chain scratch of every slot: tile counters, and head partials of `floats` per row
int ensure_chain(Ctx *c, size_t floats) {
    const size_t cbytes = sizeof(int) * chain_counter_ints(c);
    for (auto &s : c->slots)
        if (!s.counters) {
            int rc = dev_alloc(c, (void **)&s.counters, cbytes);
            if (!rc && cudaMemset(s.counters, 0, cbytes) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "counter init");
            if (!rc) rc = dev_alloc(c, &s.onehot, (size_t)c->max_batch_pad * 1024);
            if (rc) return rc;
            ++c->buf_gen;
        }
    if (floats <= c->partial_floats) return CBDFS_OK;
    const size_t pbytes = sizeof(float) * floats * c->max_batch_pad;
    for (auto &s : c->slots) {
        dev_free(c, s.partial, s.partial_bytes);
        s.partial = nullptr;
        s.partial_bytes = 0;
        int rc = dev_alloc(c, (void **)&s.partial, pbytes);
        if (rc) return rc;
        s.partial_bytes = pbytes;
    }
    c->partial_floats = floats;
    ++c->buf_gen;
    return CBDFS_OK;
}

const CUtensorMap *act_map(Slot &s, Ctx *c, int buf, int K, int elem_bytes) {
    const long long key = ((long long)buf << 40) | ((long long)elem_bytes << 32) | K;
    auto it = s.tm_act.find(key);
    if (it != s.tm_act.end()) return &it->second;
    CUtensorMap m;
    if (make_tmap_2d(&m, s.act[buf],
                     elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     elem_bytes, (uint64_t)K, c->max_batch_pad, 128 / elem_bytes, kBM))
        return nullptr;
    return &s.tm_act.emplace(key, m).first->second;
}

// TMA store maps over the activation buffers: 32-element x 32-row boxes, swizzled so that
// one row per lane lands in shared memory without bank conflicts (64 B rows: 64-byte
// swizzle; 32 B rows of E4M3: 32-byte swizzle)
const CUtensorMap *act_store_map(Slot &s, Ctx *c, int buf, int K, int elem_bytes) {
    const long long key = (1LL << 50) | ((long long)buf << 40) | ((long long)elem_bytes << 32) | K;
    auto it = s.tm_act.find(key);
    if (it != s.tm_act.end()) return &it->second;
    CUtensorMap m;
    if (make_tmap_2d(&m, s.act[buf],
                     elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     elem_bytes, (uint64_t)K, c->max_batch_pad, 32, 32,
                     elem_bytes == 1 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B))
        return nullptr;
    return &s.tm_act.emplace(key, m).first->second;
}

// TMA load map over the one-hot rows (row stride = the padded one-hot width)
const CUtensorMap *onehot_map(Slot &s, Ctx *c, int K, int elem_bytes) {
    const long long key = (2LL << 50) | ((long long)elem_bytes << 32) | K;
    auto it = s.tm_act.find(key);
    if (it != s.tm_act.end()) return &it->second;
    CUtensorMap m;
    if (make_tmap_2d(&m, s.onehot,
                     elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     elem_bytes, (uint64_t)K, c->max_batch_pad, 128 / elem_bytes, kBM))
        return nullptr;
    return &s.tm_act.emplace(key, m).first->second;
}

}  // namespace

// ------------------------------------------------------------------------------------
// the evaluation pipeline
// ------------------------------------------------------------------------------------
static int mark(Slot &s, cudaStream_t st) {
    if (!s.prof) return CBDFS_OK;
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventRecord(e, st));
    s.prof->push_back(e);
    return CBDFS_OK;
}

// the whole network in one persistent launch (mlp_chain.cu).  outs (training's forward pass):
// every hidden layer l stored to outs[l] ([out_rows][dims[l+1]] BF16) instead of the slot's
// two alternating buffers, and no last layer (the caller runs it)
static int run_chain(Ctx *c, Slot &s, const NetGPU &net, int domain, const uint64_t *d_states,
                     const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask,
                     uint32_t *d_minf, float *d_y, cudaStream_t st, void *const *outs = nullptr,
                     uint32_t out_rows = 0) {
    const bool fp8 = net.prec == CBDFS_PREC_FP8;
    const int eb = fp8 ? 1 : 2;
    const int L = net.L, nh = L - 1;
    ChainMaps maps;
    ChainParams P{};
    P.nh = nh;
    for (int l = 0; l <= L; ++l) P.dims[l] = net.dims[l];
    uint32_t rows_pad = (n + kBM - 1) / kBM * kBM;
    // small batches: 64-wide tiles, so that a layer's tiles spread over more CTAs, while the
    // widest layer's 64-wide tiles are at most 4/3 of the SM count (beyond that the extra
    // epilogues cost more than the spread gains: 15-puzzle network, 1024 wide, up to 1536
    // states; cube network, 2048 wide, up to 768); the head partials then need four times the
    // floats per row, within the slot's allocation
    int widest = 0;
    for (int l = 0; l < nh; ++l) widest = std::max(widest, net.dims[l + 1]);
    const bool small = (int)(rows_pad / kBM) * (widest / kChainBNSmall) <= c->num_sms + c->num_sms / 3;
    const int bn = small && 4 * rows_pad <= c->max_batch_pad ? kChainBNSmall : kChainBN;
    // larger batches: CTA pairs (two row blocks per tile, tcgen05 cta_group::2), when the
    // batch padded to 256 rows fits the slot and the device holds every pair at once
    const uint32_t rows_pair = (n + 2 * kBM - 1) / (2 * kBM) * (2 * kBM);
    const bool pair = net.has_w128 && bn == kChainBN && rows_pad / kBM >= kChainPairMinMBlocks && rows_pair <= c->max_batch_pad &&
                      (!outs || rows_pair <= out_rows) && (c->num_sms & 1) == 0 && chain_pairs_fit(c->num_sms);
    if (pair) rows_pad = rows_pair;
    P.mblocks = rows_pad / kBM;
    P.rows_pad = rows_pad;
    P.n = n;
    const int seq_mblocks = pair ? P.mblocks / 2 : P.mblocks;  // row blocks (pairs) in the tile sequence
    int max_tiles = 0;
    P.tile_start[0] = 0;
    P.fused_head = !outs && net.dims[L] <= kMaxHeadC && !net.head_cpad;
    P.bf16_store_layer = !P.fused_head && fp8 ? nh - 1 : -1;
    for (int l = 0; l < nh; ++l) {
        maps.w[l] = bn == kChainBNSmall ? net.tm_w64[l] : pair ? net.tm_w128[l] : net.tm_w[l];
        if (l > 0 && outs) {
            if (int rc = make_tmap_2d(&maps.a[l], outs[l - 1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                      (uint64_t)net.dims[l], out_rows, 64, kBM))
                return rc;
        } else if (l > 0) {
            const CUtensorMap *m = act_map(s, c, (l - 1) & 1, net.dims[l], eb);
            if (!m) return CBDFS_EDEVICE;
            maps.a[l] = *m;
        } else {
            const CUtensorMap *m = onehot_map(s, c, net.k1pad, eb);
            if (!m) return CBDFS_EDEVICE;
            maps.a[0] = *m;
        }
        if (outs) {
            if (int rc = make_tmap_2d(&maps.o[l], outs[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                      (uint64_t)net.dims[l + 1], out_rows, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B))
                return rc;
        } else if (l < nh - 1 || !P.fused_head) {  // stored activations: 32 x 32 boxes, by TMA stores
            const CUtensorMap *m = act_store_map(s, c, l & 1, net.dims[l + 1], l == P.bf16_store_layer ? 2 : eb);
            if (!m) return CBDFS_EDEVICE;
            maps.o[l] = *m;
        } else {
            maps.o[l] = net.tm_w[0];  // unused
        }
        P.kdim[l] = l == 0 ? net.k1pad : net.dims[l] / net.groups;
        P.nt[l] = net.dims[l + 1] / bn;
        P.group_nt[l] = l > 0 && net.groups > 1 ? P.nt[l] / net.groups : 0;
        P.tile_start[l + 1] = P.tile_start[l] + P.nt[l] * seq_mblocks;
        max_tiles = std::max(max_tiles, P.nt[l] * seq_mblocks);
        P.bias[l] = net.b32[l];
        P.acc_scale[l] = fp8 ? net.w_scale[l] * (l == 0 ? 1.f : net.a_scale[l - 1]) : 1.f;
        P.out_qscale[l] = fp8 ? 1.f / net.a_scale[l] : 1.f;
    }
    P.states = d_states;
    P.onehot = s.onehot;
    P.act[0] = s.act[0];
    P.act[1] = s.act[1];
    P.counters = s.counters;
    P.unit_rows = net.k1pad * eb <= 512 ? 16 : 8;
    P.partial = s.partial;
    P.C = net.dims[L];
    P.head_kind = net.head;
    P.max_with_md = net.max_with_md;
    P.head_param = net.head_param();
    P.w_last = net.w32[L - 1];
    P.b_last = net.b32[L - 1];
    P.g = d_g;
    P.bound = bound;
    P.h = d_h;
    P.mask = d_mask;
    P.minf = d_minf;
    P.y = d_y;
    P.err = c->d_err;
    P.wait_ns = c->wait_ns;
    P.hold_mblock = outs ? -1 : c->hold_mblock.exchange(-1);
    const int grid = pair ? 2 * std::min(c->num_sms / 2, max_tiles) : std::min(c->num_sms, max_tiles);
    if (s.trace) {
        P.trace = s.trace;
        P.trace_tiles = s.trace_tiles;
        *s.trace_grid = grid;
        CUDA_TRY(cudaMemsetAsync(s.trace, 0, sizeof(unsigned long long) * grid * s.trace_tiles * 8, st));
    }
    int rc = chain_launch(domain, fp8, bn, pair, maps, P, grid, st);
    if (rc || (rc = mark(s, st)) || P.fused_head || outs) return rc;
    // the last layer over the stored BF16 activations of the last hidden layer: on the tensor
    // cores (split FP32 weights) for a prepared classifier head, else FP32 on the CUDA cores
    if (net.head_cpad) {
        const CUtensorMap *ma = act_map(s, c, (nh - 1) & 1, net.dims[nh], 2);
        if (!ma) return CBDFS_EDEVICE;
        HeadTcParams H{};
        H.K = net.dims[nh] / net.groups;
        H.groups = net.groups;
        H.h_stride = c->max_batch_pad;
        H.C = net.dims[L];
        H.cpad = net.head_cpad;
        H.head_kind = net.head;
        H.quantile = net.quantile;
        H.max_with_md = net.max_with_md;
        H.n = n;
        H.states = d_states;
        H.g = d_g;
        H.bound = bound;
        H.b_last = net.b32[L - 1];
        H.h = d_h;
        H.mask = d_mask;
        H.minf = d_minf;
        H.y = d_y;
        H.err = c->d_err;
        rc = head_tc(domain, *ma, net.tm_wsplit, H, rows_pad, st);
    } else {
        rc = head(true, domain, net.head, s.act[(nh - 1) & 1], net.dims[nh], net.dims[L], net.w32[L - 1],
                  net.b32[L - 1], d_states, d_g, bound, n, net.max_with_md, net.head_param(), d_h, d_mask, d_minf,
                  d_y, st);
    }
    return rc ? rc : mark(s, st);
}

// Training's forward pass through the fused chain: every hidden layer of a BF16 network stored
// to outs[l] (out_rows rows); CBDFS_ENOTFOUND when the chain does not take this network or
// slot (the caller then runs the layers one by one)
int chain_forward_store(Ctx *c, Slot &s, const NetGPU &net, const uint64_t *d_states, uint32_t n,
                        void *const *outs, uint32_t out_rows, cudaStream_t st) {
    if (net.prec != CBDFS_PREC_BF16 || net.groups > 1 || !chain_ok(net) || !s.counters || !s.onehot ||
        n > out_rows)
        return CBDFS_ENOTFOUND;
    return run_chain(c, s, net, net.domain, d_states, nullptr, 255, n, nullptr, nullptr, nullptr, nullptr, st, outs,
                     out_rows);
}

int run_eval(Ctx *c, Slot &s, int heur_id, int domain, const uint64_t *d_states, const uint8_t *d_g,
             uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask, uint32_t *d_minf, float *d_y,
             cudaStream_t st) {
    CUDA_TRY(cudaMemsetAsync(d_minf, 0xFF, sizeof(uint32_t), st));
    if (n == 0) return CBDFS_OK;
    // the kernels read a cube state as one 16-byte load
    if (domain == CBDFS_DOM_RC3 && (reinterpret_cast<uintptr_t>(d_states) & 15u))
        return fail(CBDFS_EINVAL, "cube states must start on a 16-byte boundary");
    if (int r = mark(s, st)) return r;
    if (heur_id < 0) {
        int r = builtin(heur_id, domain, d_states, n, d_g, bound, d_h, d_mask, d_minf, st);
        return r ? r : mark(s, st);
    }
    if (c->heur_kind[heur_id] == 2) {
        // composite: every member into its row of the slot's member scratch (their own bound
        // tests go to scratch too), then the combination with the bound test
        const ComboGPU &cb = *c->combos[c->heur_index[heur_id]];
        if (cb.domain != domain) return fail(CBDFS_EINVAL, "composite %d is for another domain", heur_id);
        if (!s.combo) return fail(CBDFS_EINVAL, "composite heuristics need a context slot's scratch");
        const size_t stride = c->max_batch_pad;
        uint32_t *mmask = reinterpret_cast<uint32_t *>(s.combo + (size_t)kComboMaxTotal * stride);
        uint32_t *mminf = mmask + stride / 32;
        for (int grp = 0, m = 0; grp < cb.P.n_groups; m += cb.P.group_size[grp++]) {
            if (cb.fused[grp]) {  // the group's networks as one grouped network: h rows m, m+1, ...
                int r = run_chain(c, s, *cb.fused[grp], domain, d_states, d_g, 255, n, s.combo + (size_t)m * stride,
                                  mmask, mminf, nullptr, st);
                if (r) return r;
                continue;
            }
            for (int j = 0; j < cb.P.group_size[grp]; ++j) {
                int r = run_eval(c, s, cb.members[m + j], domain, d_states, d_g, 255, n, s.combo + (size_t)(m + j) * stride,
                                 mmask, mminf, nullptr, st);
                if (r) return r;
            }
        }
        int r = combine(domain, cb.P, d_states, n, s.combo, stride, d_g, bound, d_h, d_mask, d_minf, st);
        return r ? r : mark(s, st);
    }
    if (c->heur_kind[heur_id] == 1) {
        const PdbGPU &p = *c->pdbs[c->heur_index[heur_id]];
        if (p.domain != domain) return fail(CBDFS_EINVAL, "PDB %d is for another domain", heur_id);
        if (domain == CBDFS_DOM_RC3) {
            int r = rc_corner_gather(p.table[0], p.div, d_states, n, d_g, bound, d_h, d_mask, d_minf, st);
            return r ? r : mark(s, st);
        }
        PdbParams P{};
        P.n_patterns = p.n_patterns;
        const int N = p.side * p.side;
        for (int q = 0; q < p.n_patterns; ++q) {
            P.k[q] = p.k[q];
            P.table[q] = p.table[q];
            P.entries[q] = (uint32_t)p.entries[q];
            P.div = p.div;
            for (int i = 0; i < p.k[q]; ++i) {
                P.tiles[q][i] = p.tiles[q][i];
                P.weight[q][i] = (uint32_t)npk(N - 1 - i, p.k[q] - 1 - i);
            }
        }
        // L2 priorities: the smallest tables that fit in half the L2 together stay resident
        // (their lookups hit it once warm), and the larger tables' random lines are evicted
        // first so that they do not push the small ones out
        {
            size_t kept = 0;
            uint32_t order[4] = {0, 1, 2, 3};
            std::sort(order, order + p.n_patterns, [&](uint32_t a, uint32_t b) { return p.entries[a] < p.entries[b]; });
            for (int j = 0; j < p.n_patterns; ++j) {
                const uint32_t q = order[j];
                if (kept + p.entries[q] > kL2KeepBytes) break;
                kept += p.entries[q];
                P.l2_keep |= 1u << q;
            }
            if (P.l2_keep == (1u << p.n_patterns) - 1) P.l2_keep = 0;  // all fit: plain caching
        }
        int r = pdb_gather(domain, P, d_states, n, d_g, bound, d_h, d_mask, d_minf, st);
        return r ? r : mark(s, st);
    }
    const NetGPU &net = *c->nets[c->heur_index[heur_id]];
    if (net.domain != domain) return fail(CBDFS_EINVAL, "network %d is for another domain", heur_id);
    const uint32_t rows_pad = (n + kBM - 1) / kBM * kBM;
    const int L = net.L;
    int rc;
    if (net.prec == CBDFS_PREC_FP32) {
        float *a = (float *)s.act[0], *b = (float *)s.act[1];
        rc = first_gather(domain, d_states, n, net.w32[0], net.b32[0], net.dims[1], a, st);
        if (rc || (rc = mark(s, st))) return rc;
        for (int l = 1; l < L - 1; ++l) {
            rc = sgemm_relu(a, net.w32[l], net.b32[l], b, (int)rows_pad, net.dims[l + 1], net.dims[l], 1, st);
            if (rc || (rc = mark(s, st))) return rc;
            std::swap(a, b);
        }
        rc = head(false, domain, net.head, a, net.dims[L - 1], net.dims[L], net.w32[L - 1], net.b32[L - 1],
                  d_states, d_g, bound, n, net.max_with_md, net.head_param(), d_h, d_mask, d_minf, d_y, st);
        return rc ? rc : mark(s, st);
    }
    const bool fp8 = net.prec == CBDFS_PREC_FP8;
    if (s.counters && chain_ok(net) && chain_partial_floats(net) <= c->partial_floats &&
        (s.partial || chain_partial_floats(net) == 0))
        return run_chain(c, s, net, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, d_y, st);
    int cur = 0;
    for (int l = 0; l < L - 1; ++l) {
        const bool first = l == 0;
        const bool out_fp8 = fp8 && l < L - 2;  // the head reads BF16
        const int K = first ? net.k1pad : net.dims[l];
        const CUtensorMap *tmA = &net.tm_w[0];  // placeholder for the first layer
        if (!first) {
            tmA = act_map(s, c, cur, K, fp8 ? 1 : 2);
            if (!tmA) return CBDFS_EDEVICE;
        }
        const int out_buf = first ? 0 : cur ^ 1;
        const float acc_scale = fp8 ? net.w_scale[l] * (first ? 1.f : net.a_scale[l - 1]) : 1.f;
        const float out_q = out_fp8 ? 1.f / net.a_scale[l] : 1.f;
        rc = tc_layer(first, domain, fp8, out_fp8, net.bn[l], *tmA, net.tm_w[l], d_states, n, rows_pad,
                      K, net.dims[l + 1], net.b32[l], s.act[out_buf], acc_scale, out_q, c->d_err, st);
        if (rc || (rc = mark(s, st))) return rc;
        cur = out_buf;
    }
    rc = head(true, domain, net.head, s.act[cur], net.dims[L - 1], net.dims[L], net.w32[L - 1],
              net.b32[L - 1], d_states, d_g, bound, n, net.max_with_md, net.head_param(), d_h, d_mask, d_minf,
              d_y, st);
    return rc ? rc : mark(s, st);
}

bool heur_is_real(const Ctx *c, int heur_id) {
    return heur_id >= 0 && heur_id < (int)c->heur_kind.size() && c->heur_kind[heur_id] == 0 &&
           c->nets[c->heur_index[heur_id]]->head == CBDFS_HEAD_REAL;
}

}  // namespace cbdfs

using namespace cbdfs;

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

const char *cbdfs_last_error(void) { return g_err; }

size_t cbdfs_mem_used(const cbdfs_ctx *ctx) {
    return ctx ? reinterpret_cast<const Ctx *>(ctx)->mem_used : 0;
}

void cbdfs_destroy(cbdfs_ctx *ctx) {
    if (!ctx) return;
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    cudaSetDevice(c->device);
    if (c->server) cbdfs_server_stop(ctx);
    cudaDeviceSynchronize();
    for (auto &s : c->slots) {
        for (int i = 0; i < 2; ++i) dev_free(c, s.act[i], c->act_bytes);
        dev_free(c, s.d_states, (size_t)c->max_batch_pad * 16);
        dev_free(c, s.d_g, c->max_batch_pad);
        dev_free(c, s.d_h, slot_out_bytes(c));  // h, mask and minf share one allocation
        dev_free(c, s.counters, sizeof(int) * chain_counter_ints(c));
        dev_free(c, s.onehot, (size_t)c->max_batch_pad * 1024);
        dev_free(c, s.partial, s.partial_bytes);
        dev_free(c, s.combo, combo_bytes(c));
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.h_small) cudaFreeHost(s.h_small);
    }
    for (auto &n : c->nets) {
        train_free(c, n->train);
        n->train = nullptr;
        for (int l = 0; l < kMaxLayers; ++l) {
            if (n->w_lp[l]) cudaFree(n->w_lp[l]);
            if (n->w32[l]) cudaFree(n->w32[l]);
            if (n->b32[l]) cudaFree(n->b32[l]);
        }
        if (n->w_split) cudaFree(n->w_split);
    }
    for (auto &p : c->pdbs)
        for (int q = 0; q < 4; ++q)
            if (p->table[q]) cudaFree(p->table[q]);
    for (auto &cb : c->combos)
        for (auto &f : cb->fused)
            if (f) free_net_buffers(*f);
    if (c->d_err) cudaFree(c->d_err);
    delete c;
}

int cbdfs_create(const cbdfs_config *cfg, cbdfs_ctx **out) {
    if (!cfg || !out) return fail(CBDFS_EINVAL, "null argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(CBDFS_EDEVICE, "no CUDA device");
    if (cfg->device < 0 || cfg->device >= ndev) return fail(CBDFS_EINVAL, "device %d out of range", cfg->device);
    CUDA_TRY(cudaSetDevice(cfg->device));
    Ctx *c = new Ctx();
    c->device = cfg->device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cfg->device);
    if (c->num_sms <= 0) c->num_sms = 1;
    c->mem_budget = cfg->mem_budget;
    c->wait_ns = cfg->device_wait_ns ? cfg->device_wait_ns : dev::kWaitNs;
    c->max_batch = cfg->max_batch ? cfg->max_batch : 65536;
    c->max_batch_pad = (c->max_batch + kBM - 1) / kBM * kBM;
    const int nslots = 1 + (cfg->n_slots > 0 ? cfg->n_slots : 4);  // slot 0: device-buffer calls
    c->slots.resize(nslots);
    int rc = dev_alloc(c, (void **)&c->d_err, sizeof(int));
    if (!rc && cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "memset");
    for (int i = 0; i < nslots && !rc; ++i) {
        Slot &s = c->slots[i];
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            rc = fail(CBDFS_EDEVICE, "stream/event creation");
            break;
        }
        if (i == 0) continue;
        rc = dev_alloc(c, (void **)&s.d_states, (size_t)c->max_batch_pad * 16);
        if (!rc) rc = dev_alloc(c, (void **)&s.d_g, c->max_batch_pad);
        // h, mask and minf in one block (slot_out_bytes), so that one copy returns them all
        if (!rc) rc = dev_alloc(c, (void **)&s.d_h, slot_out_bytes(c));
        if (!rc) {
            s.d_mask = reinterpret_cast<uint32_t *>(s.d_h + c->max_batch_pad);
            s.d_minf = s.d_mask + c->max_batch_pad / 32;
        }
        if (!rc && cudaMallocHost(&s.h_small, 16) != cudaSuccess) rc = fail(CBDFS_ENOMEM, "pinned words");
    }
    if (rc) {
        cbdfs_destroy(reinterpret_cast<cbdfs_ctx *>(c));
        return rc;
    }
    *out = reinterpret_cast<cbdfs_ctx *>(c);
    return CBDFS_OK;
}

int cbdfs_net_load(cbdfs_ctx *ctx, const cbdfs_net_desc *d, int *heur_id) {
    if (!ctx || !d || !heur_id || !d->dims || !d->weights || !d->biases)
        return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    // a load may move the slots' scratch under the server's launches and captured graphs
    if (c->server) return fail(CBDFS_EINVAL, "stop the server before loading a heuristic");
    CUDA_TRY(cudaSetDevice(c->device));
    const int L = d->n_layers;
    if (L < 2 || L > kMaxLayers) return fail(CBDFS_EINVAL, "n_layers %d outside 2..%d", L, kMaxLayers);
    if (d->domain < 0 || d->domain > 2) return fail(CBDFS_EINVAL, "domain %d", d->domain);
    if (d->dims[0] != dom_onehot(d->domain))
        return fail(CBDFS_EINVAL, "dims[0]=%d but the domain's one-hot width is %d", d->dims[0], dom_onehot(d->domain));
    if (d->prec < 0 || d->prec > 2) return fail(CBDFS_EINVAL, "precision %d", d->prec);
    if (d->head < CBDFS_HEAD_REGRESSION || d->head > CBDFS_HEAD_QUANTILE) return fail(CBDFS_EINVAL, "head %d", d->head);
    if ((d->head == CBDFS_HEAD_REGRESSION || d->head == CBDFS_HEAD_REAL) && d->dims[L] != 1)
        return fail(CBDFS_EINVAL, "a regression head has one output");
    if (d->head == CBDFS_HEAD_QUANTILE ? !(d->quantile > 0.f && d->quantile <= 1.f) : d->quantile != 0.f)
        return fail(CBDFS_EINVAL, "quantile %g (in (0, 1], and only for the quantile head)", d->quantile);
    if (!std::isfinite(d->h_offset) || (d->head != CBDFS_HEAD_REAL && d->h_offset != 0.f))
        return fail(CBDFS_EINVAL, "h_offset %g (finite, and only for the real-valued head)", d->h_offset);
    if (d->max_with_md && d->domain == CBDFS_DOM_RC3) return fail(CBDFS_EINVAL, "Manhattan distance needs a sliding-tile domain");
    for (int l = 1; l < L; ++l)
        if (d->dims[l] % 128 != 0) return fail(CBDFS_EINVAL, "hidden width %d is not a multiple of 128", d->dims[l]);
    if (d->dims[L] < 1 || d->dims[L] > 256) return fail(CBDFS_EINVAL, "output width %d outside 1..256", d->dims[L]);
    if (d->prec == CBDFS_PREC_FP8 && !d->act_scales) return fail(CBDFS_EINVAL, "FP8 needs activation scales");
    auto net = std::make_unique<NetGPU>();
    NetGPU &N = *net;
    N.domain = d->domain; N.L = L; N.prec = d->prec; N.head = d->head; N.max_with_md = d->max_with_md;
    N.h_offset = d->h_offset;
    N.quantile = d->quantile;
    for (int l = 0; l <= L; ++l) N.dims[l] = d->dims[l];
    size_t maxw = 0;
    for (int l = 1; l < L; ++l) maxw = std::max(maxw, (size_t)d->dims[l]);
    int rc = ensure_act(c, maxw);
    if (rc) return rc;
    auto upload = [&](void **dst, const void *src, size_t bytes) -> int {
        int r = dev_alloc(c, dst, bytes);
        if (r) return r;
        N.bytes += bytes;
        if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(CBDFS_EDEVICE, "weight upload");
        return CBDFS_OK;
    };
    for (int l = 0; l < L; ++l) {
        N.host_w[l].assign(d->weights[l], d->weights[l] + (size_t)d->dims[l + 1] * d->dims[l]);
        N.host_b[l].assign(d->biases[l], d->biases[l] + d->dims[l + 1]);
    }
    // FP32 copies: biases always; weights of the last layer always; all layers for FP32
    for (int l = 0; l < L; ++l) {
        const int O = d->dims[l + 1], I = d->dims[l];
        if ((rc = upload((void **)&N.b32[l], d->biases[l], sizeof(float) * O))) return rc;
        if (l == L - 1 || d->prec == CBDFS_PREC_FP32) {
            if (l == 0) {  // the gather form reads W1 transposed
                std::vector<float> t((size_t)I * O);
                for (int o = 0; o < O; ++o)
                    for (int i = 0; i < I; ++i) t[(size_t)i * O + o] = d->weights[0][(size_t)o * I + i];
                if ((rc = upload((void **)&N.w32[0], t.data(), sizeof(float) * t.size()))) return rc;
            } else if ((rc = upload((void **)&N.w32[l], d->weights[l], sizeof(float) * (size_t)O * I))) {
                return rc;
            }
        }
    }
    if (d->prec != CBDFS_PREC_FP32) {
        const bool fp8 = d->prec == CBDFS_PREC_FP8;
        const int kblk = fp8 ? 128 : 64;
        N.k1pad = (d->dims[0] + kblk - 1) / kblk * kblk;
        int w128_layers = 0;
        for (int l = 0; l < L - 1; ++l) {
            const int O = d->dims[l + 1], I = d->dims[l];
            const int Kp = l == 0 ? N.k1pad : I;
            const float *W = d->weights[l];
            std::vector<uint8_t> buf((size_t)O * Kp * (fp8 ? 1 : 2), 0);
            if (fp8) {
                float amax = 0.f;
                for (size_t i = 0; i < (size_t)O * I; ++i) amax = std::max(amax, std::fabs(W[i]));
                const float scale = amax > 0.f ? amax / 448.0f : 1.0f;
                N.w_scale[l] = scale;
                for (int o = 0; o < O; ++o)
                    for (int i = 0; i < I; ++i)
                        buf[(size_t)o * Kp + i] =
                            (uint8_t)__nv_cvt_float_to_fp8(W[(size_t)o * I + i] / scale, __NV_SATFINITE, __NV_E4M3);
                if (l < L - 1) N.a_scale[l] = d->act_scales[l];
            } else {
                N.w_scale[l] = 1.f;
                uint16_t *b16 = reinterpret_cast<uint16_t *>(buf.data());
                for (int o = 0; o < O; ++o)
                    for (int i = 0; i < I; ++i) b16[(size_t)o * Kp + i] = f32_to_bf16_rne(W[(size_t)o * I + i]);
            }
            if ((rc = upload(&N.w_lp[l], buf.data(), buf.size()))) return rc;
            N.bn[l] = (O % 256 == 0) ? 256 : 128;
            if ((rc = make_tmap_2d(&N.tm_w[l], N.w_lp[l],
                                   fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                   fp8 ? 1 : 2, (uint64_t)Kp, (uint64_t)O, kblk, N.bn[l])))
                return rc;
            if (O % kChainBNSmall == 0 &&
                (rc = make_tmap_2d(&N.tm_w64[l], N.w_lp[l],
                                   fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                   fp8 ? 1 : 2, (uint64_t)Kp, (uint64_t)O, kblk, kChainBNSmall)))
                return rc;
            if (O % kChainBN == 0 &&
                (rc = make_tmap_2d(&N.tm_w128[l], N.w_lp[l],
                                   fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                   fp8 ? 1 : 2, (uint64_t)Kp, (uint64_t)O, kblk, kChainBN / 2)))
                return rc;
            w128_layers += O % kChainBN == 0;
        }
        N.has_w128 = w128_layers == L - 1;
    }
    // the tensor-core head: a classifier of 17..128 outputs behind BF16 / E4M3 hidden layers
    // (the fused chain stores the last hidden layer in BF16 for it); W = W1 + W2 + W3 in BF16,
    // each part the rounding of what the previous ones leave (24 bits of mantissa in all)
    const int C = d->dims[L], KL = d->dims[L - 1];
    if (d->prec != CBDFS_PREC_FP32 && (d->head == CBDFS_HEAD_CLASSIFIER || d->head == CBDFS_HEAD_QUANTILE) &&
        C > kHeadTcMinC && C <= kHeadTcMaxC && KL % 64 == 0) {
        const int cpad = (C + 15) / 16 * 16;
        std::vector<uint16_t> sp((size_t)3 * cpad * KL, 0);
        for (int c = 0; c < C; ++c)
            for (int k = 0; k < KL; ++k) {
                float r = d->weights[L - 1][(size_t)c * KL + k];
                for (int part = 0; part < 3; ++part) {
                    const uint16_t b16 = f32_to_bf16_rne(r);
                    sp[((size_t)part * cpad + c) * KL + k] = b16;
                    float back;
                    const uint32_t u = (uint32_t)b16 << 16;
                    memcpy(&back, &u, 4);
                    r -= back;  // exact: r and its BF16 rounding are within a factor of two
                }
            }
        if ((rc = upload(&N.w_split, sp.data(), sp.size() * 2))) return rc;
        if ((rc = make_tmap_2d(&N.tm_wsplit, N.w_split, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)KL,
                               (uint64_t)3 * cpad, 64, cpad)))
            return rc;
        N.head_cpad = cpad;
    }
    if ((size_t)d->dims[L] * 4 * 4 > 48 * 1024) return fail(CBDFS_EINVAL, "output width too large");
    if (chain_ok(N) && (rc = ensure_chain(c, chain_partial_floats(N)))) return rc;
    c->nets.push_back(std::move(net));
    c->heur_kind.push_back(0);
    c->heur_index.push_back((int)c->nets.size() - 1);
    *heur_id = (int)c->heur_kind.size() - 1;
    return CBDFS_OK;
}

// Replace the full table *t (n entries, on the device) by its DIV compression by k.
static int div_compress_table(Ctx *c, uint8_t **t, size_t n, uint32_t k, size_t *entries, cudaStream_t st) {
    const size_t m = (n + k - 1) / k;
    uint8_t *d = nullptr;
    int rc = dev_alloc(c, (void **)&d, m);
    if (rc) return rc;
    if ((rc = pdb_div_compress(*t, n, k, d, st)) || cudaStreamSynchronize(st) != cudaSuccess) {
        dev_free(c, d, m);
        return rc ? rc : fail(CBDFS_EDEVICE, "DIV compression");
    }
    dev_free(c, *t, n);
    *t = d;
    *entries = m;
    return CBDFS_OK;
}

// the cube's one pattern: the eight corner cubies 0..7 in order (the 8-corner PDB)
static int check_rc_corner_pattern(int n_patterns, const int *k, const int *tiles) {
    if (n_patterns != 1 || k[0] != 8) return fail(CBDFS_EINVAL, "the cube's PDB is one pattern of the 8 corners");
    for (int i = 0; i < 8; ++i)
        if (tiles[i] != i) return fail(CBDFS_EINVAL, "the cube's corner pattern lists cubies 0..7 in order");
    return CBDFS_OK;
}

int cbdfs_pdb_load(cbdfs_ctx *ctx, const cbdfs_pdb_desc *d, int *heur_id) {
    if (!ctx || !d || !heur_id || !d->k || !d->tiles) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (c->server) return fail(CBDFS_EINVAL, "stop the server before loading a heuristic");
    CUDA_TRY(cudaSetDevice(c->device));
    if (d->domain < 0 || d->domain > 2) return fail(CBDFS_EINVAL, "domain %d", d->domain);
    if (d->n_patterns < 1 || d->n_patterns > 4) return fail(CBDFS_EINVAL, "n_patterns %d outside 1..4", d->n_patterns);
    if (d->div < 0) return fail(CBDFS_EINVAL, "div %d", d->div);
    const uint32_t div = d->div > 1 ? (uint32_t)d->div : 1u;
    if (d->domain == CBDFS_DOM_RC3) {
        int rc = check_rc_corner_pattern(d->n_patterns, d->k, d->tiles);
        if (rc) return rc;
        auto p = std::make_unique<PdbGPU>();
        p->domain = d->domain;
        p->n_patterns = 1;
        p->k[0] = 8;
        for (int i = 0; i < 8; ++i) p->tiles[0][i] = i;
        p->entries[0] = rc_corner_entries();
        if ((rc = dev_alloc(c, (void **)&p->table[0], p->entries[0]))) return rc;
        p->bytes = p->entries[0];
        if (d->tables && d->tables[0]) {
            CUDA_TRY(cudaMemcpy(p->table[0], d->tables[0], p->entries[0], cudaMemcpyHostToDevice));
        } else if ((rc = rc_corner_build_device(c, p->table[0], c->slots[0].stream))) {
            return rc;
        }
        if (div > 1) {
            if ((rc = div_compress_table(c, &p->table[0], p->entries[0], div, &p->entries[0], c->slots[0].stream)))
                return rc;
            p->bytes = p->entries[0];
            p->div = div;
        }
        c->pdbs.push_back(std::move(p));
        c->heur_kind.push_back(1);
        c->heur_index.push_back((int)c->pdbs.size() - 1);
        *heur_id = (int)c->heur_kind.size() - 1;
        return CBDFS_OK;
    }
    auto p = std::make_unique<PdbGPU>();
    p->domain = d->domain;
    p->side = dom_side(d->domain);
    p->n_patterns = d->n_patterns;
    const int N = p->side * p->side;
    int off = 0;
    uint32_t used = 0;
    for (int q = 0; q < d->n_patterns; ++q) {
        if (d->k[q] < 1 || d->k[q] > 8) return fail(CBDFS_EINVAL, "pattern size %d outside 1..8", d->k[q]);
        p->k[q] = d->k[q];
        for (int i = 0; i < d->k[q]; ++i) {
            const int t = d->tiles[off + i];
            if (t < 1 || t >= N || (used & (1u << t))) return fail(CBDFS_EINVAL, "bad or repeated tile %d", t);
            used |= 1u << t;
            p->tiles[q][i] = t;
        }
        off += d->k[q];
        p->entries[q] = npk(N, d->k[q]);
        int rc = dev_alloc(c, (void **)&p->table[q], p->entries[q]);
        if (rc) return rc;
        p->bytes += p->entries[q];
        if (d->tables && d->tables[q]) {
            CUDA_TRY(cudaMemcpy(p->table[q], d->tables[q], p->entries[q], cudaMemcpyHostToDevice));
        } else {
            rc = pdb_build_device(c, p->side, p->tiles[q], p->k[q], p->table[q], c->slots[0].stream);
            if (rc) return rc;
        }
        if (div > 1) {
            p->bytes -= p->entries[q];
            if ((rc = div_compress_table(c, &p->table[q], p->entries[q], div, &p->entries[q], c->slots[0].stream)))
                return rc;
            p->bytes += p->entries[q];
        }
    }
    p->div = div;
    c->pdbs.push_back(std::move(p));
    c->heur_kind.push_back(1);
    c->heur_index.push_back((int)c->pdbs.size() - 1);
    *heur_id = (int)c->heur_kind.size() - 1;
    return CBDFS_OK;
}

// A group's networks as one grouped network, when they are two or more BF16 networks of one
// shape with the tensor-core head: weights and biases stacked by member (device copies).
// Returns with *out null when the group does not qualify.
static int fuse_group(Ctx *c, const int *ids, int k, std::unique_ptr<NetGPU> *out) {
    out->reset();
    if (k < 2) return CBDFS_OK;
    for (int j = 0; j < k; ++j)
        if (ids[j] < 0 || c->heur_kind[ids[j]] != 0) return CBDFS_OK;
    const NetGPU &a = *c->nets[c->heur_index[ids[0]]];
    if (a.prec != CBDFS_PREC_BF16 || !a.head_cpad || !chain_ok(a)) return CBDFS_OK;
    for (int j = 1; j < k; ++j) {
        const NetGPU &b = *c->nets[c->heur_index[ids[j]]];
        if (b.domain != a.domain || b.L != a.L || b.prec != a.prec || b.head != a.head || b.quantile != a.quantile ||
            b.max_with_md != a.max_with_md || b.head_cpad != a.head_cpad || b.k1pad != a.k1pad)
            return CBDFS_OK;
        for (int l = 0; l <= a.L; ++l)
            if (b.dims[l] != a.dims[l]) return CBDFS_OK;
    }
    auto f = std::make_unique<NetGPU>();
    NetGPU &F = *f;
    const int L = a.L, E = k;
    F.domain = a.domain; F.L = L; F.prec = a.prec; F.head = a.head; F.quantile = a.quantile;
    F.max_with_md = a.max_with_md; F.k1pad = a.k1pad; F.head_cpad = a.head_cpad; F.groups = E;
    F.dims[0] = a.dims[0];
    for (int l = 1; l < L; ++l) F.dims[l] = E * a.dims[l];
    F.dims[L] = a.dims[L];
    auto stack = [&](void **dst, size_t each, auto member_ptr) -> int {
        int rc = dev_alloc(c, dst, each * E);
        if (rc) return rc;
        F.bytes += each * E;
        for (int j = 0; j < E; ++j)
            CUDA_TRY(cudaMemcpy(static_cast<uint8_t *>(*dst) + each * j, member_ptr(*c->nets[c->heur_index[ids[j]]]),
                                each, cudaMemcpyDeviceToDevice));
        return CBDFS_OK;
    };
    int rc;
    size_t maxw = 0;
    for (int l = 0; l < L - 1; ++l) {
        const int O = a.dims[l + 1], Kp = l == 0 ? a.k1pad : a.dims[l];
        if ((rc = stack(&F.w_lp[l], (size_t)O * Kp * 2, [&](const NetGPU &n) { return n.w_lp[l]; }))) return rc;
        if ((rc = stack((void **)&F.b32[l], (size_t)O * 4, [&](const NetGPU &n) { return (const void *)n.b32[l]; })))
            return rc;
        F.w_scale[l] = F.a_scale[l] = 1.f;
        F.bn[l] = a.bn[l];
        if ((rc = make_tmap_2d(&F.tm_w[l], F.w_lp[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)Kp, (uint64_t)E * O,
                               64, F.bn[l])) ||
            (rc = make_tmap_2d(&F.tm_w64[l], F.w_lp[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)Kp,
                               (uint64_t)E * O, 64, kChainBNSmall)) ||
            (rc = make_tmap_2d(&F.tm_w128[l], F.w_lp[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)Kp,
                               (uint64_t)E * O, 64, kChainBN / 2)))
            return rc;
        maxw = std::max(maxw, (size_t)E * O);
    }
    F.has_w128 = true;  // the grouped network runs on the chain only (every hidden width a multiple of 256)
    const int C = a.dims[L], KL = a.dims[L - 1], cpad = a.head_cpad;
    if ((rc = stack(&F.w_split, (size_t)3 * cpad * KL * 2, [&](const NetGPU &n) { return (const void *)n.w_split; })) ||
        (rc = stack((void **)&F.b32[L - 1], (size_t)C * 4, [&](const NetGPU &n) { return (const void *)n.b32[L - 1]; })))
        return rc;
    if ((rc = make_tmap_2d(&F.tm_wsplit, F.w_split, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)KL,
                           (uint64_t)E * 3 * cpad, 64, cpad)))
        return rc;
    if ((rc = ensure_act(c, maxw)) || (rc = ensure_chain(c, 0))) return rc;
    *out = std::move(f);
    return CBDFS_OK;
}

int cbdfs_combo_load(cbdfs_ctx *ctx, const cbdfs_combo_desc *d, int *heur_id) {
    if (!ctx || !d || !heur_id || !d->group_size || !d->members) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (c->server) return fail(CBDFS_EINVAL, "stop the server before loading a heuristic");
    if (d->domain < 0 || d->domain > 2) return fail(CBDFS_EINVAL, "domain %d", d->domain);
    if (d->n_groups < 1 || d->n_groups > kComboMaxGroups)
        return fail(CBDFS_EINVAL, "n_groups %d outside 1..%d", d->n_groups, kComboMaxGroups);
    if (d->add_md && d->domain == CBDFS_DOM_RC3) return fail(CBDFS_EINVAL, "Manhattan distance needs a sliding-tile domain");
    auto cb = std::make_unique<ComboGPU>();
    cb->domain = d->domain;
    cb->P.n_groups = d->n_groups;
    cb->P.add_md = d->add_md ? 1 : 0;
    int total = 0;
    for (int grp = 0; grp < d->n_groups; ++grp) {
        const int k = d->group_size[grp];
        if (k < 1 || k > kComboMaxMembers) return fail(CBDFS_EINVAL, "group size %d outside 1..%d", k, kComboMaxMembers);
        cb->P.group_size[grp] = k;
        for (int j = 0; j < k; ++j) {
            const int id = d->members[total + j];
            if (id >= (int)c->heur_kind.size() || id < CBDFS_HEUR_MD || (id == CBDFS_HEUR_MD && d->domain == CBDFS_DOM_RC3))
                return fail(CBDFS_EINVAL, "member heuristic id %d", id);
            if (id >= 0 && c->heur_kind[id] == 2) return fail(CBDFS_EINVAL, "member %d is itself a composite", id);
            if (heur_is_real(c, id)) return fail(CBDFS_EINVAL, "member %d is real-valued", id);
            const int dom = id < 0 ? d->domain
                            : c->heur_kind[id] == 0 ? c->nets[c->heur_index[id]]->domain
                                                    : c->pdbs[c->heur_index[id]]->domain;
            if (dom != d->domain) return fail(CBDFS_EINVAL, "member %d is for another domain", id);
            cb->members.push_back(id);
        }
        total += k;
        if (total > kComboMaxTotal) return fail(CBDFS_EINVAL, "more than %d members", kComboMaxTotal);
    }
    CUDA_TRY(cudaSetDevice(c->device));
    for (int grp = 0, m = 0; grp < cb->P.n_groups; m += cb->P.group_size[grp++]) {
        int rc = fuse_group(c, cb->members.data() + m, cb->P.group_size[grp], &cb->fused[grp]);
        if (rc) return rc;
    }
    for (auto &s : c->slots)
        if (!s.combo) {
            int rc = dev_alloc(c, (void **)&s.combo, combo_bytes(c));
            if (rc) return rc;
            ++c->buf_gen;
        }
    c->combos.push_back(std::move(cb));
    c->heur_kind.push_back(2);
    c->heur_index.push_back((int)c->combos.size() - 1);
    *heur_id = (int)c->heur_kind.size() - 1;
    return CBDFS_OK;
}

int pdb_build(cbdfs_ctx *ctx, int domain, const int *pattern_tiles, int k, uint8_t *table_out,
              size_t cap, size_t *entries) {
    if (!ctx || !pattern_tiles || !table_out || !entries) return fail(CBDFS_EINVAL, "null argument");
    if (domain < 0 || domain > 2) return fail(CBDFS_EINVAL, "domain %d", domain);
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    CUDA_TRY(cudaSetDevice(c->device));
    if (domain == CBDFS_DOM_RC3) {
        int rc = check_rc_corner_pattern(1, &k, pattern_tiles);
        if (rc) return rc;
        const size_t E = rc_corner_entries();
        *entries = E;
        if (cap < E) return fail(CBDFS_EINVAL, "table buffer holds %zu bytes, %zu needed", cap, E);
        uint8_t *d_tab = nullptr;
        if ((rc = dev_alloc(c, (void **)&d_tab, E))) return rc;
        rc = rc_corner_build_device(c, d_tab, c->slots[0].stream);
        if (!rc && cudaMemcpy(table_out, d_tab, E, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = fail(CBDFS_EDEVICE, "table download");
        dev_free(c, d_tab, E);
        return rc;
    }
    const int side = dom_side(domain), N = side * side;
    if (k < 1 || k > 8) return fail(CBDFS_EINVAL, "pattern size %d outside 1..8", k);
    uint32_t used = 0;
    for (int i = 0; i < k; ++i) {
        const int t = pattern_tiles[i];
        if (t < 1 || t >= N || (used & (1u << t))) return fail(CBDFS_EINVAL, "bad or repeated tile %d", t);
        used |= 1u << t;
    }
    const size_t P = npk(N, k);
    *entries = P;
    if (cap < P) return fail(CBDFS_EINVAL, "table buffer holds %zu bytes, %zu needed", cap, P);
    uint8_t *d_tab = nullptr;
    int rc = dev_alloc(c, (void **)&d_tab, P);
    if (rc) return rc;
    rc = pdb_build_device(c, side, pattern_tiles, k, d_tab, c->slots[0].stream);
    if (!rc && cudaMemcpy(table_out, d_tab, P, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = fail(CBDFS_EDEVICE, "table download");
    dev_free(c, d_tab, P);
    return rc;
}

// real: the call is one of the *_real entry points (which take exactly the real-valued heads)
static int check_eval_args(Ctx *c, int heur_id, int domain, uint32_t n, bool real = false) {
    if (domain < 0 || domain > 2) return fail(CBDFS_EINVAL, "domain %d", domain);
    if (n > c->max_batch) return fail(CBDFS_EINVAL, "n=%u exceeds max_batch=%u", n, c->max_batch);
    if (heur_id >= (int)c->heur_kind.size() || heur_id < CBDFS_HEUR_MD)
        return fail(CBDFS_EINVAL, "unknown heuristic id %d", heur_id);
    if (heur_id == CBDFS_HEUR_MD && domain == CBDFS_DOM_RC3)
        return fail(CBDFS_EINVAL, "Manhattan distance is defined for sliding-tile domains only");
    if (heur_is_real(c, heur_id) != real)
        return fail(CBDFS_EINVAL, real ? "heuristic %d is not real-valued" : "heuristic %d is real-valued: use the *_real calls",
                    heur_id);
    return CBDFS_OK;
}

// an FP32 bound as the kernels' key (its bit pattern; f >= 0 orders like the key)
static int real_bound_key(float bound, uint32_t *key) {
    if (!(bound >= 0.f)) return fail(CBDFS_EINVAL, "bound %g: a real bound is >= 0 and not NaN", bound);
    memcpy(key, &bound, 4);
    return CBDFS_OK;
}

static int eval_device(Ctx *c, int heur_id, int domain, const uint64_t *d_states, const uint8_t *d_g,
                       uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask, uint32_t *d_minf,
                       float *d_y, void *stream) {
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    Slot &s = c->slots[0];
    // slot 0 owns this call's activation scratch; order the call after its last use (a call
    // being captured into a CUDA graph is ordered by the graph instead)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (!capturing) CUDA_TRY(cudaStreamWaitEvent(st, s.done, 0));
    int rc = run_eval(c, s, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, d_y, st);
    if (!capturing) CUDA_TRY(cudaEventRecord(s.done, st));
    return rc;
}

int heur_eval_device(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states, const uint8_t *d_g,
                     uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask, uint32_t *d_minf,
                     float *d_y, void *stream) {
    if (!ctx || !d_minf || (n && (!d_states || !d_g || !d_h || !d_mask))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    int rc = check_eval_args(c, heur_id, domain, n);
    if (rc) return rc;
    return eval_device(c, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, d_y, stream);
}

int heur_eval_device_real(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                          const uint8_t *d_g, float bound, uint32_t n, float *d_h, uint32_t *d_mask,
                          float *d_minf, void *stream) {
    if (!ctx || !d_minf || (n && (!d_states || !d_g || !d_h || !d_mask))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    uint32_t key;
    int rc = check_eval_args(c, heur_id, domain, n, true);
    if (rc || (rc = real_bound_key(bound, &key))) return rc;
    // the real h goes where the raw outputs would; no uint8 h
    return eval_device(c, heur_id, domain, d_states, d_g, key, n, nullptr, d_mask,
                       reinterpret_cast<uint32_t *>(d_minf), d_h, stream);
}

// the device address of page-locked host memory (cudaMallocHost / cudaHostRegister), else false
static bool host_mapped(const void *p, void **dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

// One host-buffer batch on a free slot (slots 1..).  h8: uint8 h (null for a real-valued
// head); yf: C floats per row (the raw outputs, or for a real-valued head its h, C = 1), or
// null.  *minf_key receives the least f above the bound as the kernels' key.
// ticket_out != null: return once the batch is enqueued (the slot stays held; heur_wait finishes
// the call and releases it)
static int submit_host(Ctx *c, int heur_id, int domain, const uint64_t *states, const uint8_t *g,
                       uint32_t bound, uint32_t n, uint8_t *h8, uint32_t *mask_out, uint32_t *minf_key,
                       float *yf, int C, uint64_t *ticket_out = nullptr) {
    CUDA_TRY(cudaSetDevice(c->device));
    int si;
    {
        std::unique_lock<std::mutex> lk(c->slot_mu);
        for (;;) {
            si = -1;
            for (int i = 1; i < (int)c->slots.size(); ++i)
                if (!c->slots[i].busy) { si = i; break; }
            if (si >= 0) break;
            c->slot_cv.wait(lk);
        }
        c->slots[si].busy = true;
    }
    Slot &s = c->slots[si];
    cudaStream_t st = s.stream;
    const int w = dom_words(domain);
    int rc = CBDFS_OK;
    // Page-locked caller buffers are read and written by the kernels in place (mapped host
    // memory, over the bus inside the launch); other buffers go through the slot's device
    // staging with copies.
    void *zs = nullptr, *zg = nullptr, *zh = nullptr, *zm = nullptr, *zy = nullptr;
    const bool zero_copy = n && host_mapped(states, &zs) && host_mapped(g, &zg) && host_mapped(mask_out, &zm) &&
                           (!h8 || host_mapped(h8, &zh)) && (!yf || host_mapped(yf, &zy)) &&
                           (domain != CBDFS_DOM_RC3 || !(reinterpret_cast<uintptr_t>(zs) & 15u));
    float *d_y = nullptr;
    if (!zero_copy && yf && n) rc = dev_alloc(c, (void **)&d_y, (size_t)n * C * 4 + 4);
    if (zero_copy) {
        rc = run_eval(c, s, heur_id, domain, static_cast<const uint64_t *>(zs), static_cast<const uint8_t *>(zg),
                      bound, n, static_cast<uint8_t *>(zh), static_cast<uint32_t *>(zm), s.d_minf,
                      static_cast<float *>(zy), st);
    } else {
        if (!rc && n) {
            if (cudaMemcpyAsync(s.d_states, states, (size_t)n * 8 * w, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(s.d_g, g, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = fail(CBDFS_EDEVICE, "batch upload");
        }
        if (!rc)
            rc = run_eval(c, s, heur_id, domain, s.d_states, s.d_g, bound, n, h8 ? s.d_h : nullptr, s.d_mask,
                          s.d_minf, d_y, st);
        if (!rc && n) {
            if ((h8 && cudaMemcpyAsync(h8, s.d_h, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
                cudaMemcpyAsync(mask_out, s.d_mask, (size_t)(n + 31) / 32 * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                (d_y && cudaMemcpyAsync(yf, d_y, (size_t)n * C * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess))
                rc = fail(CBDFS_EDEVICE, "result download");
        }
    }
    // the least f above the bound and the device error flag, read in stream order
    if (!rc && (cudaMemcpyAsync(s.h_small, s.d_minf, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(s.h_small + 1, c->d_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = fail(CBDFS_EDEVICE, "result download");
    if (ticket_out && !rc && !d_y) {
        if (cudaEventRecord(s.done, st) != cudaSuccess) {
            rc = fail(CBDFS_EDEVICE, "event record");
        } else {
            std::lock_guard<std::mutex> lk(c->pending_mu);
            *ticket_out = c->next_ticket++;
            c->pending[*ticket_out] = Ctx::Pending{si, minf_key};
            return CBDFS_OK;
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = fail(CBDFS_EDEVICE, "evaluation: %s", cudaGetErrorString(e));
    if (d_y) dev_free(c, d_y, (size_t)n * C * 4 + 4);
    if (!rc) {
        *minf_key = s.h_small[0];
        if (s.h_small[1]) rc = fail(CBDFS_ETIMEDOUT, "a device wait ran out (code %d)", (int)s.h_small[1]);
    }
    {
        std::lock_guard<std::mutex> lk(c->slot_mu);
        s.busy = false;
    }
    c->slot_cv.notify_one();
    return rc;
}

int heur_submit_batch(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states, const uint8_t *g,
                      uint32_t bound, uint32_t n, uint8_t *h_out, uint32_t *mask_out, uint32_t *minf_out,
                      float *y_out) {
    if (!ctx || !minf_out || (n && (!states || !g || !h_out || !mask_out))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    int rc = check_eval_args(c, heur_id, domain, n);
    if (rc) return rc;
    int C = 0;
    if (y_out && heur_id >= 0 && c->heur_kind[heur_id] == 0) {
        const NetGPU &net = *c->nets[c->heur_index[heur_id]];
        C = net.dims[net.L];
    }
    return submit_host(c, heur_id, domain, states, g, bound, n, h_out, mask_out, minf_out, C ? y_out : nullptr, C);
}

int heur_submit_batch_async(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states, const uint8_t *g,
                            uint32_t bound, uint32_t n, uint8_t *h_out, uint32_t *mask_out, uint32_t *minf_out,
                            cbdfs_ticket *t) {
    if (!ctx || !minf_out || !t || (n && (!states || !g || !h_out || !mask_out))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    int rc = check_eval_args(c, heur_id, domain, n);
    if (rc) return rc;
    uint64_t id = 0;
    rc = submit_host(c, heur_id, domain, states, g, bound, n, h_out, mask_out, minf_out, nullptr, 0, &id);
    t->id = id;
    return rc;
}

int heur_wait(cbdfs_ctx *ctx, cbdfs_ticket t, uint64_t timeout_us) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Ctx::Pending p;
    {
        std::lock_guard<std::mutex> lk(c->pending_mu);
        auto it = c->pending.find(t.id);
        if (it == c->pending.end()) return fail(CBDFS_EINVAL, "unknown or collected ticket %llu", (unsigned long long)t.id);
        p = it->second;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    Slot &s = c->slots[p.slot];
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t q;
    while ((q = cudaEventQuery(s.done)) == cudaErrorNotReady) {
        if (timeout_us && std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(timeout_us))
            return fail(CBDFS_ETIMEDOUT, "ticket %llu still running", (unsigned long long)t.id);
        std::this_thread::yield();
    }
    int rc = q == cudaSuccess ? CBDFS_OK : fail(CBDFS_EDEVICE, "evaluation: %s", cudaGetErrorString(q));
    if (!rc) {
        *p.minf_out = s.h_small[0];
        if (s.h_small[1]) rc = fail(CBDFS_ETIMEDOUT, "a device wait ran out (code %d)", (int)s.h_small[1]);
    }
    {
        std::lock_guard<std::mutex> lk(c->pending_mu);
        c->pending.erase(t.id);
    }
    {
        std::lock_guard<std::mutex> lk(c->slot_mu);
        s.busy = false;
    }
    c->slot_cv.notify_one();
    return rc;
}

int heur_submit_batch_real(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states, const uint8_t *g,
                           float bound, uint32_t n, float *h_out, uint32_t *mask_out, float *minf_out) {
    if (!ctx || !minf_out || (n && (!states || !g || !h_out || !mask_out))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    uint32_t key, mkey = 0xFFFFFFFFu;
    int rc = check_eval_args(c, heur_id, domain, n, true);
    if (rc || (rc = real_bound_key(bound, &key))) return rc;
    rc = submit_host(c, heur_id, domain, states, g, key, n, nullptr, mask_out, &mkey, h_out, 1);
    if (rc) return rc;
    if (mkey == 0xFFFFFFFFu) *minf_out = INFINITY;
    else memcpy(minf_out, &mkey, 4);
    return CBDFS_OK;
}

int cbdfs_eval_profile(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                       const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask,
                       uint32_t *d_minf, void *stream, float *stage_ms, int cap, int *n_stages) {
    if (!ctx || !stage_ms || !n_stages || !d_minf || (n && (!d_states || !d_g || !d_h || !d_mask)))
        return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    int rc = check_eval_args(c, heur_id, domain, n);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    Slot &s = c->slots[0];
    std::vector<cudaEvent_t> evs;
    CUDA_TRY(cudaStreamWaitEvent(st, s.done, 0));
    s.prof = &evs;
    rc = run_eval(c, s, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, nullptr, st);
    s.prof = nullptr;
    if (!rc && cudaEventRecord(s.done, st) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "event record");
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "profile sync");
    *n_stages = 0;
    for (size_t i = 1; i < evs.size() && !rc; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, evs[i - 1], evs[i]) != cudaSuccess) {
            rc = fail(CBDFS_EDEVICE, "event timing");
            break;
        }
        if (*n_stages < cap) stage_ms[(*n_stages)++] = ms;
    }
    for (auto e : evs) cudaEventDestroy(e);
    return rc;
}

int cbdfs_eval_trace(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states, const uint8_t *d_g,
                     uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask, uint32_t *d_minf,
                     void *stream, uint64_t *d_trace, int tiles_per_cta, int *ctas) {
    if (!ctx || !d_trace || !ctas || tiles_per_cta < 1 || !d_minf || (n && (!d_states || !d_g || !d_h || !d_mask)))
        return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    int rc = check_eval_args(c, heur_id, domain, n);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(c->device_call_mu);
    Slot &s = c->slots[0];
    CUDA_TRY(cudaStreamWaitEvent(st, s.done, 0));
    *ctas = 0;
    s.trace = reinterpret_cast<unsigned long long *>(d_trace);
    s.trace_tiles = tiles_per_cta;
    s.trace_grid = ctas;
    rc = run_eval(c, s, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, nullptr, st);
    s.trace = nullptr;
    s.trace_grid = nullptr;
    if (!rc && cudaEventRecord(s.done, st) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "event record");
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "trace sync");
    return rc;
}

int cbdfs_debug_withhold_publish(cbdfs_ctx *ctx, int row_block) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    reinterpret_cast<Ctx *>(ctx)->hold_mblock.store(row_block < 0 ? -1 : row_block);
    return CBDFS_OK;
}

int cbdfs_device_status(cbdfs_ctx *ctx) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    int flag = 0;
    CUDA_TRY(cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        // a wait that ran out may have left chain counts behind: zero every slot's counters
        for (Slot &s : c->slots)
            if (s.counters) CUDA_TRY(cudaMemset(s.counters, 0, sizeof(int) * chain_counter_ints(c)));
    }
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    return flag;
}

}  // extern "C"
