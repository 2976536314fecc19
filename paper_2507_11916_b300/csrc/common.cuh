// common.cuh -- internal declarations shared by the library's translation units:
// the context, the loaded heuristics, the device-side PTX wrappers (mbarrier, TMA,
// tcgen05) and the packed-state decoders.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cbdfs.h"

namespace cbdfs {

// ------------------------------------------------------------------------------------
// host-side error plumbing
// ------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return ::cbdfs::fail(CBDFS_EDEVICE, "%s failed: %s (%s:%d)", #expr,          \
                                 cudaGetErrorString(_e), __FILE__, __LINE__);            \
    } while (0)

// device error codes written to the context's flag by a wait that ran out
enum DevErr : int {
    DEVERR_NONE = 0,
    DEVERR_TMA_FULL = 1,     // MMA issuer waited for a TMA stage
    DEVERR_STAGE_EMPTY = 2,  // producer waited for the MMA to free a stage
    DEVERR_ACCUM = 3,        // epilogue waited for the accumulator
    DEVERR_ENCODE = 4,
    DEVERR_DEPENDENCY = 5,   // a chain tile waited for the previous layer's row block
};

// ------------------------------------------------------------------------------------
// loaded heuristics
// ------------------------------------------------------------------------------------
constexpr int kMaxLayers = 8;
constexpr int kBM = 128;  // rows (states) per tensor-core tile

struct TrainState;  // train.cu
void train_free(struct Ctx *c, TrainState *T);

struct NetGPU {
    int domain = 0, L = 0, prec = 0, head = 0, max_with_md = 0;
    float h_offset = 0.f;              // CBDFS_HEAD_REAL: added to y
    float quantile = 0.f;              // CBDFS_HEAD_QUANTILE: the CDF level
    // the head's parameter as the final kernels take it (the offset, or the quantile)
    float head_param() const { return head == CBDFS_HEAD_QUANTILE ? quantile : h_offset; }
    int dims[kMaxLayers + 1] = {};
    int k1pad = 0;                     // one-hot width padded to the MMA K block
    // tensor-core layers 0..L-2: low-precision weights [dims[l+1]][Kpad] (K-major)
    void *w_lp[kMaxLayers] = {};
    float w_scale[kMaxLayers] = {};    // FP8: weight scale per layer (1 for BF16)
    float a_scale[kMaxLayers] = {};    // FP8: activation scale of layer l's OUTPUT
    CUtensorMap tm_w[kMaxLayers];      // TMA maps of w_lp (k-block x bn rows)
    CUtensorMap tm_w64[kMaxLayers];    // the same with 64-row boxes (small-batch chain tiles)
    CUtensorMap tm_w128[kMaxLayers];   // the same with 128-row boxes (a CTA pair's half of a tile)
    bool has_w128 = false;             // tm_w128 is built for every hidden layer (CTA pairs allowed)
    int bn[kMaxLayers] = {};           // N tile per layer
    // classifier heads of 17..128 outputs on a BF16/E4M3 network: the last layer split into three
    // BF16 parts [3][head_cpad][K] for the tensor-core head (head_cpad = 0: none)
    void *w_split = nullptr;
    CUtensorMap tm_wsplit;
    int head_cpad = 0;
    // an ensemble run as one network (composite heuristics): `groups` members stacked along
    // every hidden width, each hidden layer after the first grouped (a member reads only its
    // own columns); dims[1..L-1] are the stacked widths, dims[L] one member's outputs
    int groups = 1;
    // FP32 weights for every layer (the FP32 path; the last layer for every path)
    float *w32[kMaxLayers] = {};
    float *b32[kMaxLayers] = {};
    size_t bytes = 0;
    // FP32 weights as loaded (host), the training masters' starting point
    std::vector<float> host_w[kMaxLayers], host_b[kMaxLayers];
    TrainState *train = nullptr;
};

struct PdbGPU {
    int domain = 0, side = 0, n_patterns = 0;
    int k[4] = {}, tiles[4][16] = {};
    uint8_t *table[4] = {};
    size_t entries[4] = {};            // stored entries (after DIV compression)
    uint32_t div = 1;                  // DIV compression: entry = min over div adjacent ranks
    size_t bytes = 0;
};

// the additive PDB gather's parameters (pdb.cu): per pattern its tiles, rank weights and table
struct PdbParams {
    int n_patterns;
    int k[4];
    int tiles[4][8];
    uint32_t weight[4][8];   // (N-1-i)! / (N-k)!
    uint32_t entries[4];     // table sizes: N!/(N-k)!, or ceil of that / div
    uint32_t div;            // DIV compression of every table (1: none)
    const uint8_t *table[4];
    uint32_t l2_keep;        // bit q: table q's lines are kept in L2 (evict-last), the other
                             // tables' lines go first (evict-first); 0: no priorities
};

// composite heuristic: [MD] + sum over groups of the minimum over each group's members
constexpr int kComboMaxGroups = 4, kComboMaxMembers = 8, kComboMaxTotal = 16;
struct ComboParams {
    int n_groups;
    int group_size[kComboMaxGroups];
    int add_md;
};
struct ComboGPU {
    int domain = 0;
    ComboParams P{};
    std::vector<int> members;          // heuristic ids, group by group
    // per group: its networks run as one grouped network (null: the members one by one)
    std::unique_ptr<NetGPU> fused[kComboMaxGroups];
};

// one evaluation slot: a stream plus the scratch a batch needs
struct Slot {
    cudaStream_t stream = nullptr;
    void *act[2] = {};                 // ping-pong activations (max_batch_pad x max_width x 4 B)
    uint64_t *d_states = nullptr;      // staging for host-buffer calls
    uint8_t *d_g = nullptr, *d_h = nullptr;
    uint32_t *d_mask = nullptr, *d_minf = nullptr;
    float *d_y = nullptr;
    uint32_t *h_small = nullptr;       // pinned host words: [0] minf, [1] the device error flag
    // TMA maps of the activation buffers, keyed by (buffer, width, dtype bytes)
    std::map<long long, CUtensorMap> tm_act;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<cudaEvent_t> *prof = nullptr;  // when set, an event follows every launch
    // fused-chain scratch (null: the per-layer kernels are used)
    int *counters = nullptr;           // tile counts per (layer, row block) + head counts
    float *partial = nullptr;          // head partials [n-tiles][rows][C]
    void *onehot = nullptr;            // one-hot input rows [max_batch_pad][1 KB]
    size_t partial_bytes = 0;
    // composite heuristics: member h rows [kComboMaxTotal][max_batch_pad], then a member
    // mask [max_batch_pad / 32] and minf word (written by the members, not read)
    uint8_t *combo = nullptr;
    // when set, the fused chain stamps its tile timeline here (see cbdfs_eval_trace)
    unsigned long long *trace = nullptr;
    int trace_tiles = 0;
    int *trace_grid = nullptr;
};

struct Server;  // serve.cpp
void server_free(struct Ctx *c, Server *S);

struct Ctx {
    int device = 0;
    size_t mem_budget = 0, mem_used = 0;
    uint32_t max_batch = 0, max_batch_pad = 0;
    size_t act_bytes = 0;              // bytes per activation buffer
    int *d_err = nullptr;              // device error flag
    uint64_t wait_ns = 0;              // bound on each fused-kernel wait (cbdfs_config.device_wait_ns)
    std::atomic<int> hold_mblock{-1};  // cbdfs_debug_withhold_publish: the next chain launch's held row block
    std::vector<std::unique_ptr<NetGPU>> nets;    // heur ids 0..: nets and PDBs interleaved
    std::vector<std::unique_ptr<PdbGPU>> pdbs;
    std::vector<std::unique_ptr<ComboGPU>> combos;
    std::vector<int> heur_kind;        // 0 = net, 1 = pdb, 2 = composite
    std::vector<int> heur_index;
    std::vector<Slot> slots;
    std::mutex slot_mu;
    std::condition_variable slot_cv;
    std::mutex device_call_mu;         // heur_eval_device scratch (slot 0)
    std::atomic<int> cancel{0};
    size_t max_width = 0;
    size_t partial_floats = 0;         // per-row head partials the chain scratch holds
    int num_sms = 0;
    uint64_t buf_gen = 0;              // bumped whenever slot scratch moves (captured graphs hold its pointers)
    // heur_submit_batch_async: tickets of batches still holding their slot
    struct Pending {
        int slot;
        uint32_t *minf_out;
    };
    std::mutex pending_mu;
    std::map<uint64_t, Pending> pending;
    uint64_t next_ticket = 1;
    Server *server = nullptr;
};

// allocation through the context's budget
int dev_alloc(Ctx *c, void **p, size_t bytes);
void dev_free(Ctx *c, void *p, size_t bytes);

// TMA map creation (driver entry point fetched once)
int make_tmap_2d(CUtensorMap *map, void *base, CUtensorMapDataType dt, int elem_bytes,
                 uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer,
                 CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B);

// the evaluation pipeline on a stream with a slot's scratch (device pointers)
int run_eval(Ctx *c, Slot &s, int heur_id, int domain, const uint64_t *d_states,
             const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h, uint32_t *d_mask,
             uint32_t *d_minf, float *d_y, cudaStream_t st);

// the bound test of the requests packed into one served launch, each starting on a 32-row
// boundary (segbound.cu): word w of the mask is request word_req[w]'s (0xFFFF: padding), its
// rows end at req_end and pass at g + h <= req_bound; minw[w] gets the word's least f above
// the bound (0xFFFFFFFF: none) and h_out a copy of h (pointers may be mapped host memory)
int segment_bound(const uint8_t *d_h, const uint8_t *d_g, const uint16_t *d_word_req, const uint32_t *d_req_end,
                  const uint32_t *d_req_bound, uint32_t n_words, uint8_t *h_out, uint32_t *d_mask, uint32_t *d_minw,
                  cudaStream_t st);

// a slot's outputs, one allocation: h [max_batch_pad] bytes, then mask [max_batch_pad / 32]
// words, then minf (one word)
// a network with the real-valued head (FP32 bounds and f-costs)
bool heur_is_real(const Ctx *c, int heur_id);

inline size_t combo_bytes(const Ctx *c) {
    return (size_t)kComboMaxTotal * c->max_batch_pad + c->max_batch_pad / 8 + 4;
}

inline size_t slot_out_bytes(const Ctx *c) { return (size_t)c->max_batch_pad + c->max_batch_pad / 8 + 4; }

// per-domain facts
inline int dom_words(int d) { return d == CBDFS_DOM_RC3 ? 2 : 1; }
inline int dom_side(int d) { return d == CBDFS_DOM_STP3 ? 3 : 4; }
inline int dom_onehot(int d) { return d == CBDFS_DOM_STP3 ? 81 : d == CBDFS_DOM_STP4 ? 256 : 480; }

}  // namespace cbdfs

// ======================================================================================
// device helpers
// ======================================================================================
#ifdef __CUDACC__
namespace cbdfs {
namespace dev {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: the default bound on a device wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after limit_ns (or 2^30 polls), records `code` in *err unless
// another wait recorded its code first (the first cause is kept), and returns false.  Never
// traps.  A wait also gives up at once when the error flag is already set (another wait
// failed).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, int code,
                                          unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1; i < (1u << 30); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*reinterpret_cast<volatile int *>(err) != 0) return false;
            if (globaltimer() - t0 > limit_ns) break;
        }
    }
    atomicCAS(err, 0, code);
    return false;
}

// Bounded wait for work that always completes (issued MMAs, issued TMA loads) before the
// memory it writes is released: unlike mbar_wait it does not give up when the error flag is
// already set, only after limit_ns.
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity, int *err, int code,
                                                unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1; i < (1u << 30); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && globaltimer() - t0 > limit_ns) break;
    }
    atomicCAS(err, 0, code);
    return false;
}

// ---- TMA ----
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// shared -> global tensor store (bulk group of the issuing thread)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most N of this thread's bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// wait until all of this thread's bulk groups are complete (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// ---- tcgen05 ----
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// same with E4M3 inputs (kind::f8f6f4)
__device__ __forceinline__ void umma_fp8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
// ---- CTA pairs (a cluster of two CTAs on neighbouring SMs, tcgen05 cta_group::2) ----
// The pair's MMA (issued by the even CTA, the leader) computes an M = 256 tile: each CTA's
// shared memory holds its 128 rows of A and its half of the N columns of B at the same
// offsets, and each CTA's TMEM receives its own 128 rows of the accumulator.
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(saddr), "r"(rank));
    return d;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init_cluster() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive on an mbarrier of another CTA of the cluster (address from mapa_shared)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an mbarrier of either
// CTA of the pair (bar: a shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// both CTAs of the pair allocate (and later free) the same TMEM columns, one warp each
__device__ __forceinline__ void tmem_alloc_pair(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_fp8_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the pair's MMAs issued so far arrive on the mbarrier at offset `bar` of both CTAs
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((uint16_t)3)
        : "memory");
}

// 32 lanes x 32 columns of 32-bit: thread i of the warp gets row (lane base + i),
// columns col..col+31
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand stored in the 128-byte swizzle
// layout that TMA's SWIZZLE_128B writes: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version for sm_100 family
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M x N tile.
// a_fmt/b_fmt: kind::f16 -> 1 = BF16; kind::f8f6f4 -> 0 = E4M3.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, int a_fmt, int b_fmt) {
    return (1u << 4) | ((uint32_t)a_fmt << 7) | ((uint32_t)b_fmt << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- packed-state helpers ----
template <int SIDE>
__device__ __forceinline__ int manhattan(uint64_t s) {
    constexpr int N = SIDE * SIDE;
    int md = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
        int t = (int)((s >> (4 * p)) & 15u);
        int dr = p / SIDE - t / SIDE, dc = p % SIDE - t % SIDE;
        int d = (dr < 0 ? -dr : dr) + (dc < 0 ? -dc : dc);
        md += t ? d : 0;
    }
    return md;
}
template <int SIDE>
__device__ __forceinline__ bool stp_is_goal(uint64_t s) {
    constexpr int N = SIDE * SIDE;
    uint64_t g = 0;
#pragma unroll
    for (int t = 0; t < N; ++t) g |= (uint64_t)t << (4 * t);
    return s == g;
}
__device__ __forceinline__ bool rc_is_goal(uint64_t w0, uint64_t w1) {
    uint64_t g0 = 0, g1 = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) g0 |= (uint64_t)(k * 3) << (5 * k);
#pragma unroll
    for (int k = 0; k < 12; ++k) g1 |= (uint64_t)(k * 2) << (5 * k);
    return w0 == g0 && w1 == g1;
}

// ---- the real-valued regression rule (CBDFS_HEAD_REAL) ----
// h = max(y + offset, 0), max'ed with the Manhattan distance md (md < 0: none), 0 at the
// goal.  f = g + h is an FP32 sum; bounds and least-f values travel as FP32 bit patterns,
// which order like the values since f >= 0 (the integer heads' uint32 compares and
// atomicMin then serve both).  NaN outputs give h = 0 (fmaxf drops NaN).
__device__ __forceinline__ float real_h(float y, float offset, int md, bool goal) {
    const float h = fmaxf(fmaxf(__fadd_rn(y, offset), 0.f), (float)md);
    return goal ? 0.f : h;
}
__device__ __forceinline__ uint32_t real_f_key(uint32_t g, float h) {
    return __float_as_uint(__fadd_rn((float)g, h));
}
// ---- the classifier quantile (CBDFS_HEAD_QUANTILE) ----
// The smallest class c whose softmax cumulative probability reaches q, from the logits y(0..C)
// in FP32: with m the largest logit and e_c = exp(y_c - m), the first c where e_0 + ... + e_c
// >= q (e_0 + ... + e_{C-1}); C-1 if rounding keeps every partial sum below that.
template <typename Y>
__device__ __forceinline__ int quantile_class(const Y &y, int C, float q) {
    float m = y(0);
    for (int c = 1; c < C; ++c) m = fmaxf(m, y(c));
    float S = 0.f;
    for (int c = 0; c < C; ++c) S += expf(y(c) - m);
    const float T = q * S;
    float acc = 0.f;
    for (int c = 0; c < C; ++c) {
        acc += expf(y(c) - m);
        if (acc >= T) return c;
    }
    return C - 1;
}

// the uint8 h written beside a real h: its ceiling (an admissible integer h when h is, since
// path costs are integers), clamped to 255
__device__ __forceinline__ uint8_t real_h_u8(float h) { return (uint8_t)fminf(ceilf(h), 255.f); }

}  // namespace dev
}  // namespace cbdfs
#endif
