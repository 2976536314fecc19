/*
 * cbdfs.h -- C ABI of the batched cost-bounded DFS heuristic library (sm_103a).
 *
 * The library evaluates heuristics for batches of search states on one GPU, the way the
 * batch-processing thread of the paper's Batch CB-DFS does (arXiv 2507.11916, section
 * "SingleGPU Batch CB-DFS": copy the batch to the GPU, evaluate h_M, return the values),
 * and runs the CPU side of that search (Algorithms 1-3) with C++ worker threads.
 *
 * Conventions shared by every call:
 *   - The return value is a status (cbdfs_status); results come back through out-pointers.
 *     On failure a message is available from cbdfs_last_error() in the calling thread.
 *   - "Host" pointers are ordinary CPU memory owned by the caller; the library copies from
 *     them before the call returns (page-locked memory makes those copies faster).
 *     "Device" pointers are CUDA global memory on the context's device, owned by the caller.
 *     The library owns everything it allocates (weights, tables, scratch, streams).
 *   - Packed states (the ABI's state format):
 *       sliding-tile puzzle (CBDFS_DOM_STP3 3x3, CBDFS_DOM_STP4 4x4): one uint64 per state;
 *         nibble p (bits 4p..4p+3) = tile on cell p, 0 = blank; the goal has tile t on
 *         cell t.  Blank moves: 0 up, 1 left, 2 right, 3 down.
 *       Rubik's cube (CBDFS_DOM_RC3): two uint64 per state.  Word 0: for corner cubie
 *         c = 0..7 the 5-bit field (bits 5c..) slot*3 + twist; word 1: for edge cubie
 *         e = 0..11 the field slot*2 + flip.  Corner slots URF UFL ULB UBR DFR DLF DBL DRB,
 *         edge slots UR UF UL UB DR DF DL DB FR FL BL BR; cubie i is home in slot i.
 *         Move m = 3*face + (quarter turns - 1), faces U R F D L B, clockwise turns.
 *   - Heuristic values are uint8; the goal state always gets h = 0.
 *   - A context is bound to one device.  heur_submit_batch and cbdfs_solve may be called
 *     from several threads at once on one context; the other calls may not.
 *   - Environment: CBDFS_PLAIN_CLUSTER_LAUNCH=1 (read once per process) launches the fused
 *     network kernel's CTA pairs without the cooperative attribute, for profilers that cannot
 *     replay a cooperative cluster launch.  Use it only where one evaluation is in flight at a
 *     time: a partly started plain launch can stall against a launch on another stream until
 *     the device waits run out (CBDFS_ETIMEDOUT).
 */
#ifndef CBDFS_H
#define CBDFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CBDFS_OK = 0,
    CBDFS_EINVAL = -1,      /* bad argument: null pointer, unknown id, size out of range */
    CBDFS_ENOMEM = -2,      /* device or host allocation failed, or the memory budget is spent */
    CBDFS_ETIMEDOUT = -3,   /* a bounded wait (host or device) ran out */
    CBDFS_EDEVICE = -4,     /* a CUDA call failed; the message names it */
    CBDFS_ECANCELED = -5,   /* cbdfs_cancel() stopped the call */
    CBDFS_ENOTFOUND = -6    /* no solution within the limits; a file that does not exist */
} cbdfs_status;

typedef enum { CBDFS_DOM_STP3 = 0, CBDFS_DOM_STP4 = 1, CBDFS_DOM_RC3 = 2 } cbdfs_domain;
typedef enum { CBDFS_PREC_FP32 = 0, CBDFS_PREC_BF16 = 1, CBDFS_PREC_FP8 = 2 } cbdfs_prec;
typedef enum {
    CBDFS_HEAD_REGRESSION = 0,
    CBDFS_HEAD_CLASSIFIER = 1,
    CBDFS_HEAD_REAL = 2,
    CBDFS_HEAD_QUANTILE = 3
} cbdfs_head;
typedef enum { CBDFS_ALGO_IDA = 0, CBDFS_ALGO_BTS = 1 } cbdfs_algo;

/* Built-in heuristic ids (network and PDB ids from the load calls are >= 0). */
#define CBDFS_HEUR_ZERO (-1)    /* h = 0 */
#define CBDFS_HEUR_MD (-2)      /* Manhattan distance, sliding-tile domains only */
#define CBDFS_HEUR_NONE (-100)  /* "no heuristic" (cbdfs_search_cfg.fixed_tree_heur: off) */

typedef struct cbdfs_ctx cbdfs_ctx;
/* identifies an asynchronous batch (heur_submit_batch_async) or a served request */
typedef struct { uint64_t id; } cbdfs_ticket;

typedef struct {
    int device;             /* CUDA device ordinal */
    size_t mem_budget;      /* bytes of device memory the context may allocate; 0 = no limit */
    uint32_t max_batch;     /* largest n one heuristic call accepts (sizes the scratch); 0 = 65536 */
    int n_slots;            /* concurrent evaluation slots (stream + scratch each); 0 = 4 */
    uint64_t device_wait_ns; /* bound on a tile's wait for the previous layer's rows inside the
                               fused network kernel, in ns of %globaltimer; 0 = 2 s.  Its stage
                               and accumulator waits get twice this bound, so that a row count
                               that never comes is the wait that runs out first.  A wait that
                               runs out sets the device error flag (cbdfs_device_status; the
                               first cause is kept) and the kernel winds down; too small a bound
                               makes an ordinary launch report a timeout */
} cbdfs_config;

/* Create a context on cfg->device.  *out receives it.  Errors: EINVAL, EDEVICE, ENOMEM. */
int cbdfs_create(const cbdfs_config *cfg, cbdfs_ctx **out);
/* Free everything the context owns.  Safe on NULL. */
void cbdfs_destroy(cbdfs_ctx *ctx);
/* The last failure message of the calling thread ("" if none).  Valid until its next call. */
const char *cbdfs_last_error(void);
/* Device memory the context holds now, in bytes. */
size_t cbdfs_mem_used(const cbdfs_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Network heuristic h_M (paper: "Experimental Setup" -- a classifier and a regression
 * network, evaluated in batches; Algorithm 3 adds TensorRepresentation(s) to the batch).
 * The network input is the one-hot encoding of the packed state:
 *   STP with N cells: index tile*N + cell (blank included), width N*N (81 or 256);
 *   RC: corner cubie c at c*24 + (slot*3 + twist), edge e at 192 + e*24 + (slot*2 + flip),
 *   width 480.
 * Layers: z_l = W_l a_{l-1} + b_l, ReLU after every layer but the last.  The last layer
 * always runs in FP32.  With CBDFS_PREC_BF16 / _FP8 the hidden layers run on the tensor
 * cores with FP32 accumulation (FP8: E4M3, per-tensor weight scale amax/448 and the given
 * static activation scales).
 * Integer h (the fused epilogue):
 *   regression: h = max(rint(y), 0) (round half to even), max'ed with Manhattan distance
 *               when max_with_md != 0, clamped to 255;
 *   classifier: h = argmax over the outputs (lowest index on ties), max'ed with Manhattan
 *               distance when max_with_md != 0.
 *   quantile:   the classifier quantile (Related Work: ordered classes let the quantile of
 *               the predicted class be lowered for admissibility): with p = softmax(y) in
 *               FP32, h = the smallest class c with p_0 + ... + p_c >= quantile (the last
 *               class if rounding keeps the total below it), max'ed with Manhattan distance
 *               when max_with_md != 0.
 * Real-valued h (section "Regression-Based Neural Heuristics"; Experimental Setup: the
 * regression model's predictions minus 2.2):
 *   real:       one output; h = max(y + h_offset, 0) in FP32, max'ed with Manhattan distance
 *               when max_with_md != 0; the goal gets 0.  f = g + h is an FP32 sum and the
 *               bound is an FP32 value: these networks are evaluated through the *_real
 *               calls below, and cbdfs_solve searches them with real thresholds.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int domain;                     /* cbdfs_domain */
    int n_layers;                   /* L >= 2 */
    const int *dims;                /* L+1 widths; dims[0] must equal the domain's one-hot width */
    const float *const *weights;    /* host, L pointers; layer l is dims[l+1] x dims[l], row-major */
    const float *const *biases;     /* host, L pointers of dims[l+1] floats */
    int prec;                       /* cbdfs_prec */
    int head;                       /* cbdfs_head */
    int max_with_md;                /* STP only */
    const float *act_scales;        /* FP8 only: L-1 activation scales (host), else NULL */
    float h_offset;                 /* CBDFS_HEAD_REAL: added to y (the paper: -2.2); else 0 */
    float quantile;                 /* CBDFS_HEAD_QUANTILE: q in (0, 1]; else 0 */
} cbdfs_net_desc;

/* Copy a network into device memory.  Weights are rounded there to the precision (FP32
 * master values -> BF16 round-to-nearest-even, or -> E4M3 with the scale).  *heur_id
 * receives its id.  Hidden widths must be multiples of 128 for BF16/FP8.
 * Errors: EINVAL (shape; a server is running on the context), ENOMEM, EDEVICE. */
int cbdfs_net_load(cbdfs_ctx *ctx, const cbdfs_net_desc *d, int *heur_id);

/* ---------------------------------------------------------------------------------------
 * Additive pattern database (paper: "Background, Heuristics": abstraction distances are
 * admissible; Experimental Setup uses additive tile PDBs for the STP).  Pattern q lists
 * k[q] tiles; its table is indexed by the lexicographic rank of the cells holding those
 * tiles (in list order) among all k-permutations of the N cells:
 *   rank = sum_i d_i * (N-1-i)!/(N-k)!,  d_i = cell_i - #{j < i : cell_j < cell_i}.
 * h = sum over patterns of table_q[rank_q].
 * The cube (CBDFS_DOM_RC3; Experimental Setup: the 8-corner PDB) takes one pattern, the
 * corner cubies 0..7 in order: with p_c the slot and t_c the twist of corner cubie c,
 *   index = rank(p) * 3^7 + sum_{c<7} t_c 3^c,  rank(p) = sum_i (p_i - #{j<i: p_j<p_i}) (7-i)!,
 * 8! * 3^7 = 88,179,840 entries.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int domain;                     /* any cbdfs_domain (the cube: the corner pattern only) */
    int n_patterns;                 /* 1..4 */
    const int *k;                   /* tiles per pattern */
    const int *tiles;               /* concatenated tile lists */
    const uint8_t *const *tables;   /* host tables, N!/(N-k)! entries each; NULL: build them
                                       on the GPU with pdb_build */
    int div;                        /* 0 or 1: as given; k >= 2: DIV-compressed on the device
                                       (Background, PDB compression: entry j keeps the least of
                                       the k entries j*k .. j*k+k-1; h reads entry rank / k) */
} cbdfs_pdb_desc;

/* Register an additive PDB (copying the tables to the device, or building them there).
 * *heur_id receives its id.  Errors: EINVAL (also while a server runs), ENOMEM, EDEVICE. */
int cbdfs_pdb_load(cbdfs_ctx *ctx, const cbdfs_pdb_desc *d, int *heur_id);

/* Build one pattern's table on the GPU by breadth-first search over the abstract space
 * (pattern-tile cells plus the blank cell; a blank move that displaces a pattern tile costs
 * 1, any other costs 0; the entry is the least distance over blank cells).  table_out
 * (host, cap bytes) receives N!/(N-k)! entries; *entries receives that count.  For the cube
 * (pattern_tiles = 0..7, k = 8): the 8-corner table, by breadth-first search over corner
 * configurations under the 18 face turns (88,179,840 entries, largest distance 11).
 * Errors: EINVAL (cap too small, bad tiles), ENOMEM, EDEVICE. */
int pdb_build(cbdfs_ctx *ctx, int domain, const int *pattern_tiles, int k, uint8_t *table_out,
              size_t cap, size_t *entries);

/* PDB table files (the tables are built offline and reused): a 128-byte header, then the
 * table bytes.  Header, little-endian: "CBDFSPDB" (8 bytes), format version 1 (uint32),
 * domain (int32), k (int32), the pattern's tiles (16 x int32, unused ones 0), the DIV factor
 * (uint32; 1 = a full table), the entry count (uint64), the FNV-1a 64-bit hash of the table
 * bytes (uint64), zero padding.  Host-only calls: no context, no GPU.
 * `entries` must be the table size the pattern implies: N!/(N-k)! for k tiles of a sliding-tile
 * puzzle of N = 9 or 16 cells (k <= N-1), 8! * 3^7 for the cube's 8-corner table (k = 8), in
 * both cases divided by the DIV factor and rounded up.
 * cbdfs_pdb_file_write writes `entries` bytes of `table`.  Errors: EINVAL (arguments, an entry
 * count the pattern does not imply), EDEVICE (the file could not be written).
 * cbdfs_pdb_file_read fills the header fields (tiles: 16 ints) and *entries; with table
 * non-NULL it also reads the bytes (cap >= entries) and checks the hash.  Errors: EINVAL (not
 * such a file, version, a domain, DIV factor or entry count that is not a valid table's, cap
 * too small, hash mismatch, short file), ENOTFOUND (no file). */
int cbdfs_pdb_file_write(const char *path, int domain, const int *tiles, int k, uint32_t div,
                         const uint8_t *table, uint64_t entries);
int cbdfs_pdb_file_read(const char *path, int *domain, int *tiles, int *k, uint32_t *div,
                        uint8_t *table, uint64_t cap, uint64_t *entries);

/* ---------------------------------------------------------------------------------------
 * Composite heuristic (Related Work: the minimum over an ensemble of networks keeps a
 * learned heuristic admissible; Experimental Setup: the 15-puzzle h_M adds to Manhattan
 * distance two ensembles, each trained on one pattern's PDB minus Manhattan distance):
 *   h = [MD if add_md] + sum over groups g of (min over the members of g of h_member),
 * clamped to 255; the goal gets 0.  Members are loaded heuristic ids (networks with integer
 * heads, PDBs, CBDFS_HEUR_MD / _ZERO) of the same domain: at most 4 groups of 1..8 members,
 * 16 members in all.  A group of two or more BF16 networks of one shape whose head runs on
 * the tensor cores (classifier or quantile, 17..128 outputs) is evaluated as one grouped
 * network (the ensemble as a grouped GEMM: one fused launch for the hidden layers, one for the
 * heads); the load copies those members' weights, so train members before combining them.
 * Other members run their own pipelines one after another; then one kernel combines them and
 * applies the bound test.  Not on the allocation-free entry (heur_eval_device_static).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int domain;
    int n_groups;
    const int *group_size;          /* n_groups member counts */
    const int *members;             /* the member ids, group after group */
    int add_md;                     /* sliding-tile domains: add Manhattan distance */
} cbdfs_combo_desc;

/* *heur_id receives the composite's id.  Errors: EINVAL (members, sizes, domain; a server is
 * running), ENOMEM, EDEVICE. */
int cbdfs_combo_load(cbdfs_ctx *ctx, const cbdfs_combo_desc *d, int *heur_id);

/* ---------------------------------------------------------------------------------------
 * Batched heuristic evaluation with the bound test (Algorithm 3: a node is expanded when
 * f = g + h is within the bound; the smallest f above the bound is the next IDA*
 * threshold, "lowest unexpanded f-cost").
 *   states  n packed states (1 or 2 words each, see above)
 *   g       n path costs (uint8)
 *   bound   the cost bound
 *   h_out   n heuristic values
 *   mask_out ceil(n/32) words: bit i%32 of word i/32 is set iff g_i + h_i <= bound
 *   minf_out the least g_i + h_i above the bound, 0xFFFFFFFF if none
 *   y_out   optional (may be NULL): the raw FP32 network outputs, n x dims[L] row-major
 *           (ignored for PDB / built-in heuristics)
 * n = 0 is allowed (mask nothing, minf 0xFFFFFFFF).  n > max_batch: EINVAL.  A network with
 * the real-valued head is refused here (EINVAL): use heur_submit_batch_real.
 * ------------------------------------------------------------------------------------- */

/* Host buffers; returns when the results are in h_out/mask_out/minf_out.  When states, g,
 * h_out and mask_out are all page-locked (cudaMallocHost / cudaHostRegister) and y_out is
 * NULL, the kernels read and write them in place over the bus (no staging copies); other
 * buffers are copied through the slot's device staging.  The buffers must not change
 * until the call returns. */
int heur_submit_batch(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states,
                      const uint8_t *g, uint32_t bound, uint32_t n, uint8_t *h_out,
                      uint32_t *mask_out, uint32_t *minf_out, float *y_out);

/* Device buffers, enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream).
 * Cube states (two words each) must start on a 16-byte boundary (EINVAL otherwise);
 * returns without waiting.  All device-buffer calls on one context share one set of
 * activation scratch, and the library orders each call after the previous one on the GPU.
 * The call may be captured into a CUDA graph (the library then leaves the ordering to the
 * graph): replays of such a graph must not overlap other device-buffer calls on the same
 * context.  Errors are those detected before enqueueing; a device-side timeout sets the
 * flag read by cbdfs_device_status(). */
int heur_eval_device(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                     const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h,
                     uint32_t *d_mask, uint32_t *d_minf, float *d_y, void *stream);

/* Asynchronous form (no y_out): holds a free slot, enqueues the batch on its stream and returns
 * with *t at once; the results are in h_out, mask_out and minf_out when heur_wait(t) has
 * returned CBDFS_OK, and no buffer may change before.  Fully asynchronous when the buffers are
 * page-locked (the kernels then read and write them in place); pageable ones are copied, and a
 * copy to pageable memory waits for the batch.  Each batch holds one of the context's host
 * slots until it is waited on: a submit that finds none free blocks until another thread's
 * wait releases one.  Thread-safe.  Errors: those of heur_submit_batch. */
int heur_submit_batch_async(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states,
                            const uint8_t *g, uint32_t bound, uint32_t n, uint8_t *h_out,
                            uint32_t *mask_out, uint32_t *minf_out, cbdfs_ticket *t);

/* Wait up to timeout_us (0: without limit) for an asynchronous batch.  CBDFS_ETIMEDOUT if it is
 * still running (the ticket stays valid); otherwise the batch's status, and the ticket and its
 * slot are released.  EINVAL for an unknown or collected ticket. */
int heur_wait(cbdfs_ctx *ctx, cbdfs_ticket t, uint64_t timeout_us);

/* Real-valued heuristic (a network loaded with CBDFS_HEAD_REAL), host buffers: the bound
 * test with f = g + h in FP32 (Algorithm 3's expansion test with real f-costs).
 *   bound    a finite or infinite FP32 bound >= 0 (negative or NaN: EINVAL)
 *   h_out    n real heuristic values
 *   mask_out ceil(n/32) words, bit i set iff g_i + h_i <= bound
 *   minf_out the least g_i + h_i above the bound; +infinity if none
 * Other heuristics are refused (EINVAL).  Returns when the results are in the buffers. */
int heur_submit_batch_real(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states,
                           const uint8_t *g, float bound, uint32_t n, float *h_out,
                           uint32_t *mask_out, float *minf_out);

/* The same on device buffers, enqueued on `stream` as heur_eval_device.  *d_minf receives
 * the least f above the bound, or the bit pattern 0xFFFFFFFF (a NaN) if none. */
int heur_eval_device_real(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                          const uint8_t *d_g, float bound, uint32_t n, float *d_h,
                          uint32_t *d_mask, float *d_minf, void *stream);

/* Like heur_eval_device, for callers that cannot allocate device memory when they evaluate
 * a batch (a real-time or latency-budgeted caller that must not enter the allocator, or a
 * process whose device memory another framework's allocator owns).  The paper has no
 * counterpart; this is a library-usage variant.
 *   - The call allocates nothing: the layers' activation scratch is a file-scope device
 *     array of 2 x 16 MiB that every device holding the library keeps until the process
 *     exits.  The network (or PDB) must already be loaded on the context.
 *   - Limit: the padded batch (n rounded up to 128) times the widest hidden layer times 2
 *     bytes (4 for FP32 networks) must fit 16 MiB, e.g. 8192 states of a 1024-wide BF16
 *     network; a larger n fails with CBDFS_EINVAL and says the largest n that fits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.
 *   - Every call shares the array, which keeps the previous call's contents; nothing in it
 *     needs to start at zero (each call writes every activation row it reads).  Calls that
 *     overlap on the GPU (other streams, other threads) race on the array: order them.
 * Errors: EINVAL (arguments, size limit, a real-valued network), EDEVICE. */
int heur_eval_device_static(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                            const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h,
                            uint32_t *d_mask, uint32_t *d_minf, void *stream);

/* Like heur_eval_device, and then waits: stage_ms[i] receives the device time of the i-th
 * kernel of the pipeline (network: layer 1 .. layer L-1, then the head; PDB / built-in: the
 * one kernel), measured with CUDA events recorded between the launches on `stream`.
 * *n_stages receives the number of kernels (at most cap are written).  The pipeline's
 * results are written as for heur_eval_device.  Errors: those of heur_eval_device, EDEVICE. */
int cbdfs_eval_profile(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                       const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h,
                       uint32_t *d_mask, uint32_t *d_minf, void *stream, float *stage_ms, int cap,
                       int *n_stages);

/* Like cbdfs_eval_profile, for the fused network kernel: records its tile timeline.  d_trace
 * (device, caller-owned) holds ctas_max x tiles_per_cta x 8 uint64 %globaltimer stamps (ns):
 * for the i-th tile a CTA processes, [0] producer start, [1] its layer dependency satisfied,
 * [2] its last load issued, [3] first MMA issue, [4] last MMA committed, [5] epilogue start,
 * [6] epilogue end, [7] unused; 0 = not reached.  *ctas receives the grid size (at most the
 * SM count).  Networks not run by the fused kernel record nothing (*ctas = 0).  Waits for
 * completion.  Errors: those of heur_eval_device, EDEVICE. */
int cbdfs_eval_trace(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *d_states,
                     const uint8_t *d_g, uint32_t bound, uint32_t n, uint8_t *d_h,
                     uint32_t *d_mask, uint32_t *d_minf, void *stream, uint64_t *d_trace,
                     int tiles_per_cta, int *ctas);

/* Reads and clears the device-side error flag (0 = none; otherwise a code naming the
 * wait that ran out).  Synchronises the context's device.  A set flag also resets every slot's
 * dependency counters of the fused network kernel (a launch whose wait ran out may leave them
 * counted); until this call, every evaluation on the context reports ETIMEDOUT. */
int cbdfs_device_status(cbdfs_ctx *ctx);

/* Failure-detection testing (no counterpart in the paper): the next launch of the fused network
 * kernel on this context skips the first hidden layer's completion count of one 128-state row
 * block (row_block < 0: nothing skipped), so that the second layer's tiles of that row block
 * wait for rows that never come.  Their wait runs out after cbdfs_config.device_wait_ns, the
 * evaluation returns CBDFS_ETIMEDOUT (or, for device-buffer calls, cbdfs_device_status returns
 * the wait's code, 5), and the kernel ends normally; nothing faults and the context stays
 * usable once cbdfs_device_status has cleared the flag.  One launch only; the setting is then
 * cleared.  Errors: EINVAL (null context). */
int cbdfs_debug_withhold_publish(cbdfs_ctx *ctx, int row_block);

/* ---------------------------------------------------------------------------------------
 * Serving: continuous batching of requests from many threads (paper: the batch-processing
 * thread of SingleGPU Batch CB-DFS gathers states from the searching threads, evaluates
 * them on the GPU and keeps more than one batch in flight).  A server thread takes queued
 * requests of one heuristic, in arrival order, into one launch of up to bucket_max states
 * as soon as an evaluation slot is free and the memory budget allows, replays the CUDA
 * graph captured for (slot, heuristic, size bucket = next power of two), and lets launches
 * on different slots overlap on the device.  Each request's h is exactly what it would get
 * alone (rows are independent); each request starts on a 32-row boundary of its launch, so
 * its mask and least f above its own bound are formed on the device in the same graph.
 * Caller buffers must stay valid until heur_request_wait returns.
 * ------------------------------------------------------------------------------------- */

typedef struct {
    int max_inflight;       /* launches on the device at once (slots taken); 0 = all free slots */
    uint32_t bucket_min;    /* smallest launch size (0 = 32) */
    uint32_t bucket_max;    /* largest launch size and largest request (0 = 4096) */
    size_t mem_budget;      /* device bytes in-flight launches may use; 0 = no limit */
    int coalesce;           /* 1: merge queued requests of one heuristic into a launch */
    int direct;             /* 1: enqueue each launch's pipeline on the slot's stream instead of
                               replaying the captured graph of its bucket */
} cbdfs_server_cfg;

typedef struct {
    uint64_t requests, states, launches;
    double p50_us, p99_us, mean_us;   /* request latency, submit to completion */
    double states_per_s;              /* states completed / (last completion - first submit) */
    /* the server thread's time per launch: taking requests, staging and launching; from the
       launch until its completion was seen; copying results out and waking the callers */
    double stage_us_per_launch, flight_us_per_launch, finish_us_per_launch;
    double replay_us_per_launch;      /* of the staging time: the graph launch call itself */
} cbdfs_server_stats;

/* Start the server (at most one per context).  Errors: EINVAL (no free slot, buckets),
 * ENOMEM, EDEVICE.  Load networks before starting: loads are refused while it runs. */
int cbdfs_server_start(cbdfs_ctx *ctx, const cbdfs_server_cfg *cfg);
/* Finish every queued request, then stop the server and release its slots. */
int cbdfs_server_stop(cbdfs_ctx *ctx);
/* Queue a request (arguments as heur_submit_batch, 1 <= n <= bucket_max); *t identifies it.
 * Thread-safe.  Errors: EINVAL, ECANCELED (stopping). */
int heur_request_submit(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states,
                        const uint8_t *g, uint32_t bound, uint32_t n, uint8_t *h_out,
                        uint32_t *mask_out, uint32_t *minf_out, cbdfs_ticket *t);
/* Wait up to timeout_us (0: just test) for a request; its results are then in the caller's
 * buffers.  Returns OK, ETIMEDOUT (still running; wait again), EINVAL (unknown or already
 * collected ticket), or the launch's error. */
int heur_request_wait(cbdfs_ctx *ctx, cbdfs_ticket t, uint64_t timeout_us);
/* Latency and throughput of the requests completed so far. */
int cbdfs_server_get_stats(cbdfs_ctx *ctx, cbdfs_server_stats *out);
/* Forget the statistics gathered so far (for instance after a warm-up). */
int cbdfs_server_reset_stats(cbdfs_ctx *ctx);
/* Capture the CUDA graph of every size bucket of one heuristic on every server slot now,
 * instead of on each bucket's first request (a capture takes milliseconds).  Waits for slots
 * in use.  Errors: EINVAL (no server, heuristic id), EDEVICE. */
int cbdfs_server_prepare(cbdfs_ctx *ctx, int heur_id, int domain);

/* One request of cbdfs_server_drive (the arguments of heur_request_submit; caller-owned
 * buffers that stay valid until the call returns). */
typedef struct {
    int heur_id, domain;
    const uint64_t *states;
    const uint8_t *g;
    uint32_t bound, n;
    uint8_t *h_out;
    uint32_t *mask_out, *minf_out;
} cbdfs_request;

/* Measurement of the running server with native clients (no counterpart in the paper; the
 * paper's clients are its search threads): `threads` client threads take the requests in
 * order, each the next one not yet taken, and each keeps at most `depth` of its own requests
 * outstanding (depth 1: a client blocks on every request, as a search thread blocks on its
 * batch).  Returns when every request is done; *seconds is the wall time from the moment every
 * client thread is running to the last completion.  Errors: EINVAL, or the first failed
 * request's status. */
int cbdfs_server_drive(cbdfs_ctx *ctx, const cbdfs_request *reqs, uint32_t n_reqs, int threads, int depth,
                       double *seconds);

/* ---------------------------------------------------------------------------------------
 * Learning the network heuristic (paper: Experimental Setup -- the heuristics are trained
 * from PDB values).  BF16 networks only.  One step on a batch: BF16 tensor-core forward
 * (activations kept), FP32 last layer and loss, backward with BF16 tensor-core GEMMs and
 * FP32 accumulation (dW = dZ^T A, dA = dZ W, ReLU masks), FP32 Adam on FP32 master weights
 * (bias-corrected), then the BF16 weights the heuristic evaluates are rewritten in place.
 * The masters start from the FP32 weights given to cbdfs_net_load.
 * ------------------------------------------------------------------------------------- */
typedef enum { CBDFS_LOSS_CE = 0, CBDFS_LOSS_MSE = 1 } cbdfs_loss;

typedef struct {
    float lr, beta1, beta2, eps;    /* Adam (1e-3, 0.9, 0.999, 1e-8) */
    uint32_t batch;                 /* states per step (<= max_batch) */
    int epochs;                     /* passes over the set */
    uint64_t seed;                  /* epoch e visits the states in the Fisher-Yates order drawn
                                       from splitmix64(seed + (e+1)*0x9E3779B97F4A7C15) */
    int loss;                       /* cbdfs_loss: cross-entropy over classes = labels, or
                                       0.5*(y - label)^2 on one output */
    int64_t max_steps;              /* stop after this many steps (0: no limit) */
} cbdfs_train_cfg;

typedef struct {
    int64_t steps, samples;
    double seconds;
    float first_loss, last_loss;    /* mean batch loss of the first and last step */
} cbdfs_train_report;

/* Train network heur_id on n (state, label) pairs (host buffers, copied).  Labels are class
 * indices (< outputs) for cross-entropy, target values for MSE.
 * Errors: EINVAL (not a BF16 network, label range, sizes, a server is running), ENOMEM,
 * EDEVICE, ETIMEDOUT. */
int net_train(cbdfs_ctx *ctx, int heur_id, const uint64_t *states, const uint8_t *labels,
              uint64_t n, const cbdfs_train_cfg *cfg, cbdfs_train_report *rep);

/* Loss and gradients of the mean loss over one batch of n states at the current weights,
 * without updating (host buffers; gw_out[l] is dims[l+1] x dims[l], gb_out[l] dims[l+1];
 * NULL entries are skipped).  n <= max_batch. */
int cbdfs_train_grad(cbdfs_ctx *ctx, int heur_id, const uint64_t *states, const uint8_t *labels,
                     uint32_t n, int loss, float *loss_out, float *const *gw_out,
                     float *const *gb_out);

/* The network's FP32 weights (the training masters once trained), host buffers as in
 * cbdfs_net_desc. */
int cbdfs_net_read(cbdfs_ctx *ctx, int heur_id, float *const *w_out, float *const *b_out);

/* Training checkpoints: the network's training state (FP32 master weights and biases, Adam's
 * first and second moments, the step count that drives Adam's bias correction) to a file,
 * and back.  After cbdfs_train_load the heuristic evaluates the loaded masters (its BF16
 * weights and FP32 last layer are rewritten) and net_train continues from the loaded state,
 * exactly as if it had not stopped (same data and seed: the same weights).  File: "CBDFSTRN"
 * (8 bytes), version 1 (uint32), L (uint32), dims[0..8] (uint32, unused 0), the padded
 * one-hot width (uint32), the step (int64), the payload bytes (uint64), the FNV-1a 64-bit
 * hash of the payload (uint64); then per layer l: W_l [dims[l+1]][K_l], b_l, m(W_l), v(W_l),
 * m(b_l), v(b_l), FP32, K_0 the padded one-hot width, K_l = dims[l] otherwise.
 * Errors: EINVAL (not a BF16 network, another shape, not such a file, hash mismatch, a
 * server is running), ENOTFOUND (no file), EDEVICE (I/O or device), ENOMEM. */
int cbdfs_train_save(cbdfs_ctx *ctx, int heur_id, const char *path);
int cbdfs_train_load(cbdfs_ctx *ctx, int heur_id, const char *path);

/* n sliding-tile states from random walks of the blank from the goal, walk i = first..:
 * its splitmix64 stream starts at mix((tag << 32) | (i mod 2^32)); the walk's length is
 * 1 + (draw mod max_len); each move is drawn (draw mod #choices) among the legal blank
 * moves (up, left, right, down order) except the reverse of the previous one.  Host output.
 * Errors: EINVAL, ENOMEM, EDEVICE. */
int cbdfs_gen_walk_states(cbdfs_ctx *ctx, int domain, uint32_t tag, uint64_t first, uint64_t n,
                          int max_len, uint64_t *states_out);

/* ---------------------------------------------------------------------------------------
 * Domain helpers (product-side domain code; the search uses the same routines).
 * ------------------------------------------------------------------------------------- */

/* Apply `n` moves to a packed state (words as above).  Returns EINVAL on an illegal STP
 * move (blank off the board) or a move number out of range. */
int cbdfs_apply_moves(int domain, const uint64_t *start, const int *moves, int n, uint64_t *out);
/* Manhattan distance of an STP state (host). */
int cbdfs_manhattan(int domain, uint64_t state);

/* ---------------------------------------------------------------------------------------
 * Batch CB-DFS search: IDA* (Algorithm 1) or BTS (Batch BTS enhancements) over C++ worker
 * threads (Algorithm 2), each round-robining over work_num subtree stacks (Algorithm 3),
 * with heuristic evaluation batched on the GPU through the slots.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int threads;            /* worker threads (>= 1) */
    int work_num;           /* subtrees per thread (>= 1) */
    int d_init;             /* depth of the initial partition (GenerateWork); -1 = automatic */
    uint32_t batch;         /* target states per GPU batch (<= max_batch) */
    uint32_t timeout_us;    /* flush a partly filled batch after this long (paper: 4 ms) */
    int complete_final;     /* finish the iteration that reaches a goal and return the least
                               goal cost in it (deterministic counts); 0 = stop at the first */
    int fixed_tree_heur;    /* CBDFS_HEUR_NONE: prune with heur_id; else prune with this
                               heuristic while still evaluating heur_id on every generated node
                               (the paper's fixed-tree evaluation) */
    uint64_t bts_n0;        /* BTS: initial growth base (paper: 10,000) */
    int bts_c1, bts_c2;     /* BTS: accept >= c1*N expansions, limit c2*N (0 = 2 and 8) */
    uint64_t node_limit;    /* stop with ECANCELED after this many expansions; 0 = none */
    double time_limit_s;    /* stop with ETIMEDOUT after this long; 0 = none */
} cbdfs_search_cfg;

#define CBDFS_MAX_ITERS 256
#define CBDFS_BATCH_HIST 16

typedef struct {
    int cost;                       /* solution cost (-1 if none) */
    int path_len;                   /* moves in path[] */
    int path[256];                  /* moves from the start to the goal */
    int n_iters;                    /* CB-DFS searches run (IDA* iterations / BTS searches) */
    int64_t iter_bound[CBDFS_MAX_ITERS];
    int64_t iter_expanded[CBDFS_MAX_ITERS];
    int64_t iter_generated[CBDFS_MAX_ITERS];
    int64_t iter_limit[CBDFS_MAX_ITERS];   /* BTS expansion limit (-1 none) */
    int iter_cut[CBDFS_MAX_ITERS];         /* BTS: the limit stopped that search */
    int64_t expanded, generated;    /* totals over all searches */
    int64_t batches;                /* GPU batches evaluated */
    int64_t evaluated;              /* states evaluated on the GPU */
    double seconds;                 /* wall time of the solve */
    int d_init;                     /* initial partition depth used */
    int64_t work_items;             /* subtrees in the shared work queue */
    double batch_fill_us;           /* mean time from a batch's first state to its submission */
    double batch_flight_us;         /* mean time from submission to its results being readable */
    double submit_us;               /* mean host time the batch processor spends submitting one */
    int real_valued;                /* 1: the pruning heuristic is real-valued (CBDFS_HEAD_REAL);
                                       its bounds are in iter_bound_real, iter_bound holds 0 */
    double iter_bound_real[CBDFS_MAX_ITERS];  /* every search's bound as a real number */
    int64_t batch_hist[CBDFS_BATCH_HIST];     /* GPU batches by size (those of the initial
                                                 partition too): entry i counts the batches of
                                                 2^i .. 2^(i+1)-1 states (the last: 2^15 and
                                                 more); the entries add up to `batches` */
    double gpu_busy_s;              /* wall time during which at least one GPU batch was in flight
                                       (from its submission until the batch processor saw it
                                       complete); gpu_busy_s / seconds bounds the GPU's busy
                                       fraction from above */
} cbdfs_result;

/* Solve from `start` (packed words).  heur_id: a network, a PDB or a built-in id.
 * Errors: EINVAL, ENOTFOUND (tree exhausted), ETIMEDOUT, ECANCELED, EDEVICE. */
int cbdfs_solve(cbdfs_ctx *ctx, int domain, const uint64_t *start, int algo, int heur_id,
                const cbdfs_search_cfg *cfg, cbdfs_result *out);

/* Fill a search configuration with the defaults documented above. */
void cbdfs_search_defaults(cbdfs_search_cfg *cfg);

/* Ask running calls on ctx to stop (they return ECANCELED). */
void cbdfs_cancel(cbdfs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CBDFS_H */
