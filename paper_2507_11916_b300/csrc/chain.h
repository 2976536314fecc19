// chain.h -- what the host side and the fused network kernel (mlp_chain.cu) share.
#pragma once
#include "common.cuh"

namespace cbdfs {

constexpr int kChainBN = 256;     // output columns of a tile (one TMEM accumulator)
constexpr int kChainBNSmall = 64; // the same for small batches (more tiles in flight per layer)
constexpr int kChainStages = 4;
constexpr int kChainPairStages = 6;  // CTA pairs: 32 KB k-block stages (A rows + half the weights)
constexpr int kChainPairMinMBlocks = 8;  // CTA pairs from this many 128-state row blocks on
constexpr int kChainThreads = 192;
constexpr int kMaxHeadC = 32;     // widest last layer the in-epilogue head takes

struct ChainMaps {
    CUtensorMap w[kMaxLayers];  // weights of hidden layer l, [N][K] K-major, boxes of bn rows
    CUtensorMap a[kMaxLayers];  // A of hidden layer l: the one-hot rows (l = 0) or activations
    CUtensorMap o[kMaxLayers];  // activations written by hidden layer l (32 x 32 store boxes)
};

struct ChainParams {
    int nh;                        // hidden layers (tensor-core layers) = L-1
    int dims[kMaxLayers + 1];
    int kdim[kMaxLayers];          // K of hidden layer l (layer 0: padded one-hot width; a
                                   // grouped layer: one member's K)
    int group_nt[kMaxLayers];      // grouped layer (an ensemble run as one network): n-tiles per
                                   // member, whose A is its own K-column block; 0: dense
    int nt[kMaxLayers];            // n-tiles of hidden layer l
    int tile_start[kMaxLayers + 1];
    int mblocks;
    uint32_t n;
    const uint64_t *states;
    void *onehot;                  // [rows_pad][kdim[0]] one-hot input, written by the pre-pass
    void *act[2];
    const float *bias[kMaxLayers];
    float acc_scale[kMaxLayers], out_qscale[kMaxLayers];
    int *counters;                 // [mblocks] one-hot units (kBM / unit_rows = all rows), then [nh][mblocks]
                                   // stored warp-tiles (4 per tile), then [mblocks] head counts;
                                   // zero at launch; zeroed again once nothing reads them
    int unit_rows;                 // rows of a one-hot pre-pass unit: 8 or 16
    float *partial;                // [nt_last][rows_pad][C]
    int rows_pad;
    int fused_head;                // 1: the last layer runs in the last hidden layer's epilogue;
                                   // 0: every hidden layer is stored and a separate kernel
                                   // runs the last layer
    int bf16_store_layer;          // hidden layer whose stored output is BF16 in an E4M3
                                   // network (the separate last layer reads BF16); -1 none
    int C;                         // outputs of the last layer
    int head_kind, max_with_md;
    float head_param;              // CBDFS_HEAD_REAL: the offset; CBDFS_HEAD_QUANTILE: q
    const float *w_last, *b_last;  // [C][dims[nh]], [C]
    const uint8_t *g;
    uint32_t bound;                // CBDFS_HEAD_REAL: the FP32 bound's bit pattern
    uint8_t *h;                    // may be null for CBDFS_HEAD_REAL
    uint32_t *mask, *minf;
    float *y;                      // raw outputs; CBDFS_HEAD_REAL: the real h
    int *err;
    unsigned long long wait_ns;    // bound on each wait (ns of %globaltimer)
    int hold_mblock;               // failure-detection testing: the row block whose first-layer
                                   // completion count this launch skips (-1: none)
    unsigned long long *trace;     // optional: [grid][trace_tiles][8] %globaltimer stamps
    int trace_tiles;
};

// the last layer of a classifier network (17..128 outputs) on the tensor cores (head_tc.cu)
constexpr int kHeadTcMinC = 16, kHeadTcMaxC = 128;
struct HeadTcParams {
    int K;             // input width, a multiple of 64
    int C, cpad;       // outputs, and their padding to a multiple of 16 (<= 128)
    int head_kind;     // CBDFS_HEAD_CLASSIFIER or CBDFS_HEAD_QUANTILE
    float quantile;
    int max_with_md;
    uint32_t n;
    const uint64_t *states;
    const uint8_t *g;
    uint32_t bound;
    const float *b_last;
    uint8_t *h;        // null: only the logits (y), no rule and no bound test
    uint32_t *mask, *minf;
    float *y;          // optional [n][C] logits
    int *err;
    // an ensemble run as one network: member e (blockIdx.y) reads A columns [e K, e K + K) and
    // weight rows from e 3 cpad, writes h to h + e h_stride; no mask or minf then (0: one network)
    int groups;
    size_t h_stride;
};

int head_tc(int domain, const CUtensorMap &tmA, const CUtensorMap &tmW, const HeadTcParams &P, uint32_t rows_pad,
            cudaStream_t st);

// bn: kChainBN, or kChainBNSmall (maps.w with 64-row boxes).  pair: CTA pairs (bn = kChainBN,
// maps.w with 128-row boxes, an even number of row blocks and of CTAs; the tile sequence in
// P counts pair tiles)
int chain_launch(int domain, bool fp8, int bn, bool pair, const ChainMaps &maps, const ChainParams &P, int grid,
                 cudaStream_t st);
// whether the device holds all the CTA pairs of a one-CTA-per-SM launch at once
bool chain_pairs_fit(int num_sms);

}  // namespace cbdfs
