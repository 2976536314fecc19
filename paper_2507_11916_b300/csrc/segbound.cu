// segbound.cu -- the bound test of many requests evaluated in one launch (serving).
//
// The server packs the requests of a launch so that each starts on a 32-row boundary: mask
// word w then belongs to one request, word_req[w] (0xFFFF: padding).  Row r of that word
// passes when g[r] + h[r] <= the request's own bound (Algorithm 3's expansion test, read as
// g + h <= bound), rows at or past the request's end are zero bits, and the word's least f
// above the bound is written beside it (UpdateThreshold's candidate; the server takes the
// least over a request's words).  The launch's inputs and outputs may be page-locked host
// memory, read and written in place: h is copied out with the mask.
#include "common.cuh"

namespace cbdfs {
namespace {

__global__ void __launch_bounds__(256)
k_segment_bound(const uint8_t *__restrict__ h, const uint8_t *__restrict__ g,
                const uint16_t *__restrict__ word_req, const uint32_t *__restrict__ req_end,
                const uint32_t *__restrict__ req_bound, uint32_t n_words, uint8_t *__restrict__ h_out,
                uint32_t *__restrict__ mask, uint32_t *__restrict__ minw) {
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= n_words) return;  // whole warps: the ballot below sees every lane
    const uint32_t k = word_req[w];
    if (k == 0xFFFFu) {
        if (lane == 0) {
            mask[w] = 0;
            minw[w] = 0xFFFFFFFFu;
        }
        return;
    }
    const uint32_t r = w * 32 + lane;
    const bool valid = r < req_end[k];
    const uint32_t hv = h[r];
    h_out[r] = (uint8_t)hv;
    const uint32_t f = valid ? (uint32_t)g[r] + hv : 0xFFFFFFFFu;
    const bool pass = valid && f <= req_bound[k];
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
    const uint32_t m = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
    if (lane == 0) {
        mask[w] = bits;
        minw[w] = m;
    }
}

}  // namespace

int segment_bound(const uint8_t *d_h, const uint8_t *d_g, const uint16_t *d_word_req, const uint32_t *d_req_end,
                  const uint32_t *d_req_bound, uint32_t n_words, uint8_t *h_out, uint32_t *d_mask, uint32_t *d_minw,
                  cudaStream_t st) {
    if (n_words == 0) return CBDFS_OK;
    const uint32_t blocks = (n_words + 7) / 8;
    k_segment_bound<<<blocks, 256, 0, st>>>(d_h, d_g, d_word_req, d_req_end, d_req_bound, n_words, h_out, d_mask,
                                            d_minw);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

}  // namespace cbdfs
