// rc_pdb.cu -- the cube's 8-corner pattern database (Experimental Setup: the cube's h_PDB is
// the 8-corner PDB; section "Fixed-Tree Evaluation": it prunes while the network is
// evaluated on every node).
//
// Index of a corner configuration, with p_c the slot of corner cubie c and t_c its twist
// (field c of the packed word 0 is 3 p_c + t_c):
//   index = rank(p) * 3^7 + sum_{c<7} t_c 3^c,  rank(p) = sum_i (p_i - #{j<i : p_j<p_i}) (7-i)!
// 8! * 3^7 = 88,179,840 one-byte entries; t_7 follows from the twist sum being 0 mod 3.
//
// k_corner_level: one thread per index; an entry at distance d applies the 18 face turns to
// its configuration and marks every unseen result d+1 (writers of one entry in one level all
// write d+1, so the race is benign).  Levels run until one marks nothing.
// k_corner_gather: one state per lane; the table byte (at index / div for a DIV-compressed
// table), the goal rule and the bound test
// (ballot mask word, warp and block minimum of f above the bound, one atomicMin per block).
#include "common.cuh"
#include "domain.h"

namespace cbdfs {
namespace {

using namespace dev;

constexpr uint32_t kCornerEntries = 40320u * 2187u;

__constant__ uint8_t c_dst[18][8], c_add[18][8];

__device__ __forceinline__ uint32_t corner_index(const int (&p)[8], const int (&t)[8]) {
    constexpr uint32_t F[8] = {5040, 720, 120, 24, 6, 2, 1, 1};
    uint32_t seen = 0, r = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        r += (uint32_t)(p[i] - __popc(seen & ((1u << p[i]) - 1u))) * F[i];
        seen |= 1u << p[i];
    }
    uint32_t tw = 0, pw = 1;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        tw += (uint32_t)t[c] * pw;
        pw *= 3;
    }
    return r * 2187u + tw;
}

__global__ void __launch_bounds__(256) k_corner_level(uint8_t *table, int d, int *grew) {
    constexpr uint32_t F[8] = {5040, 720, 120, 24, 6, 2, 1, 1};
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kCornerEntries || table[idx] != d) return;
    int p[8], t[8];
    uint32_t r = idx / 2187u, tr = idx % 2187u, used = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t k = r / F[i];
        r %= F[i];
        int s = 0;
        for (; s < 8; ++s) {  // the k-th free slot
            if (used & (1u << s)) continue;
            if (k == 0) break;
            --k;
        }
        p[i] = s;
        used |= 1u << s;
    }
    int sum = 0;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        t[c] = (int)(tr % 3u);
        tr /= 3u;
        sum += t[c];
    }
    t[7] = (3 - sum % 3) % 3;
    bool found = false;
    for (int m = 0; m < 18; ++m) {
        int np[8], nt[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            np[c] = c_dst[m][p[c]];
            nt[c] = (t[c] + c_add[m][p[c]]) % 3;
        }
        const uint32_t v = corner_index(np, nt);
        if (table[v] == 255) {
            table[v] = (uint8_t)(d + 1);
            found = true;
        }
    }
    if (found) atomicExch(grew, 1);
}

__global__ void __launch_bounds__(256)
k_corner_gather(const uint64_t *__restrict__ states, uint32_t n, const uint8_t *__restrict__ table, uint32_t div,
                const uint8_t *__restrict__ g, uint32_t bound, uint8_t *__restrict__ h_out,
                uint32_t *__restrict__ mask, uint32_t *__restrict__ minf) {
    __shared__ uint32_t warp_min[8];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    uint32_t f = 0xFFFFFFFFu;
    bool pass = false;
    if (valid) {
        const ulonglong2 w = reinterpret_cast<const ulonglong2 *>(states)[i];
        int p[8], t[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int fld = (int)((w.x >> (5 * c)) & 31u);
            p[c] = fld / 3;
            t[c] = fld % 3;
        }
        // a malformed word (a field above 23, or two cubies on one slot) would index past the
        // table: clamp, so that such input gives a meaningless h but no out-of-bounds read
        uint32_t hv = __ldg(table + min(corner_index(p, t), kCornerEntries - 1u) / div);
        hv = rc_is_goal(w.x, w.y) ? 0u : hv;
        h_out[i] = (uint8_t)hv;
        f = (uint32_t)g[i] + hv;
        pass = f <= bound;
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
    const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
    if (lane == 0) {
        if (i < n) mask[i >> 5] = bits;
        warp_min[warp] = mn;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t mm = __reduce_min_sync(0xFFFFFFFFu, lane < (int)(blockDim.x >> 5) ? warp_min[lane] : 0xFFFFFFFFu);
        if (lane == 0 && mm != 0xFFFFFFFFu) atomicMin(minf, mm);
    }
}

}  // namespace

size_t rc_corner_entries() { return kCornerEntries; }

// div: the table's DIV compression (1: none)
int rc_corner_gather(const uint8_t *table, uint32_t div, const uint64_t *states, uint32_t n, const uint8_t *g,
                     uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf, cudaStream_t st) {
    if (n == 0) return CBDFS_OK;
    k_corner_gather<<<(n + 255) / 256, 256, 0, st>>>(states, n, table, div, g, bound, h, mask, minf);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

// The 8-corner table into the device buffer `table` (kCornerEntries bytes).
int rc_corner_build_device(Ctx *c, uint8_t *table, cudaStream_t st) {
    uint8_t dst[18][8], add[18][8];
    rc_corner_moves(dst, add);
    CUDA_TRY(cudaMemcpyToSymbolAsync(c_dst, dst, sizeof(dst), 0, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyToSymbolAsync(c_add, add, sizeof(add), 0, cudaMemcpyHostToDevice, st));
    int *grew = nullptr;
    int rc = dev_alloc(c, (void **)&grew, sizeof(int));
    if (rc) return rc;
    const uint8_t zero = 0;
    int status = CBDFS_OK;
    if (cudaMemsetAsync(table, 255, kCornerEntries, st) != cudaSuccess ||
        cudaMemcpyAsync(table, &zero, 1, cudaMemcpyHostToDevice, st) != cudaSuccess)  // the solved corners: index 0
        status = fail(CBDFS_EDEVICE, "corner table init");
    const unsigned blocks = (kCornerEntries + 255) / 256;
    for (int d = 0; d < 254 && status == CBDFS_OK; ++d) {
        int h_grew = 0;
        cudaMemsetAsync(grew, 0, sizeof(int), st);
        k_corner_level<<<blocks, 256, 0, st>>>(table, d, grew);
        cudaMemcpyAsync(&h_grew, grew, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess)
            status = fail(CBDFS_EDEVICE, "corner table level %d: %s", d, cudaGetErrorString(cudaGetLastError()));
        else if (!h_grew)
            break;
    }
    dev_free(c, grew, sizeof(int));
    return status;
}

}  // namespace cbdfs
