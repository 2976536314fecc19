// pdb.cu -- additive pattern databases on the GPU.
//
// k_pdb_gather: the plain heuristic and fallback.  One state per lane: the packed state is
// inverted in registers (where[tile] = cell, a 64-bit nibble word), each pattern's cells
// are ranked lexicographically among the k-permutations of the N cells with popcounts, the
// table bytes are gathered (all patterns' loads issued together; when the host marks some
// tables to keep in L2, with an evict-last priority for theirs and evict-first for the
// others') and summed; the warp then
// forms the bound-test mask word with a ballot and the least f above the bound with a
// reduction.  (Paper, Background: PDB heuristics; Experimental Setup: additive tile PDBs.)
//
// pdb_build: breadth-first search over the abstract space (cells of the pattern tiles +
// blank cell).  dist[r*16 + b] holds the distance of placement rank r with the blank on cell
// b.  Per cost level d:
//   k_closure  one thread per rank: flood-fills the blank over the empty cells (zero-cost
//              moves) from the cells at distance d, in 16-bit masks;
//   k_expand   one thread per rank with cells at level d: every blank move that pushes a
//              pattern tile (cost 1) marks the new (rank, blank) entry d+1 if unseen.
// The closure of level d finishes before any level-d+1 entry is written, so no entry that
// deserves d is ever marked d+1.  k_reduce then takes the minimum over blank cells.
#include "common.cuh"

namespace cbdfs {

namespace {

using namespace dev;

// a table byte through L2 with an eviction priority (a cache-policy operand from createpolicy)
__device__ __forceinline__ uint32_t ld_table_byte(const uint8_t *p, uint64_t policy) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
    return v;
}

template <int SIDE>
__global__ void __launch_bounds__(256)
k_pdb_gather(const uint64_t *__restrict__ states, uint32_t n, const PdbParams P,
             const uint8_t *__restrict__ g, uint32_t bound, uint8_t *__restrict__ h_out,
             uint32_t *__restrict__ mask, uint32_t *__restrict__ minf) {
    constexpr int N = SIDE * SIDE;
    __shared__ uint32_t warp_min[8];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    uint64_t goal = 0;
#pragma unroll
    for (int t = 0; t < N; ++t) goal |= (uint64_t)t << (4 * t);
    const uint64_t s = valid ? __ldg(states + i) : goal;
    const uint32_t gi = valid ? (uint32_t)__ldg(g + i) : 0u;
    uint64_t where = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) where |= (uint64_t)p << (4 * ((s >> (4 * p)) & 15u));
    // Both loops are unrolled to their maxima so that every PdbParams field is read at a
    // constant offset (an instruction operand), never by a dynamic index into the
    // parameter bank; the pattern sizes are the same for all threads, so the guards are
    // uniform branches.
    uint32_t rank[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t seen = 0, r = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (q < P.n_patterns && j < P.k[q]) {
                const uint32_t c = (uint32_t)(where >> (4 * P.tiles[q][j])) & 15u;
                r += (c - __popc(seen & ((1u << c) - 1u))) * P.weight[q][j];
                seen |= 1u << c;
            }
        }
        rank[q] = r;
    }
    uint32_t v[4];
#pragma unroll
    // a malformed state (a repeated tile) can rank past its table: clamp, so that such input
    // gives a meaningless h but no out-of-bounds read
    if (P.l2_keep) {
        // the kept tables' lines are evicted last, the others' first (L2 eviction priority)
        uint64_t keep, stream;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[q] = (q < P.n_patterns)
                       ? ld_table_byte(P.table[q] + min(rank[q] / P.div, P.entries[q] - 1u),
                                       ((P.l2_keep >> q) & 1u) ? keep : stream)
                       : 0u;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (q < P.n_patterns) ? __ldg(P.table[q] + min(rank[q] / P.div, P.entries[q] - 1u)) : 0u;
    }
    uint32_t hv = v[0] + v[1] + v[2] + v[3];
    hv = (s == goal) ? 0u : min(hv, 255u);
    uint32_t f = 0xFFFFFFFFu;
    bool pass = false;
    if (valid) {
        h_out[i] = (uint8_t)hv;
        f = gi + hv;
        pass = f <= bound;
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pass);
    const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, pass ? 0xFFFFFFFFu : f);
    if (lane == 0) {
        if (i < n) mask[i >> 5] = bits;
        warp_min[warp] = mn;
    }
    // one atomic per block for the least f above the bound
    __syncthreads();
    if (warp == 0) {
        const uint32_t m = __reduce_min_sync(0xFFFFFFFFu, lane < (int)(blockDim.x >> 5) ? warp_min[lane] : 0xFFFFFFFFu);
        if (lane == 0 && m != 0xFFFFFFFFu) atomicMin(minf, m);
    }
}

// DIV compression: entry j = the least of the k entries j*k .. j*k+k-1 that exist
__global__ void __launch_bounds__(256) k_div_compress(const uint8_t *__restrict__ src, uint64_t n, uint32_t k,
                                                     uint8_t *__restrict__ dst, uint64_t m) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const uint64_t lo = j * k, hi = lo + k < n ? lo + k : n;
    uint32_t best = 255;
    for (uint64_t i = lo; i < hi; ++i) best = min(best, (uint32_t)__ldg(src + i));
    dst[j] = (uint8_t)best;
}

// ---- builder ---------------------------------------------------------------------------
struct BuildParams {
    int side, k;
    int tiles[8];
    uint32_t weight[8];
    uint64_t P;  // number of placements
};

__device__ __forceinline__ uint32_t unrank_mask(const BuildParams &B, uint64_t r, int (&pos)[8]) {
    uint32_t used = 0;
    for (int i = 0; i < B.k; ++i) {
        uint32_t d = (uint32_t)(r / B.weight[i]);
        r %= B.weight[i];
        // the d-th free cell
        int c = 0;
        for (; c < 16; ++c) {
            if (used & (1u << c)) continue;
            if (d == 0) break;
            --d;
        }
        pos[i] = c;
        used |= 1u << c;
    }
    return used;
}

__device__ __forceinline__ uint32_t rank_of(const BuildParams &B, const int (&pos)[8]) {
    uint32_t seen = 0, r = 0;
    for (int i = 0; i < B.k; ++i) {
        const uint32_t c = pos[i];
        r += (c - __popc(seen & ((1u << c) - 1u))) * B.weight[i];
        seen |= 1u << c;
    }
    return r;
}

// neighbours of a cell set on a side x side board
__device__ __forceinline__ uint32_t nbr_mask(uint32_t m, int side) {
    const int N = side * side;
    uint32_t colL = 0, colR = 0;  // cells in the first / last column
    for (int r = 0; r < side; ++r) {
        colL |= 1u << (r * side);
        colR |= 1u << (r * side + side - 1);
    }
    const uint32_t all = (N == 32) ? 0xFFFFFFFFu : ((1u << N) - 1u);
    return (((m & ~colL) >> 1) | ((m & ~colR) << 1) | (m >> side) | (m << side)) & all;
}

__global__ void k_closure(uint8_t *dist, BuildParams B, int d) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.P) return;
    uint4 *row4 = reinterpret_cast<uint4 *>(dist + r * 16);
    uint4 v = *row4;
    uint8_t *e = reinterpret_cast<uint8_t *>(&v);
    const int N = B.side * B.side;
    uint32_t F = 0, seen = 0;
    for (int b = 0; b < N; ++b) {
        if (e[b] == d) F |= 1u << b;
        if (e[b] != 255) seen |= 1u << b;
    }
    if (!F) return;
    int pos[8];
    const uint32_t occ = unrank_mask(B, r, pos);
    const uint32_t empty = ((1u << N) - 1u) & ~occ;
    uint32_t reach = F, grow;
    while ((grow = nbr_mask(reach, B.side) & empty & ~seen & ~reach)) reach |= grow;
    const uint32_t add = reach & ~F & ~seen;
    if (!add) return;
    for (int b = 0; b < N; ++b)
        if (add & (1u << b)) e[b] = (uint8_t)d;
    *row4 = v;
}

__global__ void k_expand(uint8_t *dist, BuildParams B, int d, int *grew) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.P) return;
    const uint4 v = *reinterpret_cast<const uint4 *>(dist + r * 16);
    const uint8_t *e = reinterpret_cast<const uint8_t *>(&v);
    const int N = B.side * B.side;
    uint32_t F = 0;
    for (int b = 0; b < N; ++b)
        if (e[b] == d) F |= 1u << b;
    if (!F) return;
    int pos[8];
    unrank_mask(B, r, pos);
    int found = 0;
    for (int b = 0; b < N; ++b) {
        if (!(F & (1u << b))) continue;
        const int br = b / B.side, bc = b % B.side;
        const int nb[4] = {br > 0 ? b - B.side : -1, bc > 0 ? b - 1 : -1,
                           bc < B.side - 1 ? b + 1 : -1, br < B.side - 1 ? b + B.side : -1};
        for (int m = 0; m < 4; ++m) {
            const int c = nb[m];
            if (c < 0) continue;
            for (int i = 0; i < B.k; ++i) {
                if (pos[i] != c) continue;
                int np[8];
                for (int j = 0; j < 8; ++j) np[j] = pos[j];
                np[i] = b;  // the tile slides into the blank's cell; the blank goes to c
                const uint64_t vi = (uint64_t)rank_of(B, np) * 16 + c;
                if (dist[vi] == 255) {
                    dist[vi] = (uint8_t)(d + 1);
                    found = 1;
                }
            }
        }
    }
    if (found) atomicExch(grew, 1);
}

__global__ void k_reduce(const uint8_t *dist, BuildParams B, uint8_t *table) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.P) return;
    const uint4 v = *reinterpret_cast<const uint4 *>(dist + r * 16);
    const uint8_t *e = reinterpret_cast<const uint8_t *>(&v);
    uint8_t best = 255;
    for (int b = 0; b < B.side * B.side; ++b) best = e[b] < best ? e[b] : best;
    table[r] = best;
}

}  // namespace

uint64_t npk(int n, int k) {
    uint64_t r = 1;
    for (int i = 0; i < k; ++i) r *= (uint64_t)(n - i);
    return r;
}

int pdb_gather(int domain, const PdbParams &P, const uint64_t *states, uint32_t n, const uint8_t *g,
               uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf, cudaStream_t st) {
    if (n == 0) return CBDFS_OK;
    const unsigned blocks = (n + 255) / 256;
    if (domain == CBDFS_DOM_STP3)
        k_pdb_gather<3><<<blocks, 256, 0, st>>>(states, n, P, g, bound, h, mask, minf);
    else
        k_pdb_gather<4><<<blocks, 256, 0, st>>>(states, n, P, g, bound, h, mask, minf);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

int pdb_div_compress(const uint8_t *src, uint64_t n, uint32_t k, uint8_t *dst, cudaStream_t st) {
    const uint64_t m = (n + k - 1) / k;
    k_div_compress<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(src, n, k, dst, m);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

// Build one pattern's table into the device buffer `table` (npk(N,k) bytes).
int pdb_build_device(Ctx *c, int side, const int *tiles, int k, uint8_t *table, cudaStream_t st) {
    const int N = side * side;
    BuildParams B{};
    B.side = side;
    B.k = k;
    for (int i = 0; i < k; ++i) {
        B.tiles[i] = tiles[i];
        B.weight[i] = (uint32_t)npk(N - 1 - i, k - 1 - i) / 1;
    }
    // weight_i = (N-1-i)!/(N-k)! = npk(N-1-i, k-1-i)
    B.P = npk(N, k);
    const size_t bytes = B.P * 16;
    uint8_t *dist = nullptr;
    int *grew = nullptr;
    int rc = dev_alloc(c, (void **)&dist, bytes);
    if (rc) return rc;
    rc = dev_alloc(c, (void **)&grew, sizeof(int));
    if (rc) { dev_free(c, dist, bytes); return rc; }
    auto cleanup = [&]() { dev_free(c, dist, bytes); dev_free(c, grew, sizeof(int)); };
    if (cudaMemsetAsync(dist, 255, bytes, st) != cudaSuccess) { cleanup(); return fail(CBDFS_EDEVICE, "memset"); }
    int pos[8];
    for (int i = 0; i < k; ++i) pos[i] = tiles[i];
    uint64_t r0 = 0;
    {
        uint32_t seen = 0;
        for (int i = 0; i < k; ++i) {
            uint32_t cc = pos[i];
            r0 += (uint64_t)(cc - __builtin_popcount(seen & ((1u << cc) - 1u))) * B.weight[i];
            seen |= 1u << cc;
        }
    }
    const uint8_t zero = 0;
    if (cudaMemcpyAsync(dist + r0 * 16 + 0, &zero, 1, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cleanup();
        return fail(CBDFS_EDEVICE, "seed copy");
    }
    const unsigned blocks = (unsigned)((B.P + 255) / 256);
    int status = CBDFS_OK;
    for (int d = 0; d < 254; ++d) {
        k_closure<<<blocks, 256, 0, st>>>(dist, B, d);
        int h_grew = 0;
        cudaMemsetAsync(grew, 0, sizeof(int), st);
        k_expand<<<blocks, 256, 0, st>>>(dist, B, d, grew);
        cudaMemcpyAsync(&h_grew, grew, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            status = fail(CBDFS_EDEVICE, "pdb_build level %d: %s", d, cudaGetErrorString(cudaGetLastError()));
            break;
        }
        if (!h_grew) {
            // one more closure pass is not needed: level d was closed before expanding
            break;
        }
    }
    if (status == CBDFS_OK) {
        k_reduce<<<blocks, 256, 0, st>>>(dist, B, table);
        if (cudaStreamSynchronize(st) != cudaSuccess)
            status = fail(CBDFS_EDEVICE, "pdb_build reduce: %s", cudaGetErrorString(cudaGetLastError()));
    }
    cleanup();
    return status;
}

}  // namespace cbdfs
