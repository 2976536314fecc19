// combo.cu -- composite heuristics: h = [MD] + sum over groups of the minimum over the
// group's members (Related Work: the minimum over an ensemble of networks keeps the learned
// heuristic admissible; Experimental Setup: the 15-puzzle h_M adds two ensembles, each
// trained on one pattern's PDB minus Manhattan distance).
//
// Each member runs its own pipeline into the slot's member rows (run_eval in api.cu, with
// no bound test of its own); k_combine then reads the M member bytes of each state, forms the
// composite, applies the goal rule and the bound test (ballot mask word, warp and block
// minimum of f above the bound, one atomicMin per block).
#include "common.cuh"

namespace cbdfs {
namespace {

using namespace dev;

template <int DOMAIN>
__global__ void __launch_bounds__(256)
k_combine(const uint64_t *__restrict__ states, uint32_t n, const uint8_t *__restrict__ member_h,
          size_t member_stride, ComboParams C, const uint8_t *__restrict__ g, uint32_t bound,
          uint8_t *__restrict__ h_out, uint32_t *__restrict__ mask, uint32_t *__restrict__ minf) {
    __shared__ uint32_t warp_min[8];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    uint32_t f = 0xFFFFFFFFu;
    bool pass = false;
    if (valid) {
        uint32_t hv = 0;
        int m = 0;
        // groups and members unrolled to their maxima: constant parameter offsets, uniform guards
#pragma unroll
        for (int grp = 0; grp < kComboMaxGroups; ++grp) {
            if (grp < C.n_groups) {
                uint32_t lo = 255;
#pragma unroll
                for (int j = 0; j < kComboMaxMembers; ++j)
                    if (j < C.group_size[grp]) lo = min(lo, (uint32_t)member_h[(size_t)(m + j) * member_stride + i]);
                hv += lo;
                m += C.group_size[grp];
            }
        }
        bool goal;
        if (DOMAIN == CBDFS_DOM_RC3) {
            goal = rc_is_goal(states[2 * i], states[2 * i + 1]);
        } else {
            constexpr int SIDE = DOMAIN == CBDFS_DOM_STP3 ? 3 : 4;
            const uint64_t s = states[i];
            if (C.add_md) hv += (uint32_t)manhattan<SIDE>(s);
            goal = stp_is_goal<SIDE>(s);
        }
        hv = goal ? 0u : min(hv, 255u);
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

int combine(int domain, const ComboParams &C, const uint64_t *states, uint32_t n, const uint8_t *member_h,
            size_t member_stride, const uint8_t *g, uint32_t bound, uint8_t *h, uint32_t *mask, uint32_t *minf,
            cudaStream_t st) {
    const unsigned blocks = (n + 255) / 256;
    if (domain == CBDFS_DOM_STP3)
        k_combine<CBDFS_DOM_STP3><<<blocks, 256, 0, st>>>(states, n, member_h, member_stride, C, g, bound, h, mask, minf);
    else if (domain == CBDFS_DOM_STP4)
        k_combine<CBDFS_DOM_STP4><<<blocks, 256, 0, st>>>(states, n, member_h, member_stride, C, g, bound, h, mask, minf);
    else
        k_combine<CBDFS_DOM_RC3><<<blocks, 256, 0, st>>>(states, n, member_h, member_stride, C, g, bound, h, mask, minf);
    CUDA_TRY(cudaGetLastError());
    return CBDFS_OK;
}

}  // namespace cbdfs
