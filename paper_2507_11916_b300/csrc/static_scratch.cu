// static_scratch.cu -- heur_eval_device_static: the device-buffer heuristic evaluation
// with no device-memory allocation in the call.
//
// Some callers cannot call cudaMalloc when they evaluate a batch: code that must not touch
// the allocator on its hot path (a real-time or latency-budgeted caller), a host process
// whose device memory is owned by another framework's allocator, or a caller whose budget
// is already spent.  For them the activation scratch of the network layers lives in a
// file-scope device array, reserved when the library is loaded on a device and held there
// until the process exits, instead of the context's allocated buffers.  The weights were
// placed on the device earlier, by cbdfs_net_load.
//
// Host code cannot use the array's name as a device address (in host code it names a
// host-side stand-in), so the first call on each device, with that device current, asks the
// runtime for the address with cudaGetSymbolAddress and keeps it.
#include "common.cuh"

namespace cbdfs {
namespace {

// one activation buffer; the array holds two (the layers ping-pong between them)
constexpr size_t kStaticHalf = 16ull << 20;

static __device__ __align__(256) uint8_t g_static_scratch[2 * kStaticHalf];

struct StaticDevice {
    std::mutex mu;
    bool ready = false;
    Slot slot;  // act[0], act[1] point into g_static_scratch; TMA maps cached in slot.tm_act
};
constexpr int kMaxDevices = 64;
StaticDevice g_static[kMaxDevices];

// bytes one activation buffer needs for n states of this network
size_t need_bytes(const NetGPU &net, uint32_t n, int *elem_out) {
    const size_t rows_pad = (n + kBM - 1) / kBM * kBM;
    size_t width = 0;
    for (int l = 1; l < net.L; ++l) width = std::max(width, (size_t)net.dims[l]);
    const int elem = net.prec == CBDFS_PREC_FP32 ? 4 : 2;  // FP8 layers feed the head in BF16
    *elem_out = elem;
    return rows_pad * width * elem;
}

}  // namespace
}  // namespace cbdfs

using namespace cbdfs;

extern "C" int heur_eval_device_static(cbdfs_ctx *ctx, int heur_id, int domain,
                                       const uint64_t *d_states, const uint8_t *d_g, uint32_t bound,
                                       uint32_t n, uint8_t *d_h, uint32_t *d_mask, uint32_t *d_minf,
                                       void *stream) {
    if (!ctx || !d_minf || (n && (!d_states || !d_g || !d_h || !d_mask))) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (domain < 0 || domain > 2) return fail(CBDFS_EINVAL, "domain %d", domain);
    if (n > c->max_batch) return fail(CBDFS_EINVAL, "n=%u exceeds max_batch=%u", n, c->max_batch);
    if (heur_id >= (int)c->heur_kind.size() || heur_id < CBDFS_HEUR_MD)
        return fail(CBDFS_EINVAL, "unknown heuristic id %d", heur_id);
    if (heur_id == CBDFS_HEUR_MD && domain == CBDFS_DOM_RC3)
        return fail(CBDFS_EINVAL, "Manhattan distance is defined for sliding-tile domains only");
    if (heur_is_real(c, heur_id)) return fail(CBDFS_EINVAL, "heuristic %d is real-valued", heur_id);
    if (heur_id >= 0 && c->heur_kind[heur_id] == 2) return fail(CBDFS_EINVAL, "heuristic %d is a composite", heur_id);
    if (c->device < 0 || c->device >= kMaxDevices) return fail(CBDFS_EINVAL, "device %d", c->device);
    CUDA_TRY(cudaSetDevice(c->device));
    StaticDevice &D = g_static[c->device];
    std::lock_guard<std::mutex> lk(D.mu);
    if (!D.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(CBDFS_EDEVICE, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        D.slot.act[0] = p;
        D.slot.act[1] = static_cast<uint8_t *>(p) + kStaticHalf;
        D.ready = true;
    }
    if (heur_id >= 0 && c->heur_kind[heur_id] == 0) {
        const NetGPU &net = *c->nets[c->heur_index[heur_id]];
        int elem = 2;
        const size_t need = need_bytes(net, n, &elem);
        if (need > kStaticHalf) {
            size_t width = need / ((n + kBM - 1) / kBM * kBM) / elem;
            const size_t max_states = kStaticHalf / (width * elem) / kBM * kBM;
            return fail(CBDFS_EINVAL,
                        "n=%u needs %zu bytes per static activation buffer, above the limit of %zu "
                        "bytes (at most %zu states for this network)",
                        n, need, kStaticHalf, max_states);
        }
        if (net.prec != CBDFS_PREC_FP32) {
            // TMA maps over the static buffers, keyed as the evaluation pipeline looks them
            // up (buffer << 40 | element bytes << 32 | width), with the rows the buffer holds
            const int eb = net.prec == CBDFS_PREC_FP8 ? 1 : 2;
            for (int l = 1; l < net.L - 1; ++l)
                for (int buf = 0; buf < 2; ++buf) {
                    const int K = net.dims[l];
                    const long long key = ((long long)buf << 40) | ((long long)eb << 32) | K;
                    if (D.slot.tm_act.count(key)) continue;
                    CUtensorMap m;
                    int rc = make_tmap_2d(&m, D.slot.act[buf],
                                          eb == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                          eb, (uint64_t)K, kStaticHalf / ((size_t)K * eb), 128 / eb, kBM);
                    if (rc) return rc;
                    D.slot.tm_act.emplace(key, m);
                }
        }
    }
    return run_eval(c, D.slot, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, nullptr,
                    reinterpret_cast<cudaStream_t>(stream));
}
