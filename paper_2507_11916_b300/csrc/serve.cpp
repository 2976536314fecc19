// serve.cpp -- continuous batching of heuristic requests (the paper's batch-processing
// thread, section "SingleGPU Batch CB-DFS": states from many searching threads are gathered
// into batches, evaluated on the GPU and handed back; more than one batch is kept in flight).
//
// A server thread owns some of the context's slots.  Requests (host buffers) queue up from
// any number of threads.  Whenever a slot is free and the device-memory budget allows, the
// server takes queued requests for one heuristic, in arrival order, into one launch of up to
// bucket_max states, copies them into the slot's pinned staging buffer and replays the CUDA
// graph captured for (slot, heuristic, bucket), bucket = the next power of two >= the states
// taken.  The graph holds the upload, the evaluation pipeline and the download; launches on
// different slots overlap on the device.  At completion each request gets its rows of h and
// its own bound test (mask, least f above its bound), computed from its g and bound.  Every
// row's h depends only on that row's state, so a request's result is the same whatever it
// was batched with.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>

#include <cuda_runtime.h>

#include "common.cuh"

namespace cbdfs {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    int heur, domain;
    const uint64_t *states;
    const uint8_t *g;
    uint32_t bound, n;
    uint8_t *h_out;
    uint32_t *mask_out, *minf_out;
    Clock::time_point t_submit;
    int status = 1;  // 1 pending, 0 done, < 0 error
};

struct Launch {
    int slot;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<uint32_t> offs;
    uint32_t total, bucket;
    size_t bytes;
    cudaEvent_t ev;
};

struct SlotIO {
    uint64_t *h_states = nullptr;  // pinned staging
    uint8_t *h_g = nullptr, *h_h = nullptr;
    // (heur, domain, bucket) -> instantiated graph and the scratch generation it was captured at
    std::map<long long, std::pair<uint64_t, cudaGraphExec_t>> graphs;
};

}  // namespace

struct Server {
    Ctx *c = nullptr;
    cbdfs_server_cfg cfg{};
    std::vector<int> slots;
    std::vector<SlotIO> io;
    std::vector<char> slot_busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> table;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thr;
    size_t mem_inflight = 0;
    // statistics
    std::vector<double> lat_us;
    uint64_t n_req = 0, n_states = 0, n_launch = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
    int error = 0;
    std::string error_msg;
};

namespace {

size_t launch_bytes(Ctx *c, uint32_t bucket) {
    // activation scratch a launch of this size touches (two BF16 buffers of the widest layer)
    return (size_t)bucket * std::max<size_t>(c->max_width, 1) * 2 * 2 + (size_t)bucket * 16;
}

int get_graph(Server &S, int si, int heur, int domain, uint32_t bucket, cudaGraphExec_t *out) {
    Ctx *c = S.c;
    SlotIO &io = S.io[si];
    const long long key = ((long long)heur << 40) ^ ((long long)domain << 32) ^ bucket;
    auto it = io.graphs.find(key);
    if (it != io.graphs.end()) {
        if (it->second.first == c->buf_gen) {
            *out = it->second.second;
            return CBDFS_OK;
        }
        cudaGraphExecDestroy(it->second.second);  // captured against scratch that has since moved
        io.graphs.erase(it);
    }
    Slot &sl = c->slots[S.slots[si]];
    cudaStream_t st = sl.stream;
    const int w = dom_words(domain);
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = CBDFS_OK;
    if (cudaMemcpyAsync(sl.d_states, io.h_states, (size_t)bucket * 8 * w, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(sl.d_g, io.h_g, bucket, cudaMemcpyHostToDevice, st))
        rc = fail(CBDFS_EDEVICE, "capture upload");
    if (!rc)
        rc = run_eval(c, sl, heur, domain, sl.d_states, sl.d_g, 255, bucket, sl.d_h, sl.d_mask, sl.d_minf,
                      nullptr, st);
    if (!rc && cudaMemcpyAsync(io.h_h, sl.d_h, bucket, cudaMemcpyDeviceToHost, st))
        rc = fail(CBDFS_EDEVICE, "capture download");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (!rc && e != cudaSuccess) rc = fail(CBDFS_EDEVICE, "graph capture: %s", cudaGetErrorString(e));
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CBDFS_EDEVICE, "graph instantiate: %s", cudaGetErrorString(e));
    io.graphs.emplace(key, std::make_pair(c->buf_gen, ex));
    *out = ex;
    return CBDFS_OK;
}

uint32_t bucket_of(const Server &S, uint32_t n) {
    uint32_t b = std::max<uint32_t>(S.cfg.bucket_min, 1);
    while (b < n) b <<= 1;
    return b;
}

void finish(Server &S, Launch &L) {
    const SlotIO &io = S.io[L.slot];
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(S.mu);
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request &r = *L.reqs[k];
        const uint8_t *h = io.h_h + L.offs[k];
        memcpy(r.h_out, h, r.n);
        uint32_t minf = 0xFFFFFFFFu;
        for (uint32_t w = 0; w < (r.n + 31) / 32; ++w) r.mask_out[w] = 0;
        for (uint32_t i = 0; i < r.n; ++i) {
            const uint32_t f = (uint32_t)r.g[i] + h[i];
            if (f <= r.bound) r.mask_out[i >> 5] |= 1u << (i & 31);
            else minf = std::min(minf, f);
        }
        *r.minf_out = minf;
        r.status = 0;
        S.lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
        S.n_req++;
        S.n_states += r.n;
    }
    S.t_last = now;
    S.mem_inflight -= L.bytes;
    S.slot_busy[L.slot] = 0;
    S.cv_done.notify_all();
}

void fail_launch(Server &S, Launch &L, int rc) {
    std::lock_guard<std::mutex> lk(S.mu);
    for (auto &r : L.reqs) r->status = rc;
    S.mem_inflight -= L.bytes;
    S.slot_busy[L.slot] = 0;
    S.cv_done.notify_all();
}

void server_loop(Server *Sp) {
    Server &S = *Sp;
    Ctx *c = S.c;
    cudaSetDevice(c->device);
    std::vector<Launch> inflight;
    for (;;) {
        bool progress = false;
        // completions
        for (size_t i = 0; i < inflight.size();) {
            const cudaError_t q = cudaEventQuery(inflight[i].ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (q == cudaSuccess) finish(S, inflight[i]);
            else fail_launch(S, inflight[i], fail(CBDFS_EDEVICE, "request launch: %s", cudaGetErrorString(q)));
            cudaEventDestroy(inflight[i].ev);
            inflight[i] = std::move(inflight.back());
            inflight.pop_back();
            progress = true;
        }
        // admissions
        for (;;) {
            Launch L;
            {
                std::unique_lock<std::mutex> lk(S.mu);
                if (S.stop && S.queue.empty() && inflight.empty()) return;
                if (S.queue.empty()) break;
                int si = -1;
                for (size_t k = 0; k < S.slot_busy.size(); ++k)
                    if (!S.slot_busy[k]) { si = (int)k; break; }
                if (si < 0) break;
                // take requests of the first queued heuristic, in order, up to bucket_max
                const int heur = S.queue.front()->heur, dom = S.queue.front()->domain;
                uint32_t total = 0;
                std::vector<std::shared_ptr<Request>> take;
                for (auto it = S.queue.begin(); it != S.queue.end();) {
                    Request &r = **it;
                    if (r.heur != heur || r.domain != dom) {
                        if (!S.cfg.coalesce) break;
                        ++it;
                        continue;
                    }
                    if (!take.empty() && (!S.cfg.coalesce || total + r.n > S.cfg.bucket_max)) break;
                    take.push_back(*it);
                    total += r.n;
                    it = S.queue.erase(it);
                }
                const uint32_t bucket = bucket_of(S, total);
                const size_t bytes = launch_bytes(c, bucket);
                if (S.cfg.mem_budget && S.mem_inflight + bytes > S.cfg.mem_budget && !inflight.empty()) {
                    // over the budget: put them back and wait for a completion
                    for (auto r = take.rbegin(); r != take.rend(); ++r) S.queue.push_front(*r);
                    break;
                }
                S.slot_busy[si] = 1;
                S.mem_inflight += bytes;
                L.slot = si;
                L.reqs = std::move(take);
                L.total = total;
                L.bucket = bucket;
                L.bytes = bytes;
            }
            // stage and launch (outside the lock)
            SlotIO &io = S.io[L.slot];
            const int w = dom_words(L.reqs[0]->domain);
            uint32_t off = 0;
            for (auto &r : L.reqs) {
                L.offs.push_back(off);
                memcpy(io.h_states + (size_t)off * w, r->states, (size_t)r->n * 8 * w);
                memcpy(io.h_g + off, r->g, r->n);
                off += r->n;
            }
            memset(io.h_states + (size_t)off * w, 0, (size_t)(L.bucket - off) * 8 * w);
            memset(io.h_g + off, 0, L.bucket - off);
            cudaGraphExec_t ex = nullptr;
            int rc = get_graph(S, L.slot, L.reqs[0]->heur, L.reqs[0]->domain, L.bucket, &ex);
            Slot &sl = c->slots[S.slots[L.slot]];
            if (!rc && cudaGraphLaunch(ex, sl.stream) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "graph launch");
            if (!rc && cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess)
                rc = fail(CBDFS_EDEVICE, "event");
            if (!rc && cudaEventRecord(L.ev, sl.stream) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "event record");
            if (rc) {
                fail_launch(S, L, rc);
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(S.mu);
                S.n_launch++;
            }
            inflight.push_back(std::move(L));
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(S.mu);
            if (S.stop && S.queue.empty() && inflight.empty()) return;
            if (inflight.empty()) S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
            else {
                lk.unlock();
                std::this_thread::yield();
            }
        }
    }
}

}  // namespace

void server_free(Ctx *c, Server *S) {
    if (!S) return;
    for (auto &io : S->io) {
        for (auto &kv : io.graphs) cudaGraphExecDestroy(kv.second.second);
        cudaFreeHost(io.h_states);
        cudaFreeHost(io.h_g);
        cudaFreeHost(io.h_h);
    }
    {
        std::lock_guard<std::mutex> lk(c->slot_mu);
        for (int i : S->slots) c->slots[i].busy = false;
    }
    c->slot_cv.notify_all();
    delete S;
}

}  // namespace cbdfs

using namespace cbdfs;

extern "C" {

int cbdfs_server_start(cbdfs_ctx *ctx, const cbdfs_server_cfg *cfg) {
    if (!ctx || !cfg) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (c->server) return fail(CBDFS_EINVAL, "a server is already running on this context");
    cbdfs_server_cfg sc = *cfg;
    if (sc.bucket_min == 0) sc.bucket_min = 32;
    if (sc.bucket_max == 0) sc.bucket_max = 4096;
    if (sc.bucket_max > c->max_batch || sc.bucket_min > sc.bucket_max)
        return fail(CBDFS_EINVAL, "buckets %u..%u outside 1..max_batch", sc.bucket_min, sc.bucket_max);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(CBDFS_EDEVICE, "cudaSetDevice");
    auto *S = new Server();
    S->c = c;
    S->cfg = sc;
    {
        std::lock_guard<std::mutex> lk(c->slot_mu);
        const int want = sc.max_inflight > 0 ? sc.max_inflight : (int)c->slots.size() - 1;
        for (int i = 1; i < (int)c->slots.size() && (int)S->slots.size() < want; ++i)
            if (!c->slots[i].busy) {
                c->slots[i].busy = true;
                S->slots.push_back(i);
            }
    }
    if (S->slots.empty()) {
        server_free(c, S);
        return fail(CBDFS_EINVAL, "no free slot for the server");
    }
    S->io.resize(S->slots.size());
    S->slot_busy.assign(S->slots.size(), 0);
    for (auto &io : S->io) {
        const size_t b = sc.bucket_max;
        if (cudaMallocHost(&io.h_states, b * 16) || cudaMallocHost(&io.h_g, b) || cudaMallocHost(&io.h_h, b)) {
            server_free(c, S);
            return fail(CBDFS_ENOMEM, "pinned staging");
        }
    }
    c->server = S;
    S->thr = std::thread(server_loop, S);
    return CBDFS_OK;
}

int cbdfs_server_stop(cbdfs_ctx *ctx) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return CBDFS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->thr.join();
    c->server = nullptr;
    server_free(c, S);
    return CBDFS_OK;
}

int heur_request_submit(cbdfs_ctx *ctx, int heur_id, int domain, const uint64_t *states, const uint8_t *g,
                        uint32_t bound, uint32_t n, uint8_t *h_out, uint32_t *mask_out, uint32_t *minf_out,
                        cbdfs_ticket *t) {
    if (!ctx || !states || !g || !h_out || !mask_out || !minf_out || !t || n == 0)
        return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    if (n > S->cfg.bucket_max) return fail(CBDFS_EINVAL, "n=%u above the largest bucket %u", n, S->cfg.bucket_max);
    if (domain < 0 || domain > 2) return fail(CBDFS_EINVAL, "domain %d", domain);
    if (heur_id >= (int)c->heur_kind.size() || heur_id < CBDFS_HEUR_MD ||
        (heur_id == CBDFS_HEUR_MD && domain == CBDFS_DOM_RC3))
        return fail(CBDFS_EINVAL, "heuristic id %d", heur_id);
    if (heur_is_real(c, heur_id)) return fail(CBDFS_EINVAL, "heuristic %d is real-valued", heur_id);
    auto r = std::make_shared<Request>();
    r->heur = heur_id;
    r->domain = domain;
    r->states = states;
    r->g = g;
    r->bound = bound;
    r->n = n;
    r->h_out = h_out;
    r->mask_out = mask_out;
    r->minf_out = minf_out;
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(CBDFS_ECANCELED, "the server is stopping");
        r->id = S->next_id++;
        S->table[r->id] = r;
        S->queue.push_back(r);
        if (!S->any) {
            S->any = true;
            S->t_first = r->t_submit;
        }
    }
    S->cv_work.notify_one();
    t->id = r->id;
    return CBDFS_OK;
}

int heur_request_wait(cbdfs_ctx *ctx, cbdfs_ticket t, uint64_t timeout_us) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->table.find(t.id);
    if (it == S->table.end()) return fail(CBDFS_EINVAL, "unknown ticket %llu", (unsigned long long)t.id);
    std::shared_ptr<Request> r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    while (r->status == 1) {
        if (timeout_us == 0 || S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (r->status == 1) return fail(CBDFS_ETIMEDOUT, "request %llu not done", (unsigned long long)t.id);
        }
    }
    S->table.erase(t.id);
    return r->status;
}

int cbdfs_server_get_stats(cbdfs_ctx *ctx, cbdfs_server_stats *out) {
    if (!ctx || !out) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->requests = S->n_req;
    out->states = S->n_states;
    out->launches = S->n_launch;
    if (!S->lat_us.empty()) {
        std::vector<double> v = S->lat_us;
        std::sort(v.begin(), v.end());
        out->p50_us = v[v.size() / 2];
        out->p99_us = v[std::min(v.size() - 1, (size_t)(0.99 * v.size()))];
        double s = 0;
        for (double x : v) s += x;
        out->mean_us = s / v.size();
        const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
        out->states_per_s = span > 0 ? S->n_states / span : 0;
    }
    return CBDFS_OK;
}

}  // extern "C"
