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
// different slots overlap on the device.  A completion thread copies results out and wakes
// callers while the server thread stages the next launch.  Each request starts on a 32-row
// boundary of the
// launch, so its bound test (mask words, least f above its own bound) runs on the device in
// the same graph (segbound.cu); at completion the server copies each request's rows of h, its
// mask words and its minimum out and wakes that request's waiters only.  Every row's h
// depends only on that row's state, so a request's result is the same whatever it was
// batched with.
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
    int status = 1;  // 1 pending, 0 done, < 0 error (under m)
    std::mutex m;    // its status and its waiters: a waiter never holds the server's mutex
    std::condition_variable cv;
};

void set_status(Request &r, int status) {
    {
        std::lock_guard<std::mutex> lk(r.m);
        r.status = status;
    }
    r.cv.notify_all();
}

struct Launch {
    int slot;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<uint32_t> offs;
    uint32_t total, bucket;
    size_t bytes;
    cudaEvent_t ev;
    Clock::time_point t_launch;
};

// A slot's staging, all in mapped page-locked host memory that the kernels read and write in
// place (no copies in a launch): the rows' states and g, the request table (the request of
// every 32-row mask word, 0xFFFF for padding; each request's row end and bound), and the
// results (h, mask words, each word's least f above its request's bound).
template <typename T> struct Mapped {
    T *h = nullptr;  // host address
    T *d = nullptr;  // device address
};
struct SlotIO {
    Mapped<uint64_t> states;
    Mapped<uint8_t> g, h;
    Mapped<uint16_t> word_req;
    Mapped<uint32_t> req;   // [max_req] row ends, then [max_req] bounds
    Mapped<uint32_t> out;   // [cap / 32] mask words, then [cap / 32] word minima
    cudaEvent_t ev = nullptr;  // the slot's launch is complete (one launch per slot at a time)
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
    std::thread thr, thr_done;   // the server (launch) thread and the completion thread
    size_t mem_inflight = 0;
    int n_inflight = 0;           // launches handed to the completion thread, not yet finished
    std::mutex fl_mu;             // the launches in flight, oldest first, and the end flag
    std::condition_variable fl_cv;
    std::deque<Launch> flight;
    bool launcher_done = false;
    // statistics
    std::vector<double> lat_us;
    uint64_t n_req = 0, n_states = 0, n_launch = 0;
    double stage_ns = 0, flight_ns = 0, finish_ns = 0, replay_ns = 0;  // time per part, summed
    Clock::time_point t_first, t_last;
    bool any = false;
    int error = 0;
    std::string error_msg;
};

namespace {

// rows a launch can hold: bucket_max rounded up to whole 32-row mask words (the staging size)
uint32_t cap_rows(const Server &S) { return (S.cfg.bucket_max + 31) / 32 * 32; }
// requests one launch can hold: each takes at least one 32-row mask word
uint32_t max_requests(const Server &S) { return cap_rows(S) / 32; }

// n elements of mapped page-locked memory: the host address and the device's
template <typename T> int map_alloc(Mapped<T> &m, size_t n) {
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, n * sizeof(T), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return 1;
    m.h = static_cast<T *>(h);
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) return 1;
    m.d = static_cast<T *>(d);
    return 0;
}

size_t launch_bytes(Ctx *c, uint32_t bucket) {
    // activation scratch a launch of this size touches (two BF16 buffers of the widest layer)
    return (size_t)bucket * std::max<size_t>(c->max_width, 1) * 2 * 2 + (size_t)bucket * 16;
}

// one launch's pipeline on the slot's stream: upload the staged rows, g and request table,
// evaluate, bound-test each request, download h, the mask words and the minima
int enqueue_pipeline(Server &S, int si, int heur, int domain, uint32_t bucket) {
    Ctx *c = S.c;
    SlotIO &io = S.io[si];
    Slot &sl = c->slots[S.slots[si]];
    const uint32_t words = bucket / 32, mr = max_requests(S), cw = cap_rows(S) / 32;
    int rc = run_eval(c, sl, heur, domain, io.states.d, io.g.d, 255, bucket, sl.d_h, sl.d_mask, sl.d_minf, nullptr,
                      sl.stream);
    if (!rc)
        rc = segment_bound(sl.d_h, io.g.d, io.word_req.d, io.req.d, io.req.d + mr, words, io.h.d, io.out.d,
                           io.out.d + cw, sl.stream);
    return rc;
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
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_pipeline(S, si, heur, domain, bucket);
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
    // upload now, so that the first replay does not pay for it
    if ((e = cudaGraphUpload(ex, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        cudaGraphExecDestroy(ex);
        return fail(CBDFS_EDEVICE, "graph upload: %s", cudaGetErrorString(e));
    }
    io.graphs.emplace(key, std::make_pair(c->buf_gen, ex));
    *out = ex;
    return CBDFS_OK;
}

// the size class of a launch of n rows (n a multiple of 32): the next power-of-two multiple of
// bucket_min, in whole 32-row words, at most the staging size
uint32_t bucket_of(const Server &S, uint32_t n) {
    uint32_t b = std::max<uint32_t>(S.cfg.bucket_min, 1);
    while (b < n) b <<= 1;
    b = (b + 31) / 32 * 32;
    return std::min(b, cap_rows(S));
}

void finish(Server &S, Launch &L) {
    const SlotIO &io = S.io[L.slot];
    // h, the mask words and the least f above the bound, all from the device, into the
    // callers' buffers (no lock: only this thread writes them until the status is set)
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request &r = *L.reqs[k];
        const uint32_t w0 = L.offs[k] / 32, nw = (r.n + 31) / 32, cw = cap_rows(S) / 32;
        memcpy(r.h_out, io.h.h + L.offs[k], r.n);
        memcpy(r.mask_out, io.out.h + w0, (size_t)nw * 4);
        uint32_t minf = 0xFFFFFFFFu;  // the least of its words' minima
        for (uint32_t w = w0; w < w0 + nw; ++w) minf = std::min(minf, io.out.h[cw + w]);
        *r.minf_out = minf;
    }
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (auto &rp : L.reqs) {
            S.lat_us.push_back(std::chrono::duration<double, std::micro>(now - rp->t_submit).count());
            S.n_req++;
            S.n_states += rp->n;
        }
        S.t_last = now;
        S.mem_inflight -= L.bytes;
        S.slot_busy[L.slot] = 0;
    }
    // the slot is free again (its results are copied out): let the server thread refill it
    // before the callers are woken one by one
    S.cv_work.notify_one();
    for (auto &rp : L.reqs) set_status(*rp, 0);
}

void fail_launch(Server &S, Launch &L, int rc) {
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.mem_inflight -= L.bytes;
        S.slot_busy[L.slot] = 0;
    }
    for (auto &r : L.reqs) set_status(*r, rc);
}

// The completion thread: waits for the oldest launch in flight, copies its results out to
// the callers' buffers, frees its slot for the server thread and wakes the callers (finish).
void completion_loop(Server *Sp) {
    Server &S = *Sp;
    cudaSetDevice(S.c->device);
    for (;;) {
        Launch L;
        {
            std::unique_lock<std::mutex> lk(S.fl_mu);
            S.fl_cv.wait(lk, [&] { return !S.flight.empty() || S.launcher_done; });
            if (S.flight.empty()) return;  // the server thread has ended and nothing is in flight
            L = std::move(S.flight.front());
            S.flight.pop_front();
        }
        const cudaError_t q = cudaEventSynchronize(L.ev);
        const auto t_done = Clock::now();
        if (q == cudaSuccess) finish(S, L);
        else fail_launch(S, L, fail(CBDFS_EDEVICE, "request launch: %s", cudaGetErrorString(q)));
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.flight_ns += std::chrono::duration<double, std::nano>(t_done - L.t_launch).count();
            S.finish_ns += std::chrono::duration<double, std::nano>(Clock::now() - t_done).count();
            S.n_inflight--;
        }
        S.cv_work.notify_one();
    }
}

// The server thread: takes queued requests into a launch whenever a slot is free, stages
// them, replays the graph of their size bucket and hands the launch to the completion thread.
void server_loop(Server *Sp) {
    Server &S = *Sp;
    Ctx *c = S.c;
    cudaSetDevice(c->device);
    for (;;) {
        Launch L;
        std::chrono::steady_clock::time_point t_adm;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            int si = -1;
            for (;;) {
                if (S.stop && S.queue.empty() && S.n_inflight == 0) {
                    lk.unlock();
                    {
                        std::lock_guard<std::mutex> fl(S.fl_mu);
                        S.launcher_done = true;
                    }
                    S.fl_cv.notify_all();
                    return;
                }
                si = -1;
                if (!S.queue.empty())
                    for (size_t k = 0; k < S.slot_busy.size(); ++k)
                        if (!S.slot_busy[k]) { si = (int)k; break; }
                if (si >= 0) {
                    // take requests of the first queued heuristic, in order, up to the
                    // staging size, each on a 32-row boundary
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
                        const uint32_t rows = (r.n + 31) / 32 * 32;
                        if (!take.empty() && (!S.cfg.coalesce || total + rows > cap_rows(S))) break;
                        take.push_back(*it);
                        total += rows;
                        it = S.queue.erase(it);
                    }
                    const uint32_t bucket = bucket_of(S, total);
                    const size_t bytes = launch_bytes(c, bucket);
                    if (!(S.cfg.mem_budget && S.mem_inflight + bytes > S.cfg.mem_budget && S.n_inflight > 0)) {
                        S.slot_busy[si] = 1;
                        S.mem_inflight += bytes;
                        S.n_inflight++;
                        L.slot = si;
                        L.reqs = std::move(take);
                        L.total = total;
                        L.bucket = bucket;
                        L.bytes = bytes;
                        break;
                    }
                    // over the memory budget: put them back and wait for a completion
                    for (auto r = take.rbegin(); r != take.rend(); ++r) S.queue.push_front(*r);
                }
                S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
            }
            t_adm = Clock::now();
        }
        // stage and launch (outside the lock): each request from a 32-row boundary, its mask
        // words marked with its index, its row end and bound in the request table.  Padding
        // rows keep what an earlier launch staged there (zeros at first): their h is computed
        // and never read, and their mask words belong to no request.
        SlotIO &io = S.io[L.slot];
        const int w = dom_words(L.reqs[0]->domain);
        uint32_t off = 0;
        const uint32_t mr = max_requests(S);
        for (uint32_t w32 = 0; w32 < L.bucket / 32; ++w32) io.word_req.h[w32] = 0xFFFFu;
        for (size_t k = 0; k < L.reqs.size(); ++k) {
            const Request &r = *L.reqs[k];
            const uint32_t rows = (r.n + 31) / 32 * 32;
            L.offs.push_back(off);
            memcpy(io.states.h + (size_t)off * w, r.states, (size_t)r.n * 8 * w);
            memcpy(io.g.h + off, r.g, r.n);
            for (uint32_t w32 = off / 32; w32 < (off + rows) / 32; ++w32) io.word_req.h[w32] = (uint16_t)k;
            io.req.h[k] = off + r.n;
            io.req.h[mr + k] = r.bound;
            off += rows;
        }
        cudaGraphExec_t ex = nullptr;
        int rc = S.cfg.direct ? CBDFS_OK : get_graph(S, L.slot, L.reqs[0]->heur, L.reqs[0]->domain, L.bucket, &ex);
        Slot &sl = c->slots[S.slots[L.slot]];
        const auto t_replay = Clock::now();
        if (S.cfg.direct) {
            if (!rc) rc = enqueue_pipeline(S, L.slot, L.reqs[0]->heur, L.reqs[0]->domain, L.bucket);
        } else if (!rc && cudaGraphLaunch(ex, sl.stream) != cudaSuccess) {
            rc = fail(CBDFS_EDEVICE, "graph launch");
        }
        L.ev = io.ev;
        if (!rc && cudaEventRecord(L.ev, sl.stream) != cudaSuccess) rc = fail(CBDFS_EDEVICE, "event record");
        if (rc) {
            fail_launch(S, L, rc);
            {
                std::lock_guard<std::mutex> lk(S.mu);
                S.n_inflight--;
            }
            continue;
        }
        L.t_launch = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.n_launch++;
            S.stage_ns += std::chrono::duration<double, std::nano>(L.t_launch - t_adm).count();
            S.replay_ns += std::chrono::duration<double, std::nano>(L.t_launch - t_replay).count();
        }
        {
            std::lock_guard<std::mutex> fl(S.fl_mu);
            S.flight.push_back(std::move(L));
        }
        S.fl_cv.notify_one();
    }
}

}  // namespace

void server_free(Ctx *c, Server *S) {
    if (!S) return;
    for (auto &io : S->io) {
        for (auto &kv : io.graphs) cudaGraphExecDestroy(kv.second.second);
        for (void *h : {(void *)io.states.h, (void *)io.g.h, (void *)io.h.h, (void *)io.word_req.h, (void *)io.req.h,
                        (void *)io.out.h})
            if (h) cudaFreeHost(h);
        if (io.ev) cudaEventDestroy(io.ev);
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
        const size_t b = cap_rows(*S), mr = max_requests(*S);
        if (map_alloc(io.states, b * 2) || map_alloc(io.g, b) || map_alloc(io.h, b) ||
            map_alloc(io.word_req, b / 32) || map_alloc(io.req, 2 * mr) || map_alloc(io.out, 2 * (b / 32))) {
            server_free(c, S);
            return fail(CBDFS_ENOMEM, "mapped page-locked staging");
        }
        if (cudaEventCreateWithFlags(&io.ev, cudaEventDisableTiming) != cudaSuccess) {
            server_free(c, S);
            return fail(CBDFS_EDEVICE, "event");
        }
        memset(io.states.h, 0, b * 16);  // padding rows start as zeros
        memset(io.g.h, 0, b);
    }
    c->server = S;
    S->thr = std::thread(server_loop, S);
    S->thr_done = std::thread(completion_loop, S);
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
    S->thr_done.join();
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
    bool wake = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(CBDFS_ECANCELED, "the server is stopping");
        r->id = S->next_id++;
        S->table[r->id] = r;
        // the server thread needs a wake-up only when the queue was empty: otherwise it is
        // staging, or waiting for a slot, which a completion signals
        wake = S->queue.empty();
        S->queue.push_back(r);
        if (!S->any) {
            S->any = true;
            S->t_first = r->t_submit;
        }
    }
    if (wake) S->cv_work.notify_one();
    t->id = r->id;
    return CBDFS_OK;
}

int heur_request_wait(cbdfs_ctx *ctx, cbdfs_ticket t, uint64_t timeout_us) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->table.find(t.id);
        if (it == S->table.end()) return fail(CBDFS_EINVAL, "unknown ticket %llu", (unsigned long long)t.id);
        r = it->second;
    }
    int status;
    {
        std::unique_lock<std::mutex> lk(r->m);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
        while (r->status == 1) {
            if (timeout_us == 0 || r->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
                if (r->status == 1) return fail(CBDFS_ETIMEDOUT, "request %llu not done", (unsigned long long)t.id);
            }
        }
        status = r->status;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->table.erase(t.id)) return fail(CBDFS_EINVAL, "ticket %llu collected twice", (unsigned long long)t.id);
    }
    return status;
}

int cbdfs_server_drive(cbdfs_ctx *ctx, const cbdfs_request *reqs, uint32_t n_reqs, int threads, int depth,
                       double *seconds) {
    if (!ctx || (!reqs && n_reqs) || threads < 1 || depth < 1 || !seconds) return fail(CBDFS_EINVAL, "arguments");
    std::atomic<int> first_error{0};
    // clients take the next request as they free up (an open stream of requests, no tail of
    // idle clients), and the clock starts once every client thread is running
    std::atomic<uint32_t> next{0};
    std::atomic<int> ready{0};
    std::atomic<bool> go{false};
    auto client = [&](int) {
        ready.fetch_add(1);
        while (!go.load(std::memory_order_acquire)) std::this_thread::yield();
        std::deque<cbdfs_ticket> pending;
        auto wait_one = [&]() {
            const int rc = heur_request_wait(ctx, pending.front(), 60000000ull);
            pending.pop_front();
            int zero = 0;
            if (rc) first_error.compare_exchange_strong(zero, rc);
        };
        for (uint32_t j = next.fetch_add(1); j < n_reqs && !first_error.load(); j = next.fetch_add(1)) {
            const cbdfs_request &q = reqs[j];
            cbdfs_ticket tk;
            const int rc = heur_request_submit(ctx, q.heur_id, q.domain, q.states, q.g, q.bound, q.n, q.h_out,
                                               q.mask_out, q.minf_out, &tk);
            if (rc) {
                int zero = 0;
                first_error.compare_exchange_strong(zero, rc);
                break;
            }
            pending.push_back(tk);
            if ((int)pending.size() >= depth) wait_one();
        }
        while (!pending.empty()) wait_one();
    };
    std::vector<std::thread> ts;
    for (int t = 0; t < threads; ++t) ts.emplace_back(client, t);
    while (ready.load() < threads) std::this_thread::yield();
    const auto t0 = std::chrono::steady_clock::now();
    go.store(true, std::memory_order_release);
    for (auto &t : ts) t.join();
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const int rc = first_error.load();
    return rc ? fail(rc, "a driven request failed (status %d)", rc) : CBDFS_OK;
}

int cbdfs_server_prepare(cbdfs_ctx *ctx, int heur_id, int domain) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    Server *S = c->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    if (domain < 0 || domain > 2 || heur_id >= (int)c->heur_kind.size() || heur_id < CBDFS_HEUR_MD ||
        (heur_id == CBDFS_HEUR_MD && domain == CBDFS_DOM_RC3) || heur_is_real(c, heur_id))
        return fail(CBDFS_EINVAL, "heuristic id %d", heur_id);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(CBDFS_EDEVICE, "cudaSetDevice");
    // every bucket's graph on every server slot: a slot is reserved (marked busy) while its
    // graphs are captured, so that no launch uses its stream meanwhile
    std::vector<char> done(S->slots.size(), 0);
    for (size_t left = S->slots.size(); left > 0;) {
        int si = -1;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t k = 0; k < S->slots.size(); ++k)
                if (!done[k] && !S->slot_busy[k]) {
                    si = (int)k;
                    S->slot_busy[k] = 1;
                    break;
                }
        }
        if (si < 0) {
            std::this_thread::sleep_for(std::chrono::microseconds(100));
            continue;
        }
        int rc = CBDFS_OK;
        for (uint32_t b = bucket_of(*S, 32);; b = bucket_of(*S, b * 2)) {
            cudaGraphExec_t ex;
            if ((rc = get_graph(*S, si, heur_id, domain, b, &ex))) break;
            if (b >= cap_rows(*S)) break;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->slot_busy[si] = 0;
        }
        S->cv_work.notify_one();
        if (rc) return rc;
        done[si] = 1;
        --left;
    }
    return CBDFS_OK;
}

int cbdfs_server_reset_stats(cbdfs_ctx *ctx) {
    if (!ctx) return fail(CBDFS_EINVAL, "null argument");
    Server *S = reinterpret_cast<Ctx *>(ctx)->server;
    if (!S) return fail(CBDFS_EINVAL, "no server is running on this context");
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_us.clear();
    S->n_req = S->n_states = S->n_launch = 0;
    S->stage_ns = S->flight_ns = S->finish_ns = S->replay_ns = 0;
    S->any = false;
    return CBDFS_OK;
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
    if (S->n_launch) {
        out->stage_us_per_launch = S->stage_ns / S->n_launch / 1e3;
        out->flight_us_per_launch = S->flight_ns / S->n_launch / 1e3;
        out->finish_us_per_launch = S->finish_ns / S->n_launch / 1e3;
        out->replay_us_per_launch = S->replay_ns / S->n_launch / 1e3;
    }
    return CBDFS_OK;
}

}  // extern "C"
