// search.cpp -- Batch CB-DFS on the host: IDA* (Algorithm 1) and BTS (Batch BTS
// enhancements) over C++ worker threads (Algorithm 2) that round-robin DoIteration
// (Algorithm 3) over work_num subtrees each, with every generated state's heuristic
// evaluated on the GPU in shared batches (section "SingleGPU Batch CB-DFS").
//
// Tree equivalence with a serial CB-DFS (the paper's correctness argument: Batch CB-DFS
// searches the same tree as classic CB-DFS):
//   * GenerateWork builds the full tree to depth d_init once, with h of every node, and no
//     duplicate removal.  Each iteration walks it serially: a node is expanded iff every
//     node on its path (itself included) has f <= bound and none is a goal; frontier nodes
//     at depth d_init that pass become the shared work queue.
//   * Workers expand a node only after the batch that holds its children has returned
//     their bound-test bits; a child is pushed iff its bit is set (f <= bound), a goal child
//     that passes is a solution.  Pruned children reach the next threshold through the
//     batch's least-f-above-bound.
// So every completed iteration expands and generates exactly the nodes a serial CB-DFS
// with the same h would; only the order differs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include <cuda_runtime.h>

#include "common.cuh"
#include "domain.h"

namespace cbdfs {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxKids = 18;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------
// shared batches
// ---------------------------------------------------------------------------------------
struct Batch {
    // page-locked host arrays; h, mask and minf lie in `out` in the slot's layout
    // (slot_out_bytes): the kernels write h and the mask there, minf comes back by one copy
    uint64_t *states = nullptr;
    uint8_t *g = nullptr, *h = nullptr, *out = nullptr;
    uint32_t *mask = nullptr, *minf = nullptr;
    uint8_t *h2 = nullptr;  // fixed-tree mode: the evaluated (not pruning) heuristic
    // the same page-locked buffers as the kernels address them (mapped host memory: the
    // kernels read the states and write h and the mask over the bus, no staging copies)
    const uint64_t *d_states = nullptr;
    const uint8_t *d_g = nullptr;
    uint8_t *d_h = nullptr, *d_h2 = nullptr;
    uint32_t *d_mask = nullptr;
    uint32_t n = 0;                       // states in the batch
    std::atomic<uint32_t> done_gen{0};    // == gen once results are readable
    uint32_t gen = 0;                     // bumped each time the buffer is reopened
    std::atomic<int> consumers{0};        // subtree requests not yet read back
    int state = 0;                        // 0 free, 1 open, 2 in flight, 3 done, 4 full
    int slot = -1;
    cudaEvent_t ev = nullptr;
    Clock::time_point first_add, submitted;
};

struct Shared;

struct Frame {
    State s;
    uint8_t g;
    int8_t move;
    int8_t nk;
    int8_t next;
    uint32_t pass;      // bound-test bits of the children
    State kid[kMaxKids];
    int8_t kmove[kMaxKids];
};

struct Subtree {
    std::vector<Frame> frames;
    int status = 0;           // 0 idle, 1 ready (top frame's bits known), 2 waiting
    Batch *batch = nullptr;
    uint32_t gen = 0, off = 0;
    int work = -1;            // index of the work item (for the path)
};

struct WorkItem {
    State s;
    uint8_t g;
    int8_t move;
    int tree_node;            // node index in the initial tree
};

struct TreeNode {
    State s;
    int parent;
    int8_t move;
    uint8_t g;
    float h;                  // pruning heuristic (an integer unless it is real-valued)
    int first_child, n_child;
};

struct Shared {
    Ctx *c = nullptr;
    const Domain *D = nullptr;
    int heur = 0, prune_heur = 0;  // evaluated / pruning heuristic ids (equal unless fixed-tree)
    uint32_t bound = 0;
    uint32_t cap = 0;
    uint64_t timeout_us = 0;
    int complete = 1;
    int64_t limit = -1;       // expansion limit of this search (-1 none)
    // work
    std::vector<WorkItem> *work = nullptr;
    std::atomic<int64_t> next_work{0};
    // batches
    std::vector<Batch *> batches;
    std::mutex open_mu;
    int open = -1;            // index of the open batch
    std::vector<int> slots;   // ctx slots owned by this solve
    std::vector<int> slot_free;
    // results
    std::atomic<int64_t> expanded{0}, generated{0}, evaluated{0}, nbatches{0};
    int64_t hist[CBDFS_BATCH_HIST] = {};  // batches by size class (processor thread only)
    int64_t fill_ns = 0, flight_ns = 0, submit_ns = 0;  // batch timing sums (processor thread)
    int64_t busy_ns = 0;                  // time with at least one batch in flight (processor thread)
    Clock::time_point busy_from;
    std::atomic<uint32_t> minf{kNone};
    std::atomic<int> found{0}, stop{0}, cut{0};
    std::mutex sol_mu;
    int best_cost = -1;
    std::vector<int> best_path;
    std::atomic<int> live_workers{0}, idle_workers{0};
    std::atomic<int> error{0};
    std::string error_msg;
    Clock::time_point deadline;
    bool has_deadline = false;
    std::atomic<int64_t> total_expanded_before{0};
    uint64_t node_limit = 0;
};

void atomic_min(std::atomic<uint32_t> &a, uint32_t v) {
    uint32_t cur = a.load(std::memory_order_relaxed);
    while (v < cur && !a.compare_exchange_weak(cur, v)) {
    }
}

// Open a free batch (caller holds open_mu).  Returns false if none is free.
bool open_batch(Shared &S) {
    for (size_t i = 0; i < S.batches.size(); ++i) {
        Batch &b = *S.batches[i];
        if (b.state == 0) {
            b.state = 1;
            b.n = 0;
            b.gen++;
            b.consumers.store(0);
            S.open = (int)i;
            return true;
        }
    }
    S.open = -1;
    return false;
}

// ---------------------------------------------------------------------------------------
// batch processor: seals the open batch when it is full, when its oldest state waited
// timeout_us, or when every live worker is idle; evaluates sealed batches on the GPU
// slots asynchronously; publishes results.
// ---------------------------------------------------------------------------------------
// the histogram class of a batch of n states: 2^i <= n < 2^(i+1), the last class open-ended
int batch_class(uint32_t n) {
    int cls = 0;
    while (cls + 1 < CBDFS_BATCH_HIST && (n >> (cls + 1)) != 0) ++cls;
    return cls;
}

int submit(Shared &S, Batch &b) {
    const auto t_in = Clock::now();
    S.fill_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(t_in - b.first_add).count();
    Ctx *c = S.c;
    const int si = S.slot_free.back();
    S.slot_free.pop_back();
    b.slot = si;
    Slot &sl = c->slots[si];
    cudaStream_t st = sl.stream;
    const uint32_t n = b.n;
    int rc = CBDFS_OK;
    if (S.prune_heur != S.heur) {
        // fixed-tree mode: evaluate the network on every state, prune with the other one
        rc = run_eval(c, sl, S.heur, S.D->dom, b.d_states, b.d_g, S.bound, n, b.d_h2, sl.d_mask,
                      sl.d_minf, nullptr, st);
        if (rc) return rc;
    }
    rc = run_eval(c, sl, S.prune_heur, S.D->dom, b.d_states, b.d_g, S.bound, n, b.d_h, b.d_mask,
                  sl.d_minf, nullptr, st);
    if (rc) return rc;
    // h and the mask are already in the batch's host buffers; the least f above the bound is
    // the one word read back
    if (cudaMemcpyAsync(b.minf, sl.d_minf, 4, cudaMemcpyDeviceToHost, st) || cudaEventRecord(b.ev, st))
        return fail(CBDFS_EDEVICE, "result download");
    b.state = 2;
    S.nbatches++;
    S.hist[batch_class(n)]++;
    S.evaluated += n;
    b.submitted = Clock::now();
    S.submit_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(b.submitted - t_in).count();
    return CBDFS_OK;
}

void processor(Shared &S) {
    cudaSetDevice(S.c->device);
    std::vector<int> inflight;
    while (true) {
        bool progress = false;
        {
            std::lock_guard<std::mutex> lk(S.open_mu);
            // completions
            for (size_t i = 0; i < inflight.size();) {
                Batch &b = *S.batches[inflight[i]];
                cudaError_t q = cudaEventQuery(b.ev);
                if (q == cudaSuccess) {
                    S.flight_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - b.submitted).count();
                    if (b.n) atomic_min(S.minf, *b.minf);
                    b.state = 3;
                    S.slot_free.push_back(b.slot);
                    b.done_gen.store(b.gen, std::memory_order_release);
                    inflight[i] = inflight.back();
                    inflight.pop_back();
                    if (inflight.empty())
                        S.busy_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - S.busy_from).count();
                    progress = true;
                    continue;
                }
                if (q != cudaErrorNotReady && !S.error.load()) {
                    S.error_msg = std::string("batch evaluation: ") + cudaGetErrorString(q);
                    S.error = CBDFS_EDEVICE;
                    S.stop = 1;
                }
                ++i;
            }
            // recycle consumed batches
            for (auto *b : S.batches)
                if (b->state == 3 && b->consumers.load(std::memory_order_acquire) == 0) b->state = 0;
            // seal: batches marked full first, then the open one when it is full, old, or
            // every live worker is waiting
            while (!S.slot_free.empty() && !S.error.load()) {
                int pick = -1;
                for (size_t i = 0; i < S.batches.size(); ++i)
                    if (S.batches[i]->state == 4) { pick = (int)i; break; }
                if (pick < 0 && S.open >= 0) {
                    Batch &b = *S.batches[S.open];
                    const int live = S.live_workers.load(), idle = S.idle_workers.load();
                    bool seal = b.n >= S.cap;
                    if (!seal && b.n > 0) {
                        const auto age = std::chrono::duration_cast<std::chrono::microseconds>(
                                             Clock::now() - b.first_add).count();
                        seal = (uint64_t)age >= S.timeout_us || (live > 0 && idle >= live);
                    }
                    if (seal) {
                        pick = S.open;
                        S.open = -1;
                    }
                }
                if (pick < 0) break;
                int rc = submit(S, *S.batches[pick]);
                if (rc) {
                    S.error_msg = cbdfs_last_error();
                    S.error = rc;
                    S.stop = 1;
                    break;
                }
                if (inflight.empty()) S.busy_from = Clock::now();
                inflight.push_back(pick);
                progress = true;
            }
            if (S.open < 0) open_batch(S);
        }
        if (S.live_workers.load() == 0 && inflight.empty()) break;
        if (!progress) std::this_thread::yield();
    }
}

// ---------------------------------------------------------------------------------------
// workers
// ---------------------------------------------------------------------------------------
struct Worker {
    Shared *S;
    std::vector<Subtree> sub;
    // staging: children waiting to be copied into the open batch
    std::vector<uint64_t> st_states;
    std::vector<uint8_t> st_g;
    std::vector<std::pair<int, int>> st_req;  // (subtree, count)
    int64_t exp_local = 0, gen_local = 0, exp_unreported = 0;

    void stage(int si, Frame &f) {
        const int w = S->D->words;
        for (int i = 0; i < f.nk; ++i) {
            st_states.push_back(f.kid[i].w[0]);
            if (w == 2) st_states.push_back(f.kid[i].w[1]);
            st_g.push_back((uint8_t)(f.g + 1));
        }
        st_req.emplace_back(si, f.nk);
        sub[si].status = 2;
        sub[si].batch = nullptr;
    }

    // Copy staged children into open batches.  A request that does not fit marks the open
    // batch full (the processor submits it at once) and moves on to a fresh one.  Returns
    // true if everything staged was placed.
    bool flush() {
        if (st_req.empty()) return true;
        const int w = S->D->words;
        size_t pos = 0;  // staged states placed
        size_t r = 0;
        {
            std::lock_guard<std::mutex> lk(S->open_mu);
            while (r < st_req.size()) {
                if (S->open < 0 && !open_batch(*S)) break;
                Batch &b = *S->batches[S->open];
                const int cnt = st_req[r].second;
                if (b.n + cnt > S->cap) {
                    b.state = 4;  // full: the processor seals it
                    S->open = -1;
                    continue;
                }
                if (b.n == 0) b.first_add = Clock::now();
                memcpy(b.states + (size_t)b.n * w, st_states.data() + pos * w, sizeof(uint64_t) * cnt * w);
                memcpy(b.g + b.n, st_g.data() + pos, cnt);
                Subtree &t = sub[st_req[r].first];
                t.batch = &b;
                t.gen = b.gen;
                t.off = b.n;
                b.n += cnt;
                b.consumers.fetch_add(1, std::memory_order_relaxed);
                pos += cnt;
                ++r;
            }
        }
        if (r == 0) return false;
        st_states.erase(st_states.begin(), st_states.begin() + pos * w);
        st_g.erase(st_g.begin(), st_g.begin() + pos);
        st_req.erase(st_req.begin(), st_req.begin() + r);
        return true;
    }

    bool expand(int si, const State &s, uint8_t g, int8_t move) {
        Subtree &t = sub[si];
        t.frames.emplace_back();
        Frame &f = t.frames.back();
        f.s = s;
        f.g = g;
        f.move = move;
        f.next = 0;
        f.pass = 0;
        f.nk = (int8_t)S->D->children(s, move, f.kid, f.kmove);
        ++exp_local;
        ++exp_unreported;
        gen_local += f.nk;
        stage(si, f);
        if (exp_unreported >= 64) {
            const int64_t tot = S->expanded.fetch_add(exp_unreported) + exp_unreported;
            exp_unreported = 0;
            if (S->limit >= 0 && tot > S->limit) {  // more expansions than the limit: cut
                S->cut = 1;
                S->stop = 1;
            }
            if (S->node_limit && (uint64_t)(tot + S->total_expanded_before.load()) >= S->node_limit) S->stop = 1;
        }
        return true;
    }

    void solution(int si, const Frame &top, int kid) {
        const int cost = top.g + 1;
        std::lock_guard<std::mutex> lk(S->sol_mu);
        if (S->best_cost < 0 || cost < S->best_cost) {
            S->best_cost = cost;
            S->best_path.clear();
            // initial-tree part is prepended by the caller (work index -> tree path)
            S->best_path.push_back(-1 - sub[si].work);
            for (size_t i = 1; i < sub[si].frames.size(); ++i) S->best_path.push_back(sub[si].frames[i].move);
            S->best_path.push_back(top.kmove[kid]);
        }
        S->found = 1;
        if (!S->complete) S->stop = 1;
    }

    // DoIteration for subtree si: returns true if it made progress
    bool step(int si) {
        Subtree &t = sub[si];
        if (t.status == 2) {
            if (!t.batch) return false;  // still staged
            if (t.batch->done_gen.load(std::memory_order_acquire) != t.gen) return false;
            Frame &top = t.frames.back();
            const uint32_t *mask = t.batch->mask;
            uint32_t bits = 0;
            for (int i = 0; i < top.nk; ++i) {
                const uint32_t j = t.off + i;
                bits |= ((mask[j >> 5] >> (j & 31)) & 1u) << i;
            }
            top.pass = bits;
            top.next = 0;
            t.batch->consumers.fetch_sub(1, std::memory_order_release);
            t.batch = nullptr;
            t.status = 1;
        }
        if (t.status != 1) return false;
        while (!t.frames.empty()) {
            Frame &top = t.frames.back();
            int i = top.next;
            while (i < top.nk && !((top.pass >> i) & 1u)) ++i;
            if (i >= top.nk) {
                t.frames.pop_back();
                continue;
            }
            top.next = (int8_t)(i + 1);
            const State &kid = top.kid[i];
            if (S->D->is_goal(kid)) {
                solution(si, top, i);
                if (S->stop.load(std::memory_order_relaxed)) return true;
                continue;
            }
            expand(si, kid, (uint8_t)(top.g + 1), top.kmove[i]);
            return true;
        }
        t.status = 0;
        return true;
    }

    bool take_work(int si) {
        const int64_t k = S->next_work.fetch_add(1);
        if (k >= (int64_t)S->work->size()) return false;
        const WorkItem &wi = (*S->work)[k];
        sub[si].work = (int)k;
        sub[si].frames.clear();
        expand(si, wi.s, wi.g, wi.move);
        return true;
    }

    void run(int work_num) {
        cudaSetDevice(S->c->device);
        sub.resize(work_num);
        for (auto &t : sub) t.frames.reserve(64);
        int terminated = 0;
        std::vector<char> term(work_num, 0);
        for (int i = 0; i < work_num; ++i)
            if (!take_work(i)) { term[i] = 1; ++terminated; }
        bool idle_marked = false;
        while (terminated < work_num && !S->stop.load(std::memory_order_relaxed)) {
            bool progress = false;
            for (int i = 0; i < work_num; ++i) {
                if (term[i]) continue;
                if (sub[i].status == 0) {
                    if (take_work(i)) progress = true;
                    else { term[i] = 1; ++terminated; continue; }
                }
                if (step(i)) progress = true;
                if (sub[i].status == 0) {
                    if (take_work(i)) progress = true;
                    else if (!term[i]) { term[i] = 1; ++terminated; }
                }
            }
            if (!st_req.empty()) {
                if (flush()) progress = true;
            }
            if (!progress) {
                if (!idle_marked) { S->idle_workers++; idle_marked = true; }
                std::this_thread::yield();
                if (S->has_deadline && Clock::now() > S->deadline) S->stop = 1;
                if (S->c->cancel.load()) S->stop = 1;
            } else if (idle_marked) {
                S->idle_workers--;
                idle_marked = false;
            }
        }
        if (idle_marked) S->idle_workers--;
        // release batch references this worker still holds (a stopped search)
        for (auto &t : sub)
            if (t.status == 2 && t.batch) {
                while (t.batch->done_gen.load(std::memory_order_acquire) != t.gen && !S->error.load())
                    std::this_thread::yield();
                t.batch->consumers.fetch_sub(1);
                t.batch = nullptr;
            }
        const int64_t tot = S->expanded.fetch_add(exp_unreported) + exp_unreported;
        if (S->limit >= 0 && tot > S->limit) S->cut = 1;
        S->generated += gen_local;
        S->live_workers--;
    }
};

// ---------------------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------------------
// f-costs as the kernels' keys: an integer f, or an FP32 f's bit pattern for a real-valued
// heuristic (f >= 0, so keys order like the values)
inline uint32_t f_key(bool real, uint32_t g, float h) {
    if (!real) return g + (uint32_t)h;
    const float f = (float)g + h;
    uint32_t k;
    memcpy(&k, &f, 4);
    return k;
}
inline float key_value(uint32_t k) {
    float f;
    memcpy(&f, &k, 4);
    return f;
}

struct Solver {
    Ctx *c;
    Domain D;
    int heur, prune;
    bool real = false;             // the pruning heuristic is real-valued (FP32 f-costs)
    float *d_hreal = nullptr;      // device: real h of a batch of initial-tree states
    cbdfs_search_cfg cfg;
    std::vector<TreeNode> tree;
    std::vector<int> level_start;  // tree nodes of depth d: [level_start[d], level_start[d+1])
    int d_init = 0;
    std::vector<int> slots;
    std::vector<std::unique_ptr<Batch>> batches;
    int64_t evaluated = 0, nbatches = 0, search_batches = 0;
    int64_t hist[CBDFS_BATCH_HIST] = {};
    int64_t fill_ns = 0, flight_ns = 0, submit_ns = 0, busy_ns = 0;
    double seconds = 0;
    int64_t expanded_total = 0;

    Solver(Ctx *c_, int dom) : c(c_), D(dom) {}

    // evaluate h (pruning heuristic) for a list of states synchronously on slot slots[0]
    int eval_states(const std::vector<State> &st, std::vector<float> &h) {
        Slot &sl = c->slots[slots[0]];
        const int w = D.words;
        h.resize(st.size());
        std::vector<uint8_t> h8(st.size());
        if (real && !d_hreal) {
            int rc = dev_alloc(c, (void **)&d_hreal, sizeof(float) * c->max_batch_pad);
            if (rc) return rc;
        }
        std::vector<uint64_t> buf;
        std::vector<uint8_t> g;
        std::vector<uint32_t> mask;
        uint32_t minf;
        for (size_t o = 0; o < st.size(); o += c->max_batch) {
            const uint32_t n = (uint32_t)std::min<size_t>(c->max_batch, st.size() - o);
            buf.resize((size_t)n * w);
            g.assign(n, 0);
            mask.resize((n + 31) / 32);
            for (uint32_t i = 0; i < n; ++i) {
                buf[(size_t)i * w] = st[o + i].w[0];
                if (w == 2) buf[(size_t)i * w + 1] = st[o + i].w[1];
            }
            cudaStream_t s = sl.stream;
            CUDA_TRY(cudaMemcpyAsync(sl.d_states, buf.data(), (size_t)n * 8 * w, cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(sl.d_g, g.data(), n, cudaMemcpyHostToDevice, s));
            if (prune != heur) {  // the evaluated network runs on every node in fixed-tree mode
                int rc = run_eval(c, sl, heur, D.dom, sl.d_states, sl.d_g, 255, n, sl.d_h, sl.d_mask, sl.d_minf, nullptr, s);
                if (rc) return rc;
            }
            int rc = run_eval(c, sl, prune, D.dom, sl.d_states, sl.d_g, 255, n, sl.d_h, sl.d_mask, sl.d_minf,
                              real ? d_hreal : nullptr, s);
            if (rc) return rc;
            if (real) CUDA_TRY(cudaMemcpyAsync(h.data() + o, d_hreal, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
            else CUDA_TRY(cudaMemcpyAsync(h8.data() + o, sl.d_h, n, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaMemcpyAsync(&minf, sl.d_minf, 4, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            evaluated += n;
            nbatches++;
            hist[batch_class(n)]++;
        }
        if (!real)
            for (size_t i = 0; i < st.size(); ++i) h[i] = (float)h8[i];
        return CBDFS_OK;
    }

    int generate_work(const State &root) {
        // automatic depth: the shallowest with at least 16 * threads * work_num leaves, capped
        // so the tree stays below 4M nodes.  Only the leaves within the bound become work, and in
        // the early iterations few do: a frontier 16x the workers' subtrees keeps more of them
        // busy (15-puzzle, 16 threads, workNum 256: depth 14-15 instead of 12-13, 25 % more
        // expanded nodes/s; deeper, the serial walk of the tree costs more than it gives)
        const int64_t want = cfg.d_init >= 0 ? -1 : (int64_t)16 * cfg.threads * cfg.work_num;
        tree.clear();
        level_start.clear();
        TreeNode r{};
        r.s = root;
        r.parent = -1;
        r.move = -1;
        r.g = 0;
        tree.push_back(r);
        level_start.push_back(0);
        level_start.push_back(1);
        int depth = 0;
        while (true) {
            const int64_t leaves = level_start[depth + 1] - level_start[depth];
            if (cfg.d_init >= 0 ? depth >= cfg.d_init : leaves >= want) break;
            if ((int64_t)tree.size() * (D.words == 2 ? 14 : 3) > 4000000) break;
            if (depth >= 60) break;
            for (int i = level_start[depth]; i < level_start[depth + 1]; ++i) {
                State kids[kMaxKids];
                int8_t mv[kMaxKids];
                const int nk = D.children(tree[i].s, tree[i].move, kids, mv);
                tree[i].first_child = (int)tree.size();
                tree[i].n_child = nk;
                for (int k = 0; k < nk; ++k) {
                    TreeNode t{};
                    t.s = kids[k];
                    t.parent = i;
                    t.move = mv[k];
                    t.g = (uint8_t)(tree[i].g + 1);
                    tree.push_back(t);
                }
            }
            level_start.push_back((int)tree.size());
            ++depth;
        }
        d_init = depth;
        for (int i = level_start[depth]; i < (int)tree.size(); ++i) tree[i].n_child = 0;
        std::vector<State> st(tree.size());
        for (size_t i = 0; i < tree.size(); ++i) st[i] = tree[i].s;
        std::vector<float> h;
        int rc = eval_states(st, h);
        if (rc) return rc;
        for (size_t i = 0; i < tree.size(); ++i) tree[i].h = D.is_goal(tree[i].s) ? 0.f : h[i];
        return CBDFS_OK;
    }

    std::vector<int> tree_path(int node) const {
        std::vector<int> p;
        while (node > 0) {
            p.push_back(tree[node].move);
            node = tree[node].parent;
        }
        return std::vector<int>(p.rbegin(), p.rend());
    }

    struct IterOut {
        int64_t expanded = 0, generated = 0;
        uint32_t minf = kNone;
        int found = 0, cost = -1, cut = 0;
        std::vector<int> path;
    };

    // One CB-DFS with threshold `bound` and expansion limit (-1 none).
    int cbdfs(uint32_t bound, int64_t limit, IterOut &o) {
        // serial walk of the initial tree
        std::vector<char> exp(tree.size(), 0);
        std::vector<WorkItem> work;
        int64_t ex = 0, gn = 0;
        uint32_t minf = kNone;
        int best = -1;
        int best_node = -1;
        bool stop = false;
        for (int d = 0; d <= d_init && !stop; ++d) {
            for (int i = level_start[d]; i < level_start[d + 1]; ++i) {
                const TreeNode &t = tree[i];
                if (t.parent >= 0 && !exp[t.parent]) continue;
                const uint32_t f = f_key(real, t.g, t.h);
                if (f > bound) {
                    minf = std::min(minf, f);
                    continue;
                }
                if (D.is_goal(t.s)) {
                    if (best < 0 || t.g < best) { best = t.g; best_node = i; }
                    if (!cfg.complete_final) { stop = true; break; }
                    continue;
                }
                if (d == d_init) {
                    work.push_back(WorkItem{t.s, t.g, t.move, i});
                    continue;
                }
                if (limit >= 0 && ex >= limit) { o.cut = 1; stop = true; break; }
                exp[i] = 1;
                ++ex;
                gn += t.n_child;
            }
        }
        o.expanded = ex;
        o.generated = gn;
        o.minf = minf;
        if (best >= 0) {
            o.found = 1;
            o.cost = best;
            o.path = tree_path(best_node);
        }
        if (stop || work.empty()) return CBDFS_OK;

        Shared S;
        S.c = c;
        S.D = &D;
        S.heur = heur;
        S.prune_heur = prune;
        S.bound = bound;
        S.cap = cfg.batch;
        S.timeout_us = cfg.timeout_us;
        S.complete = cfg.complete_final;
        S.limit = limit >= 0 ? std::max<int64_t>(0, limit - ex) : -1;
        S.work = &work;
        S.node_limit = cfg.node_limit;
        S.total_expanded_before = expanded_total + ex;
        if (cfg.time_limit_s > 0) {
            S.has_deadline = true;
            S.deadline = deadline;
        }
        if (S.limit == 0) {
            o.cut = 1;
            return CBDFS_OK;
        }
        for (auto &b : batches) {
            b->state = 0;
            b->n = 0;
            b->consumers.store(0);
            S.batches.push_back(b.get());
        }
        S.slots = slots;
        S.slot_free = slots;
        S.open = -1;
        S.live_workers = cfg.threads;
        std::thread proc(processor, std::ref(S));
        std::vector<std::thread> ws;
        std::vector<std::unique_ptr<Worker>> wk(cfg.threads);
        for (int t = 0; t < cfg.threads; ++t) {
            wk[t] = std::make_unique<Worker>();
            wk[t]->S = &S;
            ws.emplace_back([&, t] { wk[t]->run(cfg.work_num); });
        }
        for (auto &t : ws) t.join();
        proc.join();
        evaluated += S.evaluated.load();
        nbatches += S.nbatches.load();
        search_batches += S.nbatches.load();
        for (int i = 0; i < CBDFS_BATCH_HIST; ++i) hist[i] += S.hist[i];
        fill_ns += S.fill_ns;
        flight_ns += S.flight_ns;
        submit_ns += S.submit_ns;
        busy_ns += S.busy_ns;
        if (S.error.load()) return fail(S.error.load(), "%s", S.error_msg.c_str());
        o.expanded += S.expanded.load();
        o.generated += S.generated.load();
        o.minf = std::min(o.minf, S.minf.load());
        o.cut |= S.cut.load();
        if (S.found.load() && (!o.found || S.best_cost < o.cost)) {
            o.found = 1;
            o.cost = S.best_cost;
            const int work_idx = -1 - S.best_path[0];
            o.path = tree_path(work[work_idx].tree_node);
            o.path.insert(o.path.end(), S.best_path.begin() + 1, S.best_path.end());
        }
        if (c->cancel.load()) return fail(CBDFS_ECANCELED, "canceled");
        // stopped by the deadline or the node limit (not by the expansion limit, nor by a goal
        // in first-goal mode): an iteration cut short reports an error even after a goal,
        // since a later part of it may hold a cheaper one
        if (S.stop.load() && !S.cut.load() && !(S.found.load() && !S.complete)) {
            if (S.has_deadline && Clock::now() > S.deadline) return fail(CBDFS_ETIMEDOUT, "time limit reached");
            if (cfg.node_limit) return fail(CBDFS_ECANCELED, "node limit reached");
        }
        return CBDFS_OK;
    }

    Clock::time_point deadline;

    // ---- drivers ----
    void record(cbdfs_result *out, uint32_t bound, int64_t limit, const IterOut &o) {
        const int i = out->n_iters;
        if (i < CBDFS_MAX_ITERS) {
            out->iter_bound[i] = real ? 0 : bound;
            out->iter_bound_real[i] = real ? (double)key_value(bound) : (double)bound;
            out->iter_expanded[i] = o.expanded;
            out->iter_generated[i] = o.generated;
            out->iter_limit[i] = limit;
            out->iter_cut[i] = o.cut;
        }
        out->n_iters++;
        out->expanded += o.expanded;
        out->generated += o.generated;
        expanded_total += o.expanded;
    }

    int finish(cbdfs_result *out, const IterOut &o) {
        out->cost = o.cost;
        out->path_len = (int)std::min<size_t>(o.path.size(), 256);
        for (int i = 0; i < out->path_len; ++i) out->path[i] = o.path[i];
        return CBDFS_OK;
    }

    // Algorithm 1: bound = h(root); CB-DFS; UpdateThreshold = least f above the bound.
    int ida(cbdfs_result *out) {
        uint32_t bound = f_key(real, 0, tree[0].h);
        for (;;) {
            IterOut o;
            int rc = cbdfs(bound, -1, o);
            record(out, bound, -1, o);
            if (rc) return rc;
            if (o.found) return finish(out, o);
            if (o.minf == kNone) return fail(CBDFS_ENOTFOUND, "no solution: the tree is exhausted");
            bound = o.minf;
        }
    }

    // BTS: the same schedule as the oracle's reading of Batch BTS (growth base N starts at
    // n0 = 10,000, the first bound is h(root)+1; accept a bound whose search expands
    // between c1*N and c2*N nodes, found by an exponential then binary search over bounds;
    // every search runs to completion of its iteration so a goal found by an uncut search
    // carries the least goal cost of that tree).
    int bts(cbdfs_result *out) {
        const int64_t c1 = cfg.bts_c1 > 0 ? cfg.bts_c1 : 2, c2 = cfg.bts_c2 > 0 ? cfg.bts_c2 : 8;
        int64_t N = cfg.bts_n0 ? (int64_t)cfg.bts_n0 : 10000;
        int64_t nxt = (int64_t)tree[0].h + 1;  // an integer h
        IterOut done;
        int code = 0;  // 1 found, 2 exhausted
        auto run = [&](int64_t b, int64_t limit, IterOut &o) -> int {
            o = IterOut();
            int rc = cbdfs((uint32_t)b, limit, o);
            record(out, (uint32_t)b, limit, o);
            if (rc) return rc;
            if (!o.cut && o.found) { done = o; code = 1; }
            else if (!o.cut && o.minf == kNone) code = 2;
            return CBDFS_OK;
        };
        for (;;) {
            const int64_t limit = c2 * N;
            IterOut r;
            int rc = run(nxt, limit, r);
            if (rc) return rc;
            if (code) break;
            if (r.cut) {
                if ((rc = run(nxt, -1, r))) return rc;
                if (code) break;
                N = std::max<int64_t>(r.expanded, 1);
                nxt = r.minf;
                continue;
            }
            if (r.expanded >= c1 * N) {
                N = r.expanded;
                nxt = r.minf;
                continue;
            }
            int64_t lo = nxt, hi = 0;
            IterOut hi_r;
            for (int j = 0;; ++j) {
                const int64_t b = nxt + ((int64_t)1 << j);
                IterOut rr;
                if ((rc = run(b, limit, rr))) return rc;
                if (code) break;
                if (rr.cut || rr.expanded >= c1 * N) { hi = b; hi_r = rr; break; }
                lo = b;
            }
            if (code) break;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) / 2;
                IterOut rr;
                if ((rc = run(mid, limit, rr))) return rc;
                if (code) break;
                if (rr.cut || rr.expanded >= c1 * N) { hi = mid; hi_r = rr; }
                else lo = mid;
            }
            if (code) break;
            if (hi_r.cut) {
                if ((rc = run(hi, -1, hi_r))) return rc;
                if (code) break;
            }
            N = std::max<int64_t>(hi_r.expanded, 1);
            nxt = hi_r.minf;
        }
        if (code == 2) return fail(CBDFS_ENOTFOUND, "no solution: the tree is exhausted");
        return finish(out, done);
    }

    // BTS over real bounds (a real-valued heuristic): the schedule of bts() in FP32, except
    // that the binary search between the last small bound lo and the first big one hi runs
    // while some f-cost lies strictly between them (lo's least f above its bound is below
    // hi) and probes max((lo+hi)/2, that f), so that every probe can change the tree.  With
    // integer f-costs it accepts the bounds bts() accepts (the least big bound).
    int bts_real(cbdfs_result *out) {
        const int64_t c1 = cfg.bts_c1 > 0 ? cfg.bts_c1 : 2, c2 = cfg.bts_c2 > 0 ? cfg.bts_c2 : 8;
        int64_t N = cfg.bts_n0 ? (int64_t)cfg.bts_n0 : 10000;
        float nxt = tree[0].h + 1.0f;
        IterOut done;
        int code = 0;  // 1 found, 2 exhausted
        auto run = [&](float b, int64_t limit, IterOut &o) -> int {
            o = IterOut();
            const uint32_t key = f_key(true, 0, b);
            int rc = cbdfs(key, limit, o);
            record(out, key, limit, o);
            if (rc) return rc;
            if (!o.cut && o.found) { done = o; code = 1; }
            else if (!o.cut && o.minf == kNone) code = 2;
            return CBDFS_OK;
        };
        auto big = [&](const IterOut &o) { return o.cut || o.expanded >= c1 * N; };
        for (;;) {
            const int64_t limit = c2 * N;
            IterOut r;
            int rc = run(nxt, limit, r);
            if (rc) return rc;
            if (code) break;
            if (r.cut) {
                if ((rc = run(nxt, -1, r))) return rc;
                if (code) break;
                N = std::max<int64_t>(r.expanded, 1);
                nxt = key_value(r.minf);
                continue;
            }
            if (r.expanded >= c1 * N) {
                N = r.expanded;
                nxt = key_value(r.minf);
                continue;
            }
            float lo = nxt, lo_minf = key_value(r.minf), hi = 0.f;
            IterOut hi_r;
            bool have_hi = false;
            for (int j = 0; j < 120 && !have_hi; ++j) {
                const float b = nxt + std::ldexp(1.0f, j);
                IterOut rr;
                if ((rc = run(b, limit, rr))) return rc;
                if (code) break;
                if (big(rr)) { hi = b; hi_r = rr; have_hi = true; }
                else { lo = b; lo_minf = key_value(rr.minf); }
            }
            if (code) break;
            if (!have_hi) return fail(CBDFS_ENOTFOUND, "BTS: no bound below 2^120 reaches the node count");
            while (lo_minf < hi) {
                float mid = std::max((lo + hi) / 2.0f, lo_minf);
                if (mid >= hi) mid = lo_minf;
                IterOut rr;
                if ((rc = run(mid, limit, rr))) return rc;
                if (code) break;
                if (big(rr)) { hi = mid; hi_r = rr; }
                else { lo = mid; lo_minf = key_value(rr.minf); }
            }
            if (code) break;
            if (hi_r.cut) {
                if ((rc = run(hi, -1, hi_r))) return rc;
                if (code) break;
            }
            N = std::max<int64_t>(hi_r.expanded, 1);
            nxt = key_value(hi_r.minf);
        }
        if (code == 2) return fail(CBDFS_ENOTFOUND, "no solution: the tree is exhausted");
        return finish(out, done);
    }
};

}  // namespace

}  // namespace cbdfs

using namespace cbdfs;

extern "C" {

int cbdfs_solve(cbdfs_ctx *ctx, int domain, const uint64_t *start, int algo, int heur_id,
                const cbdfs_search_cfg *cfg_in, cbdfs_result *out) {
    if (!ctx || !start || !out) return fail(CBDFS_EINVAL, "null argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (domain < 0 || domain > 2) return fail(CBDFS_EINVAL, "domain %d", domain);
    if (algo != CBDFS_ALGO_IDA && algo != CBDFS_ALGO_BTS) return fail(CBDFS_EINVAL, "algorithm %d", algo);
    cbdfs_search_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else cbdfs_search_defaults(&cfg);
    if (cfg.threads < 1 || cfg.threads > 1024 || cfg.work_num < 1 || cfg.work_num > 1 << 16)
        return fail(CBDFS_EINVAL, "threads %d / work_num %d out of range", cfg.threads, cfg.work_num);
    if (cfg.batch < kMaxKids || cfg.batch > c->max_batch)
        return fail(CBDFS_EINVAL, "batch %u outside %d..max_batch=%u", cfg.batch, kMaxKids, c->max_batch);
    auto bad_heur = [&](int h) {
        return h >= (int)c->heur_kind.size() || h < CBDFS_HEUR_MD ||
               (h == CBDFS_HEUR_MD && domain == CBDFS_DOM_RC3);
    };
    if (bad_heur(heur_id)) return fail(CBDFS_EINVAL, "heuristic id %d", heur_id);
    if (cfg.fixed_tree_heur != CBDFS_HEUR_NONE && bad_heur(cfg.fixed_tree_heur))
        return fail(CBDFS_EINVAL, "fixed-tree heuristic id %d", cfg.fixed_tree_heur);
    memset(out, 0, sizeof(*out));
    out->cost = -1;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(CBDFS_EDEVICE, "cudaSetDevice");
    c->cancel = 0;
    const auto t0 = Clock::now();

    Solver sv(c, domain);
    sv.cfg = cfg;
    sv.heur = heur_id;
    sv.prune = cfg.fixed_tree_heur != CBDFS_HEUR_NONE ? cfg.fixed_tree_heur : heur_id;
    sv.real = heur_is_real(c, sv.prune);
    if (cfg.time_limit_s > 0)
        sv.deadline = t0 + std::chrono::microseconds((int64_t)(cfg.time_limit_s * 1e6));
    // take every free host slot (at least one; waits for one if all are busy)
    {
        std::unique_lock<std::mutex> lk(c->slot_mu);
        for (;;) {
            for (int i = 1; i < (int)c->slots.size(); ++i)
                if (!c->slots[i].busy) {
                    c->slots[i].busy = true;
                    sv.slots.push_back(i);
                }
            if (!sv.slots.empty()) break;
            c->slot_cv.wait(lk);
        }
    }
    int rc = CBDFS_OK;
    const int w = sv.D.words;
    for (size_t i = 0; i < 2 * sv.slots.size() && !rc; ++i) {
        auto b = std::make_unique<Batch>();
        const size_t cap = cfg.batch;
        const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
        if (cudaHostAlloc(&b->states, cap * 8 * w, fl) || cudaHostAlloc(&b->g, cap, fl) ||
            cudaHostAlloc(&b->out, slot_out_bytes(c), fl) || cudaHostAlloc(&b->h2, cap, fl) ||
            cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming))
            rc = fail(CBDFS_ENOMEM, "pinned batch buffers");
        if (!rc) {
            b->h = b->out;
            b->mask = reinterpret_cast<uint32_t *>(b->out + c->max_batch_pad);
            b->minf = b->mask + c->max_batch_pad / 32;
            void *ds = nullptr, *dg = nullptr, *dout = nullptr, *dh2 = nullptr;
            if (cudaHostGetDevicePointer(&ds, b->states, 0) || cudaHostGetDevicePointer(&dg, b->g, 0) ||
                cudaHostGetDevicePointer(&dout, b->out, 0) || cudaHostGetDevicePointer(&dh2, b->h2, 0))
                rc = fail(CBDFS_EDEVICE, "mapped batch buffers");
            b->d_states = static_cast<const uint64_t *>(ds);
            b->d_g = static_cast<const uint8_t *>(dg);
            b->d_h = static_cast<uint8_t *>(dout);
            b->d_mask = reinterpret_cast<uint32_t *>(b->d_h + c->max_batch_pad);
            b->d_h2 = static_cast<uint8_t *>(dh2);
        }
        sv.batches.push_back(std::move(b));
    }
    if (!rc) rc = sv.generate_work(sv.D.make(start));
    if (!rc) rc = algo == CBDFS_ALGO_IDA ? sv.ida(out) : sv.real ? sv.bts_real(out) : sv.bts(out);
    if (sv.d_hreal) dev_free(c, sv.d_hreal, sizeof(float) * c->max_batch_pad);
    for (auto &b : sv.batches) {
        cudaFreeHost(b->states);
        cudaFreeHost(b->g);
        cudaFreeHost(b->out);
        cudaFreeHost(b->h2);
        if (b->ev) cudaEventDestroy(b->ev);
    }
    {
        std::lock_guard<std::mutex> lk(c->slot_mu);
        for (int i : sv.slots) c->slots[i].busy = false;
    }
    c->slot_cv.notify_all();
    out->real_valued = sv.real;
    out->batches = sv.nbatches;
    for (int i = 0; i < CBDFS_BATCH_HIST; ++i) out->batch_hist[i] = sv.hist[i];
    out->evaluated = sv.evaluated;
    const double nb = (double)std::max<int64_t>(1, sv.search_batches);
    out->batch_fill_us = sv.fill_ns / nb / 1e3;
    out->batch_flight_us = sv.flight_ns / nb / 1e3;
    out->submit_us = sv.submit_ns / nb / 1e3;
    out->gpu_busy_s = sv.busy_ns / 1e9;
    out->d_init = sv.d_init;
    out->work_items = sv.tree.empty() ? 0 : (int64_t)(sv.level_start[sv.d_init + 1] - sv.level_start[sv.d_init]);
    out->seconds = std::chrono::duration<double>(Clock::now() - t0).count();
    return rc;
}

void cbdfs_search_defaults(cbdfs_search_cfg *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->threads = 4;
    cfg->work_num = 16;
    cfg->d_init = -1;
    cfg->batch = 4096;
    cfg->timeout_us = 4000;
    cfg->complete_final = 1;
    cfg->fixed_tree_heur = CBDFS_HEUR_NONE;
    cfg->bts_n0 = 10000;
    cfg->bts_c1 = 2;
    cfg->bts_c2 = 8;
}

void cbdfs_cancel(cbdfs_ctx *ctx) {
    if (ctx) reinterpret_cast<Ctx *>(ctx)->cancel = 1;
}

}  // extern "C"
