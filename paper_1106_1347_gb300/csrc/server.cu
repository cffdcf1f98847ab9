// Serving runtime: a request loop for products of uneven shapes with a
// requested accuracy tier, continuous batching, admission by an HBM budget,
// and latency statistics.  No counterpart in the paper.
//
// The caller hands the server one device arena (its HBM budget) at creation;
// the server never allocates device memory.  A worker thread:
//   * admits requests in arrival order (skipping past ones that do not fit yet)
//     when their device copies of A, B and C plus their split workspace fit
//     in the arena (first fit) -- so an admitted request can always run;
//   * whenever one of its K stream slots is free, forms a batch from every
//     admitted request of the oldest request's slice format and count (up to
//     max_batch and past the first request up to 4 ms of estimated work, a cap
//     MM_SERVER_BATCH_MS changes) and enqueues on that slot's stream: host-to-device
//     copies of A and B, the table upload, one grouped emulated launch
//     (replayed from a CUDA graph cached per slot, slice format and count, when
//     enabled -- the grouped kernels run fixed grids), device-to-host copies
//     of C, and an event;
//   * retires batches whose event has fired, frees their memory and records
//     each request's latency (arrival to result in the caller's host buffer).
// Requests that arrive while batches are on the GPU are admitted and launched
// in the next free slot, so their work overlaps the running batches.
// A plain-FP64 mode (one request at a time with mm_naive's kernel) serves the
// same trace as a baseline.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// First-fit allocator over the caller's device arena (offsets, 256-byte granules).
class ArenaAlloc {
   public:
    void init(char *base, size_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    char *alloc(size_t bytes) {
        bytes = mm::align_up(std::max<size_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return base_ + off;
        }
        return nullptr;
    }
    void release(char *p, size_t bytes) {
        if (!p) return;
        bytes = mm::align_up(std::max<size_t>(bytes, 1), 256);
        size_t off = (size_t)(p - base_);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t capacity() const { return size_; }
    size_t peak() const { return peak_; }

   private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Req {
    mm_request r;
    int s = 0, kind = MM_SLICE_BF16;  // slice count (0: plain FP64) and format
    Clock::time_point arrival, launched;
    char *block = nullptr;
    size_t block_bytes = 0;
    double *dA = nullptr, *dB = nullptr, *dC = nullptr;
};

using GraphKey = std::tuple<int, int64_t, int64_t, int64_t, int64_t, int64_t>;

struct Slot {
    cudaStream_t stream = nullptr;
    char *table_dev = nullptr;
    size_t table_cap = 0;
    unsigned char *staging = nullptr;  // pinned image of the table part
    std::map<GraphKey, cudaGraphExec_t> graphs;
    bool busy = false;
};

struct Batch {
    int slot;
    std::vector<Req *> reqs;
    cudaEvent_t start = nullptr, done = nullptr;  // timing events before the first copy and after the last
};

size_t operand_bytes(const mm_request &r) {
    return mm::align_up((size_t)(r.N * r.P) * 8, 1024) + mm::align_up((size_t)(r.P * r.M) * 8, 1024) +
           mm::align_up((size_t)(r.N * r.M) * 8, 1024);
}

// Device bytes one request holds from admission to completion: A, B, C and,
// for the emulated method, its split workspace.
size_t request_bytes(const mm_request &r, int s, int kind) {
    size_t b = operand_bytes(r);
    if (s > 0)
        b += mm::problem_data_bytes(mm_problem{r.N, r.P, r.M, nullptr, r.P, nullptr, r.M, nullptr, r.M}, s, kind);
    return b;
}

// Rough device time of one request (copies over a ~200 GB/s host link plus
// the slice products at ~1.2 (BF16) or ~2.4 (FP8) PFLOP/s per pair), used only
// to bound how much work one batch takes on.
double request_ms(const Req &q) {
    const mm_request &r = q.r;
    const double bytes = 8.0 * ((double)r.N * r.P + (double)r.P * r.M + (double)r.N * r.M);
    const double pairs = q.s * (q.s + 1) / 2.0;
    const double rate = q.kind == MM_SLICE_FP8E4M3 ? 2.4e15 : 1.2e15;
    return 1e3 * (bytes / 200e9 + 2.0 * r.N * r.P * r.M * pairs / rate);
}

// The slice format and count for a request's tier.  Method 2 takes the
// autotuner's choice for the request's shape bucket when one is recorded, else
// FP8-E4M3 slices when the tier allows them (at most 8) and their pairs, at
// twice the BF16 rate, cost less than the BF16 pairs the tier needs.  (Batches
// run the direct product: a tuned Strassen level count is not used here.)
void choose_slices(int method, const mm_request &r, int *s, int *kind) {
    *kind = MM_SLICE_BF16;
    *s = mm::emulated_slices(MM_SLICE_BF16, 0, r.tier);
    if (method != 2) return;
    int k = 0, n = 0, levels = 0, tile = 0;  // a batch runs with the default tile width
    if (mm::emulated_choice(r.N, r.P, r.M, r.tier, &k, &n, &levels, &tile) >= 0) {
        *kind = k;
        *s = n;
    }
}

}  // namespace

struct mm_server {
    int device = 0;
    ArenaAlloc arena;
    int max_batch = 64, method = 0;
    double batch_ms_cap = 4.0;  // estimated device time per batch (MM_SERVER_BATCH_MS; 0: no cap)
    double class_ratio = 0.0;   // batch only requests within this factor of the oldest one's time (0: off)
    bool use_graphs = true;
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> incoming;
    bool stop = false;
    std::thread worker;

    std::deque<Req *> pending;
    std::vector<Req *> admitted;
    std::vector<Batch> inflight;

    cudaEvent_t t0 = nullptr;  // timing origin of the batches' device intervals
    std::mutex res_mu;
    std::vector<std::pair<float, float>> intervals;  // each batch's [start, done] on the device, ms after t0
    std::deque<mm_completion> done;
    std::vector<double> latencies;
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, graph_replays = 0;
    double flops = 0.0;
    bool have_first = false;
    Clock::time_point first_arrival, last_done;
    int fatal = MM_OK;
    std::string fatal_msg;

    void set_fatal(int rc) {  // keeps the first failure's status and message
        std::lock_guard<std::mutex> g(res_mu);
        if (fatal == MM_OK) {
            fatal = rc;
            fatal_msg = mm_last_error();
        }
    }

    void finish(Req *q, int status, Clock::time_point now) {
        mm_completion c{};
        c.tag = q->r.tag;
        c.status = status;
        c.slices = q->s;
        c.kind = q->kind;
        c.queue_ms = q->launched.time_since_epoch().count() ? ms_between(q->arrival, q->launched) : 0.0;
        c.latency_ms = ms_between(q->arrival, now);
        {
            std::lock_guard<std::mutex> g(res_mu);
            done.push_back(c);
            if (status == MM_OK) {
                latencies.push_back(c.latency_ms);
                flops += 2.0 * (double)q->r.N * (double)q->r.P * (double)q->r.M;
                last_done = now;
                ++completed;
            } else {
                ++rejected;
            }
        }
        delete q;
    }

    void retire() {
        for (size_t i = 0; i < inflight.size();) {
            Batch &b = inflight[i];
            cudaError_t e = cudaEventQuery(b.done);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const Clock::time_point now = Clock::now();
            const int st = (e == cudaSuccess) ? MM_OK : MM_ERR_CUDA;
            if (e != cudaSuccess) set_fatal(mm::cuda_fail(e, "server: batch completion"));
            float ts = 0.f, te = 0.f;
            if (e == cudaSuccess && cudaEventElapsedTime(&ts, t0, b.start) == cudaSuccess &&
                cudaEventElapsedTime(&te, t0, b.done) == cudaSuccess) {
                std::lock_guard<std::mutex> g(res_mu);
                intervals.emplace_back(ts, te);
            }
            for (Req *q : b.reqs) {
                arena.release(q->block, q->block_bytes);
                finish(q, st, now);
            }
            cudaEventDestroy(b.start);
            cudaEventDestroy(b.done);
            slots[b.slot].busy = false;
            inflight.erase(inflight.begin() + i);
        }
    }

    void admit() {
        int looked = 0;
        for (auto it = pending.begin(); it != pending.end() && looked < 256; ++looked) {
            Req *q = *it;
            const size_t need = request_bytes(q->r, q->s, q->kind);
            if (need > arena.capacity()) {  // can never fit this budget
                it = pending.erase(it);
                finish(q, MM_ERR_NOMEM, Clock::now());
                continue;
            }
            char *blk = arena.alloc(need);
            if (!blk) {
                ++it;
                continue;
            }
            q->block = blk;
            q->block_bytes = need;
            q->dA = (double *)blk;
            q->dB = (double *)(blk + mm::align_up((size_t)(q->r.N * q->r.P) * 8, 1024));
            q->dC = (double *)((char *)q->dB + mm::align_up((size_t)(q->r.P * q->r.M) * 8, 1024));
            admitted.push_back(q);
            it = pending.erase(it);
        }
    }

    int launch_batch(Slot &sl, int slot_index, std::vector<Req *> &reqs) {
        cudaStream_t st = sl.stream;
        Batch b;
        b.slot = slot_index;
        std::vector<mm_problem> probs;
        std::vector<char *> data;
        const int s = reqs[0]->s, kind = reqs[0]->kind;
        if (method != 1) {
            for (Req *q : reqs) {
                probs.push_back(mm_problem{q->r.N, q->r.P, q->r.M, q->dA, q->r.P, q->dB, q->r.M, q->dC, q->r.M});
                data.push_back(q->block + operand_bytes(q->r));
            }
            if ((int)probs.size() > max_batch) return mm::fail(MM_ERR_NOMEM, "server: batch exceeds max_batch");
        }
        auto give_back = [&](int rc) {
            cudaStreamSynchronize(st);  // nothing of this batch may still touch its memory
            if (b.start) cudaEventDestroy(b.start);
            if (b.done) cudaEventDestroy(b.done);
            return rc;
        };
        const Clock::time_point now = Clock::now();
        {
            cudaError_t e = cudaEventCreate(&b.start);
            if (e == cudaSuccess) e = cudaEventRecord(b.start, st);
            if (e != cudaSuccess) {
                if (b.start) cudaEventDestroy(b.start);
                return mm::cuda_fail(e, "server: batch start event");
            }
        }
        for (Req *q : reqs) {
            q->launched = now;
            const mm_request &r = q->r;
            cudaError_t e = cudaMemcpy2DAsync(q->dA, r.P * 8, r.A, r.lda * 8, r.P * 8, r.N, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(q->dB, r.M * 8, r.B, r.ldb * 8, r.M * 8, r.P, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: host-to-device copy"));
        }
        int rc = MM_OK;
        if (method == 1) {
            Req *q = reqs[0];
            rc = mm::run_naive(q->r.N, q->r.P, q->r.M, q->dA, q->r.P, q->dB, q->r.M, q->dC, q->r.M, st);
        } else {
            std::vector<unsigned char> image;
            mm::GroupLaunch gl{};
            rc = mm::group_build(probs.data(), (int)probs.size(), max_batch, s, sl.table_dev, data.data(), image,
                                 gl, kind);
            if (rc) return give_back(rc);
            std::memcpy(sl.staging, image.data(), image.size());
            cudaError_t e = cudaMemcpyAsync(sl.table_dev, sl.staging, image.size(), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: table upload"));
            if (use_graphs) {
                // Fixed grids (the kernels stride over their units): one graph per
                // slice format and count serves every batch.
                for (int k = 0; k < 5; ++k) gl.grid[k] = mm::group_grid_cap(k);
                const GraphKey key{s + 16 * kind, gl.grid[0], gl.grid[1], gl.grid[2], gl.grid[3], gl.grid[4]};
                auto it = sl.graphs.find(key);
                if (it == sl.graphs.end()) {
                    cudaGraph_t graph = nullptr;
                    cudaGraphExec_t exec = nullptr;
                    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                    if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: begin capture"));
                    mm::prof_suspend(true);
                    rc = mm::group_kernels(gl, st);
                    mm::prof_suspend(false);
                    e = cudaStreamEndCapture(st, &graph);
                    if (rc) {
                        if (graph) cudaGraphDestroy(graph);
                        return give_back(rc);
                    }
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
                    if (graph) cudaGraphDestroy(graph);
                    if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: graph capture"));
                    it = sl.graphs.emplace(key, exec).first;
                } else {
                    std::lock_guard<std::mutex> g(res_mu);
                    ++graph_replays;
                }
                e = cudaGraphLaunch(it->second, st);
                if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: graph launch"));
            } else {
                rc = mm::group_kernels(gl, st);
            }
        }
        if (rc) return give_back(rc);
        for (Req *q : reqs) {
            const mm_request &r = q->r;
            cudaError_t e = cudaMemcpy2DAsync(r.C, r.ldc * 8, q->dC, r.M * 8, r.M * 8, r.N, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: device-to-host copy"));
        }
        cudaError_t e = cudaEventCreate(&b.done);
        if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
        if (e != cudaSuccess) return give_back(mm::cuda_fail(e, "server: completion event"));
        b.reqs = reqs;
        sl.busy = true;
        inflight.push_back(b);
        {
            std::lock_guard<std::mutex> g(res_mu);
            ++batches;
        }
        return MM_OK;
    }

    bool launch_ready() {
        bool any = false;
        for (size_t k = 0; k < slots.size() && !admitted.empty(); ++k) {
            if (slots[k].busy) continue;
            const int s = admitted.front()->s, kind = admitted.front()->kind;
            const int cap = method == 1 ? 1 : max_batch;
            const double front_ms = request_ms(*admitted.front());
            std::vector<Req *> take;
            double est_ms = 0.0;
            for (auto it = admitted.begin(); it != admitted.end() && (int)take.size() < cap;) {
                const double t = request_ms(**it);
                // The oldest request always goes; the class filter applies to the others.
                const bool same_class = take.empty() || class_ratio <= 0.0 ||
                                        (t <= class_ratio * front_ms && front_ms <= class_ratio * t);
                if ((*it)->s == s && (*it)->kind == kind && same_class) {
                    if (!take.empty() && batch_ms_cap > 0.0 && est_ms + t > batch_ms_cap) break;
                    est_ms += t;
                    take.push_back(*it);
                    it = admitted.erase(it);
                } else {
                    ++it;
                }
            }
            if (take.empty()) break;
            const int rc = launch_batch(slots[k], (int)k, take);
            if (rc == MM_OK) {
                any = true;
            } else {
                set_fatal(rc);
                const Clock::time_point now = Clock::now();
                for (Req *q : take) {
                    arena.release(q->block, q->block_bytes);
                    finish(q, rc, now);
                }
            }
        }
        return any;
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            {
                std::unique_lock<std::mutex> g(mu);
                while (!incoming.empty()) {
                    pending.push_back(incoming.front());
                    incoming.pop_front();
                }
                if (stop && pending.empty() && admitted.empty() && inflight.empty()) break;
                if (stop) {  // cancel what has not started
                    const Clock::time_point now = Clock::now();
                    for (Req *q : pending) finish(q, MM_ERR_TIMEOUT, now);
                    pending.clear();
                    for (Req *q : admitted) {
                        arena.release(q->block, q->block_bytes);
                        finish(q, MM_ERR_TIMEOUT, now);
                    }
                    admitted.clear();
                }
            }
            retire();
            admit();
            const bool launched = launch_ready();
            if (!launched) {
                std::unique_lock<std::mutex> g(mu);
                cv.wait_for(g, std::chrono::microseconds(inflight.empty() ? 500 : 20),
                            [&] { return !incoming.empty() || stop; });
            }
        }
    }
};

extern "C" {

int mm_server_create(void *arena, size_t arena_bytes, int32_t max_batch, int32_t nstreams, int32_t use_graphs,
                     int32_t method, mm_server **out) {
    if (!out) return mm::fail(MM_ERR_ARG, "mm_server_create: NULL out");
    if (!arena || arena_bytes == 0) return mm::fail(MM_ERR_ARG, "mm_server_create: empty arena");
    if (max_batch < 1 || max_batch > 4096 || nstreams < 1 || nstreams > 32 || method < 0 || method > 2)
        return mm::fail(MM_ERR_ARG, "mm_server_create: max_batch 1..4096, nstreams 1..32, method 0, 1 or 2");
    mm_server *s = new mm_server();
    cudaGetDevice(&s->device);
    s->max_batch = method == 1 ? 1 : max_batch;
    if (const char *cap = getenv("MM_SERVER_BATCH_MS")) s->batch_ms_cap = atof(cap);
    if (const char *ratio = getenv("MM_SERVER_CLASS_RATIO")) {
        // A factor below 1 would exclude every request but the oldest: values in (0, 1) count as 1.
        const double r = atof(ratio);
        s->class_ratio = r <= 0.0 ? 0.0 : std::max(1.0, r);
    }
    s->method = method;
    s->use_graphs = use_graphs != 0 && method != 1;
    const size_t table_cap = mm::group_table_bytes(s->max_batch);
    const int ns = method == 1 ? 1 : nstreams;
    // Per-slot table parts live at the front of the arena.
    if (table_cap * ns >= arena_bytes / 2) {
        delete s;
        return mm::fail(MM_ERR_NOMEM, "mm_server_create: arena too small for %d slots of %zu bytes", ns, table_cap);
    }
    s->slots.resize(ns);
    for (int k = 0; k < ns; ++k) {
        Slot &sl = s->slots[k];
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.staging, table_cap);
        if (e != cudaSuccess) {
            delete s;
            return mm::cuda_fail(e, "mm_server_create");
        }
        sl.table_dev = (char *)arena + (size_t)k * table_cap;
        sl.table_cap = table_cap;
    }
    {
        cudaError_t e = cudaEventCreate(&s->t0);
        if (e == cudaSuccess) e = cudaEventRecord(s->t0, s->slots[0].stream);
        if (e != cudaSuccess) {
            for (Slot &sl : s->slots) {
                if (sl.stream) cudaStreamDestroy(sl.stream);
                if (sl.staging) cudaFreeHost(sl.staging);
            }
            if (s->t0) cudaEventDestroy(s->t0);
            delete s;
            return mm::cuda_fail(e, "mm_server_create: timing event");
        }
    }
    s->arena.init((char *)arena + table_cap * ns, arena_bytes - table_cap * ns);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return MM_OK;
}

int mm_server_submit(mm_server *s, const mm_request *req) {
    if (!s || !req) return mm::fail(MM_ERR_ARG, "mm_server_submit: NULL argument");
    const mm_request &r = *req;
    if (r.N < 0 || r.P < 0 || r.M < 0 || r.lda < std::max<int64_t>(1, r.P) || r.ldb < std::max<int64_t>(1, r.M) ||
        r.ldc < std::max<int64_t>(1, r.M))
        return mm::fail(MM_ERR_ARG, "mm_server_submit: bad shape or leading dimension");
    if ((r.N && r.P && !r.A) || (r.P && r.M && !r.B) || (r.N && r.M && !r.C))
        return mm::fail(MM_ERR_ARG, "mm_server_submit: NULL host pointer");
    if (s->method != 1 && !(r.tier > 0.0)) return mm::fail(MM_ERR_ARG, "mm_server_submit: tier must be > 0");
    if (r.P > (int64_t(1) << 20)) return mm::fail(MM_ERR_UNSUPPORTED, "mm_server_submit: P > 2^20");
    Req *q = new Req();
    q->r = r;
    q->arrival = Clock::now();
    if (s->method != 1) choose_slices(s->method, r, &q->s, &q->kind);
    {
        std::lock_guard<std::mutex> g(s->res_mu);
        ++s->submitted;
        if (!s->have_first) {
            s->have_first = true;
            s->first_arrival = q->arrival;
        }
    }
    if (r.N == 0 || r.M == 0 || r.P == 0) {  // nothing to compute on the device
        if (r.P == 0)
            for (int64_t i = 0; i < r.N; ++i) std::memset(r.C + i * r.ldc, 0, (size_t)r.M * 8);
        s->finish(q, MM_OK, Clock::now());
        return MM_OK;
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->incoming.push_back(q);
    }
    s->cv.notify_one();
    return MM_OK;
}

int mm_server_poll(mm_server *s, mm_completion *out, int32_t cap) {
    if (!s || (cap > 0 && !out)) return mm::fail(MM_ERR_ARG, "mm_server_poll: NULL argument");
    std::lock_guard<std::mutex> g(s->res_mu);
    int n = 0;
    while (n < cap && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

int mm_server_wait(mm_server *s, int64_t timeout_ms) {
    if (!s) return mm::fail(MM_ERR_ARG, "mm_server_wait: NULL server");
    const Clock::time_point end = Clock::now() + std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0));
    for (;;) {
        {
            std::lock_guard<std::mutex> g(s->res_mu);
            if (s->completed + s->rejected >= s->submitted) return s->fatal;
        }
        if (Clock::now() >= end) return mm::fail(MM_ERR_TIMEOUT, "mm_server_wait: requests still in flight");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

int mm_server_stats(mm_server *s, mm_server_stats_t *out) {
    if (!s || !out) return mm::fail(MM_ERR_ARG, "mm_server_stats: NULL argument");
    std::lock_guard<std::mutex> g(s->res_mu);
    mm_server_stats_t st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.rejected = s->rejected;
    st.batches = s->batches;
    st.graph_replays = s->graph_replays;
    st.flops = s->flops;
    st.peak_arena_bytes = (int64_t)s->arena.peak();
    std::vector<double> lat = s->latencies;
    std::sort(lat.begin(), lat.end());
    if (!lat.empty()) {
        auto q = [&](double f) { return lat[std::min(lat.size() - 1, (size_t)(f * (double)(lat.size() - 1) + 0.5))]; };
        st.p50_ms = q(0.50);
        st.p99_ms = q(0.99);
        st.max_ms = lat.back();
        double sum = 0;
        for (double v : lat) sum += v;
        st.mean_ms = sum / (double)lat.size();
        st.busy_s = ms_between(s->first_arrival, s->last_done) / 1e3;
    }
    // Device time covered by at least one batch, and by at least two at once
    // (batches on different streams overlapping), from the batches' events.
    std::vector<std::pair<float, int>> ends;
    for (const auto &iv : s->intervals) {
        ends.emplace_back(iv.first, +1);
        ends.emplace_back(iv.second, -1);
    }
    std::sort(ends.begin(), ends.end());  // at equal times an end (-1) sorts before a start (+1)
    int active = 0;
    for (size_t i = 0; i < ends.size(); ++i) {
        if (i > 0) {
            const double dt = (double)ends[i].first - (double)ends[i - 1].first;
            if (active >= 1) st.device_busy_ms += dt;
            if (active >= 2) st.overlap_ms += dt;
        }
        active += ends[i].second;
    }
    *out = st;
    return MM_OK;
}

const char *mm_server_error(mm_server *s) {
    if (!s) return "";
    std::lock_guard<std::mutex> g(s->res_mu);
    return s->fatal_msg.c_str();
}

int mm_server_destroy(mm_server *s) {
    if (!s) return MM_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_one();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) {
        for (auto &kv : sl.graphs) cudaGraphExecDestroy(kv.second);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.staging) cudaFreeHost(sl.staging);
    }
    if (s->t0) cudaEventDestroy(s->t0);
    int fatal;
    {
        std::lock_guard<std::mutex> g(s->res_mu);
        fatal = s->fatal;
    }
    delete s;
    return fatal;
}

}  // extern "C"
