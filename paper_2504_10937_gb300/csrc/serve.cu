// Batched queries and the serving loop: many top-k queries in flight at once
// on one GPU.  Host code only; every query runs the same kernels as lds_topk.
//
// A pool of worker threads, each with its own non-blocking CUDA stream, takes
// requests from a FIFO queue.  A request is admitted when (a) its graph handle
// is idle (a handle is never used by two threads at once) and (b) its
// estimated device footprint fits in what is left of the memory budget;
// among the admissible requests the oldest goes first (continuous batching:
// requests join as slots and memory free up and leave when they finish, and
// their kernels overlap on the device through the separate streams).  While a
// worker runs a request it points the handle, and every buffer the handle
// owns, at its own stream, and afterwards back at the handle's stream: the
// buffers free themselves on the stream they follow, so a free is always
// ordered after the work that used the buffer and never names a worker stream
// that no longer exists.  The paper has no counterpart to this
// layer: it only schedules queries the paper defines.
#include <chrono>
#include <condition_variable>
#include <map>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "graph.cuh"

namespace lds {

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    int64_t ticket = 0;
    lds_query q{};
    int64_t bytes = 0;
    lds_status status = LDS_OK;
    std::string error;
    lds_result* result = nullptr;
    lds_topk_stats_t stats{};
    Clock::time_point t_submit, t_start, t_end;
    bool done = false;
};

// Estimated device bytes of one query: the Frank-Wolfe state, the view, the
// pruning and verification buffers and one refinement copy, per edge and per
// vertex (and per triangle for LTDS; a graph whose triangles are not listed
// yet is charged 16 per edge as a stand-in).
int64_t footprint(const lds_query& q) {
    const lds_graph* g = q.g;
    int64_t b = 96 * g->m + 96 * (int64_t)g->n + (1 << 20);
    if (q.d == LDS_TRIANGLE) b += 64 * (g->ntri >= 0 ? g->ntri : 16 * g->m);
    return b;
}

}  // namespace

// Index of the request to admit next, or -1: the oldest one whose graph is
// idle and whose footprint fits in `free_bytes`.
int32_t pick_next(int32_t nq, const int64_t* bytes, const uint8_t* graph_busy, int64_t free_bytes) {
    for (int32_t i = 0; i < nq; ++i)
        if (!graph_busy[i] && bytes[i] <= free_bytes) return i;
    return -1;
}

}  // namespace lds

using namespace lds;

struct lds_server {
    int device = 0;
    int64_t budget = 0;
    int64_t in_use = 0;
    bool stop = false;
    int64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> live;
    std::unordered_set<const lds_graph*> busy;
    std::vector<std::thread> workers;

    // next admissible request (mu held), removed from the queue
    std::shared_ptr<Request> take() {
        std::vector<int64_t> bytes;
        std::vector<uint8_t> gb;
        bytes.reserve(queue.size());
        gb.reserve(queue.size());
        for (auto& r : queue) {
            bytes.push_back(r->bytes);
            gb.push_back(busy.count(r->q.g) ? 1 : 0);
        }
        int32_t i = pick_next((int32_t)queue.size(), bytes.data(), gb.data(), budget - in_use);
        if (i < 0) return nullptr;
        auto r = queue[i];
        queue.erase(queue.begin() + i);
        return r;
    }

    void run(Request& r, cudaStream_t ws) {
        lds_graph* g = r.q.g;
        cudaStream_t old = g->stream;
        lds_status st = (lds_status)0;
        if (cudaStreamSynchronize(old) != cudaSuccess) {
            r.status = LDS_ECUDA;
            r.error = "lds_server: the graph's stream reported an error";
            return;
        }
        // the handle and its buffers follow the worker's stream during the query,
        // so that every stream-ordered free is ordered after the work that used it
        set_stream(g, ws);
        st = lds_topk(g, r.q.k, r.q.d, r.q.iters, r.q.p, &r.result);
        if (st != LDS_OK) r.error = lds_last_error();
        else lds_topk_last_stats(&r.stats);
        cudaStreamSynchronize(ws);
        set_stream(g, old);
        r.status = st;
    }

    void worker_main() {
        cudaSetDevice(device);
        cudaStream_t ws = nullptr;
        const bool ok = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            std::shared_ptr<Request> r;
            cv_work.wait(lk, [&] { return (r = take()) != nullptr || (stop && queue.empty()); });
            if (!r) break;
            busy.insert(r->q.g);
            in_use += r->bytes;
            r->t_start = Clock::now();
            lk.unlock();
            if (ok) {
                run(*r, ws);
            } else {
                r->status = LDS_ECUDA;
                r->error = "lds_server: could not create a worker stream";
            }
            lk.lock();
            r->t_end = Clock::now();
            busy.erase(r->q.g);
            in_use -= r->bytes;
            r->done = true;
            cv_done.notify_all();
            cv_work.notify_all();
        }
        lk.unlock();
        if (ws) cudaStreamDestroy(ws);
    }
};

namespace {

lds_status check_query(const lds_query* q) {
    return guard([&] {
        LDS_REQUIRE(q && q->g, LDS_EINVAL, "lds_server_submit: NULL query or graph");
        LDS_REQUIRE(q->k >= 1, LDS_EINVAL, "lds_server_submit: k = %d < 1", q->k);
        LDS_REQUIRE(q->d == LDS_EDGE || q->d == LDS_TRIANGLE, LDS_EINVAL, "lds_server_submit: bad density");
        LDS_REQUIRE(q->p == LDS_EXACT || q->p == LDS_FP32 || q->p == LDS_FP64, LDS_EINVAL,
                    "lds_server_submit: bad precision");
        LDS_REQUIRE(q->iters >= 1, LDS_EINVAL, "lds_server_submit: iters = %d < 1", q->iters);
    });
}

// worker counts tried by the batch autotuner, and its choice per size bucket
const int32_t kTry[] = {1, 2, 4, 8, 16};
std::mutex g_tune_mu;
std::unordered_map<int, int32_t> g_tuned;

int size_bucket(const lds_query* qs, int32_t count) {
    double s = 0;
    for (int32_t i = 0; i < count; ++i) s += (double)qs[i].g->m + 1.0;
    int b = 0;
    for (double v = s / std::max(count, 1); v >= 2.0; v /= 2.0) ++b;
    return b;
}

}  // namespace

extern "C" {

lds_status lds_server_create(int64_t budget_bytes, int32_t workers, lds_server** out) {
    return guard([&] {
        LDS_REQUIRE(out, LDS_EINVAL, "lds_server_create: out is NULL");
        *out = nullptr;
        LDS_REQUIRE(budget_bytes > 0, LDS_EINVAL, "lds_server_create: budget must be positive");
        LDS_REQUIRE(workers >= 1 && workers <= 256, LDS_EINVAL, "lds_server_create: workers = %d out of [1, 256]",
                    workers);
        LDS_REQUIRE(lds_device_count() > 0, LDS_ECUDA, "lds_server_create: no CUDA device");
        auto* s = new lds_server();
        LDS_CUDA(cudaGetDevice(&s->device));
        s->budget = budget_bytes;
        for (int32_t i = 0; i < workers; ++i) s->workers.emplace_back([s] { s->worker_main(); });
        *out = s;
    });
}

lds_status lds_server_submit(lds_server* s, const lds_query* q, int64_t* ticket) {
    lds_status st = check_query(q);
    if (st != LDS_OK) return st;
    return guard([&] {
        LDS_REQUIRE(s && ticket, LDS_EINVAL, "lds_server_submit: NULL argument");
        auto r = std::make_shared<Request>();
        r->q = *q;
        r->bytes = footprint(*q);
        LDS_REQUIRE(r->bytes <= s->budget, LDS_EBUSY,
                    "lds_server_submit: the query needs about %lld bytes, above the budget of %lld",
                    (long long)r->bytes, (long long)s->budget);
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            LDS_REQUIRE(!s->stop, LDS_EINVAL, "lds_server_submit: the server is shutting down");
            r->ticket = s->next_ticket++;
            s->queue.push_back(r);
            s->live[r->ticket] = r;
        }
        s->cv_work.notify_one();
        *ticket = r->ticket;
    });
}

lds_status lds_server_poll(lds_server* s, int64_t ticket, int32_t* done) {
    return guard([&] {
        LDS_REQUIRE(s && done, LDS_EINVAL, "lds_server_poll: NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->live.find(ticket);
        LDS_REQUIRE(it != s->live.end(), LDS_EINVAL, "lds_server_poll: unknown ticket %lld", (long long)ticket);
        *done = it->second->done ? 1 : 0;
    });
}

lds_status lds_server_wait(lds_server* s, int64_t ticket, lds_result** out, lds_request_info* info) {
    std::shared_ptr<Request> r;
    lds_status st = guard([&] {
        LDS_REQUIRE(s && out, LDS_EINVAL, "lds_server_wait: NULL argument");
        *out = nullptr;
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->live.find(ticket);
        LDS_REQUIRE(it != s->live.end(), LDS_EINVAL, "lds_server_wait: unknown ticket %lld", (long long)ticket);
        r = it->second;
        s->cv_done.wait(lk, [&] { return r->done; });
        s->live.erase(ticket);
    });
    if (st != LDS_OK) return st;
    if (info) {
        info->queue_ms = ms_between(r->t_submit, r->t_start);
        info->run_ms = ms_between(r->t_start, r->t_end);
        info->footprint_bytes = r->bytes;
        info->stats = r->stats;
    }
    if (r->status != LDS_OK) {
        set_error("%s", r->error.c_str());
        return r->status;
    }
    *out = r->result;
    r->result = nullptr;
    return LDS_OK;
}

void lds_server_destroy(lds_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->live) lds_result_free(kv.second->result);
    delete s;
}

int32_t lds_debug_pick_next(int32_t nq, const int64_t* bytes, const uint8_t* graph_busy, int64_t free_bytes) {
    if (nq <= 0 || !bytes || !graph_busy) return -1;
    return pick_next(nq, bytes, graph_busy, free_bytes);
}

lds_status lds_topk_batch(int32_t count, const lds_query* queries, int32_t workers, lds_result** results,
                          lds_status* status) {
    lds_status st = guard([&] {
        LDS_REQUIRE(count >= 0, LDS_EINVAL, "lds_topk_batch: count < 0");
        LDS_REQUIRE(count == 0 || (queries && results && status), LDS_EINVAL, "lds_topk_batch: NULL argument");
        LDS_REQUIRE(workers >= 0 && workers <= 256, LDS_EINVAL, "lds_topk_batch: workers = %d out of [0, 256]",
                    workers);
    });
    if (st != LDS_OK || count == 0) return st;
    for (int32_t i = 0; i < count; ++i) {
        results[i] = nullptr;
        status[i] = check_query(queries + i);
        if (status[i] != LDS_OK) return status[i];
    }
    if (workers == 0) {
        int32_t w = 0;
        st = lds_batch_autotune(count, queries, &w);
        if (st != LDS_OK) return st;
        workers = w;
    }
    // First rounds of the edge-density queries in one persistent launch: every
    // graph that appears in exactly one query of the batch, grouped by
    // (iterations, arithmetic); the queries then take that state as it is.
    {
        std::unordered_map<const lds_graph*, int32_t> uses;
        for (int32_t i = 0; i < count; ++i) ++uses[queries[i].g];
        std::unordered_map<int64_t, std::vector<lds_graph*>> groups;
        for (int32_t i = 0; i < count; ++i) {
            const lds_query& q = queries[i];
            if (q.d != LDS_EDGE || uses[q.g] != 1) continue;
            groups[((int64_t)q.iters << 2) | (int64_t)q.p].push_back(q.g);
        }
        for (auto& kv : groups) {
            st = lds_fw_batch((int32_t)kv.second.size(), kv.second.data(), (int32_t)(kv.first >> 2),
                              (lds_precision)(kv.first & 3), nullptr);
            if (st != LDS_OK) return st;
        }
    }
    lds_server* s = nullptr;
    st = lds_server_create(INT64_MAX, workers, &s);
    if (st != LDS_OK) return st;
    std::vector<int64_t> tickets(count, 0);
    lds_status first = LDS_OK;
    for (int32_t i = 0; i < count; ++i) {
        status[i] = lds_server_submit(s, queries + i, &tickets[i]);
        if (status[i] != LDS_OK && first == LDS_OK) first = status[i];
    }
    std::string msg;
    for (int32_t i = 0; i < count; ++i) {
        if (!tickets[i]) continue;
        status[i] = lds_server_wait(s, tickets[i], results + i, nullptr);
        if (status[i] != LDS_OK && first == LDS_OK) {
            first = status[i];
            msg = lds_last_error();
        }
    }
    lds_server_destroy(s);
    if (first != LDS_OK && !msg.empty()) set_error("%s", msg.c_str());
    return first;
}

lds_status lds_batch_autotune(int32_t count, const lds_query* queries, int32_t* workers) {
    return guard([&] {
        LDS_REQUIRE(count > 0 && queries && workers, LDS_EINVAL, "lds_batch_autotune: bad argument");
        const int bucket = size_bucket(queries, count);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(bucket);
            if (it != g_tuned.end()) {
                *workers = it->second;
                return;
            }
        }
        // the on-chip first-round Frank-Wolfe: threads per graph for every size bucket of
        // the batch's edge queries, per iteration count and arithmetic
        {
            std::map<std::pair<int32_t, int>, std::vector<lds_graph*>> groups;
            std::unordered_set<lds_graph*> seen;
            for (int32_t i = 0; i < count; ++i)
                if (queries[i].d == LDS_EDGE && seen.insert(queries[i].g).second)
                    groups[{queries[i].iters, (int)queries[i].p}].push_back(queries[i].g);
            for (auto& kv : groups)
                fw_batch_autotune((int32_t)kv.second.size(), kv.second.data(), kv.first.first,
                                  (lds_precision)kv.first.second);
        }
        // time a sample of the batch with each worker count; keep the fastest
        const int32_t sample = std::min<int32_t>(count, 64);
        double best = 1e300;
        int32_t best_w = 1;
        for (int32_t w : kTry) {
            if (w > 1 && w > sample) break;
            std::vector<lds_result*> res(sample, nullptr);
            std::vector<lds_status> sts(sample, LDS_OK);
            auto t0 = Clock::now();
            lds_status st = lds_topk_batch(sample, queries, w, res.data(), sts.data());
            const double ms = ms_between(t0, Clock::now());
            for (auto* r : res) lds_result_free(r);
            LDS_REQUIRE(st == LDS_OK, st, "lds_batch_autotune: %s", lds_last_error());
            if (ms < best) {
                best = ms;
                best_w = w;
            }
        }
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[bucket] = best_w;
        }
        *workers = best_w;
    });
}

}  // extern "C"
