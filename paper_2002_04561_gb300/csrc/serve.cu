// Serving runtime: a request queue in front of the alignment paths (not in the
// paper; its GPU mapping aligns one pair or one batch per call).
//
// Callers submit single pairs from any thread. Two service lanes, each a
// worker thread with its own context and CUDA stream, drain two queues in
// micro-batches: a lane waits at most max_wait_us after its oldest queued
// request (or until max_batch_pairs are queued). The short lane aligns its
// batch with one anyseq_align_batch call (inter-sequence parallelism); the long
// lane takes the pairs of at least long_cells cells and runs them side by side
// in one wavefront launch (intra-sequence parallelism) with one CTA per SM, so
// that the short lane's kernels still find room on every SM: short requests do
// not queue behind a long pair. Admission: the letters of queued and running
// requests may not exceed mem_budget_bytes; a submit that would exceed it is
// refused with ANYSEQ_ERR_BUDGET.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/anyseq.h"
#include "api_internal.h"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> q, s;
    int64_t t_submit = 0, t_done = 0;
    anyseq_result_t res{};
    anyseq_status_t status = ANYSEQ_OK;
    std::string error;  // the worker's message when status != ANYSEQ_OK
    bool done = false;
};

}  // namespace

// One service lane: a worker thread, its context, stream and queue.
struct ServeLane {
    anyseq_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::condition_variable cv_work;
    std::deque<Request *> queue;
};

struct anyseq_server {
    anyseq_server_config_t cfg{};
    std::vector<int8_t> matrix;  // copy of the scoring matrix
    anyseq_scoring_t sc{};
    ServeLane lane[2];           // 0: short pairs (batched kernel), 1: long pairs (wavefront)
    std::mutex mu;
    std::condition_variable cv_done;
    std::unordered_map<uint64_t, Request *> live;
    uint64_t next_ticket = 1;
    size_t held_bytes = 0;  // letters of queued and running requests
    bool stop = false;
    anyseq_status_t worker_status = ANYSEQ_OK;
    // statistics
    int64_t completed = 0, batches = 0, long_pairs = 0, rejected = 0;
    double busy_ms = 0;
};

namespace {

// A pair of at least long_cells cells that the wavefront takes.
bool is_long_pair(const anyseq_server *S, int64_t n, int64_t m) {
    const double cells = (double)n * (double)m;
    return cells >= (double)S->cfg.long_cells && n > 0 && m > 0 && S->sc.alphabet <= 4 && n < (1 << 21) &&
           m < (1 << 21) && anyseq::long_range_ok(&S->sc, n, m);
}

// Results of a finished batch: release its letters and wake the waiters.
void finish(anyseq_server *S, std::vector<Request *> &reqs, bool long_lane) {
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request *r : reqs) {
        r->done = true;
        S->held_bytes -= r->q.size() + r->s.size();
        r->q.clear();
        r->q.shrink_to_fit();
        r->s.clear();
        r->s.shrink_to_fit();
    }
    S->completed += (int64_t)reqs.size();
    if (long_lane) S->long_pairs += (int64_t)reqs.size();
    S->batches += 1;
    S->cv_done.notify_all();
}

void run_short(anyseq_server *S, std::vector<Request *> &small) {
    ServeLane &L = S->lane[0];
    std::vector<int64_t> qo(small.size() + 1, 0), so(small.size() + 1, 0);
    for (size_t k = 0; k < small.size(); k++) {
        qo[k + 1] = qo[k] + (int64_t)small[k]->q.size();
        so[k + 1] = so[k] + (int64_t)small[k]->s.size();
    }
    std::vector<uint8_t> q((size_t)qo.back() + 1), s((size_t)so.back() + 1);
    for (size_t k = 0; k < small.size(); k++) {
        if (!small[k]->q.empty()) memcpy(q.data() + qo[k], small[k]->q.data(), small[k]->q.size());
        if (!small[k]->s.empty()) memcpy(s.data() + so[k], small[k]->s.data(), small[k]->s.size());
    }
    std::vector<anyseq_result_t> out(small.size());
    uint64_t used = 0;
    const anyseq_status_t st =
        anyseq_align_batch(L.ctx, q.data(), qo.data(), s.data(), so.data(), (int64_t)small.size(), &S->sc,
                           S->cfg.mode, ANYSEQ_WANT_SCORE | ANYSEQ_WANT_END, out.data(), nullptr, 0, &used, L.stream);
    const std::string msg = st != ANYSEQ_OK ? anyseq_last_error() : "";
    const int64_t t = now_ns();
    for (size_t k = 0; k < small.size(); k++) {
        small[k]->res = out[k];
        small[k]->status = st;
        small[k]->error = msg;
        small[k]->t_done = t;
    }
    finish(S, small, false);
}

void run_long(anyseq_server *S, std::vector<Request *> &big) {
    // every long pair of the batch in one wavefront launch
    ServeLane &L = S->lane[1];
    std::vector<int64_t> qo(big.size() + 1, 0), so(big.size() + 1, 0);
    for (size_t k = 0; k < big.size(); k++) {
        qo[k + 1] = qo[k] + (int64_t)big[k]->q.size();
        so[k + 1] = so[k] + (int64_t)big[k]->s.size();
    }
    std::vector<uint8_t> q((size_t)qo.back()), s((size_t)so.back());
    for (size_t k = 0; k < big.size(); k++) {
        memcpy(q.data() + qo[k], big[k]->q.data(), big[k]->q.size());
        memcpy(s.data() + so[k], big[k]->s.data(), big[k]->s.size());
    }
    std::vector<int32_t> scores(big.size(), 0), eq(big.size(), 0), es(big.size(), 0);
    const anyseq_status_t st = anyseq::long_scores(L.ctx, q.data(), qo.data(), s.data(), so.data(),
                                                   (int64_t)big.size(), &S->sc, scores.data(), L.stream,
                                                   S->cfg.mode, eq.data(), es.data());
    const std::string msg = st != ANYSEQ_OK ? anyseq_last_error() : "";
    const int64_t t = now_ns();
    for (size_t k = 0; k < big.size(); k++) {
        Request *r = big[k];
        memset(&r->res, 0, sizeof(r->res));
        r->res.score = scores[k];
        r->res.beg_q = r->res.beg_s = -1;
        r->res.end_q = eq[k];
        r->res.end_s = es[k];
        r->res.flags = ANYSEQ_FLAG_INT32;
        r->status = st;
        r->error = msg;
        r->t_done = t;
    }
    finish(S, big, true);
}

void worker_main(anyseq_server *S, int which) {
    ServeLane &L = S->lane[which];
    if (cudaSetDevice(S->cfg.device) != cudaSuccess) {
        std::lock_guard<std::mutex> lock(S->mu);
        S->worker_status = ANYSEQ_ERR_CUDA;
        return;
    }
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            L.cv_work.wait(lock, [&] { return S->stop || !L.queue.empty(); });
            if (L.queue.empty()) break;  // stop requested and nothing left
            // batching window: until the oldest request has waited max_wait_us or the batch is full
            const int64_t deadline = L.queue.front()->t_submit + S->cfg.max_wait_us * 1000;
            while (!S->stop && (int64_t)L.queue.size() < S->cfg.max_batch_pairs) {
                const int64_t left = deadline - now_ns();
                if (left <= 0) break;
                L.cv_work.wait_for(lock, std::chrono::nanoseconds(left));
            }
            while (!L.queue.empty() && (int64_t)batch.size() < S->cfg.max_batch_pairs) {
                batch.push_back(L.queue.front());
                L.queue.pop_front();
            }
        }
        const int64_t t0 = now_ns();
        if (which == 0) run_short(S, batch);
        else run_long(S, batch);
        std::lock_guard<std::mutex> lock(S->mu);
        S->busy_ms += (double)(now_ns() - t0) * 1e-6;
    }
}

}  // namespace

extern "C" anyseq_status_t anyseq_server_create(anyseq_server **out, const anyseq_server_config_t *cfg) {
    if (!out || !cfg) return anyseq::fail(ANYSEQ_ERR_ARG, "server and config must not be NULL");
    *out = nullptr;
    const anyseq_status_t sc_st = anyseq::check_scoring(&cfg->scoring, cfg->mode);
    if (sc_st != ANYSEQ_OK) return sc_st;
    if (cfg->max_batch_pairs < 0 || cfg->max_wait_us < 0 || cfg->long_cells < 0)
        return anyseq::fail(ANYSEQ_ERR_ARG, "negative server limits");
    anyseq_server *S = new anyseq_server();
    S->cfg = *cfg;
    if (S->cfg.max_batch_pairs == 0) S->cfg.max_batch_pairs = 65536;
    if (S->cfg.max_wait_us == 0) S->cfg.max_wait_us = 200;
    if (S->cfg.long_cells == 0) S->cfg.long_cells = 1ll << 22;
    if (S->cfg.mem_budget_bytes == 0) S->cfg.mem_budget_bytes = (size_t)1 << 30;
    S->sc = cfg->scoring;
    if (cfg->scoring.matrix) {
        const int a = cfg->scoring.alphabet;
        S->matrix.assign(cfg->scoring.matrix, cfg->scoring.matrix + (size_t)a * a);
        S->sc.matrix = S->matrix.data();
    }
    for (int k = 0; k < 2; k++) {
        anyseq_status_t st = anyseq_create(&S->lane[k].ctx, cfg->device, 0);
        if (st == ANYSEQ_OK && (cudaSetDevice(cfg->device) != cudaSuccess ||
                                cudaStreamCreateWithFlags(&S->lane[k].stream, cudaStreamNonBlocking) != cudaSuccess)) {
            cudaGetLastError();
            st = anyseq::fail(ANYSEQ_ERR_CUDA, "could not create the server's streams");
        }
        if (st != ANYSEQ_OK) {
            for (int j = 0; j <= k; j++) {
                if (S->lane[j].stream) cudaStreamDestroy(S->lane[j].stream);
                if (S->lane[j].ctx) anyseq_destroy(S->lane[j].ctx);
            }
            delete S;
            return st;
        }
    }
    // Both lanes' persistent kernels must fit on every SM at once: a CTA that does
    // not fit waits for the other lane's persistent kernel to finish, and its own
    // launch ends only after it has run. The long lane's wavefront takes one CTA per
    // SM (8 warps, 32K registers). The short lane's batched kernel takes two (16K
    // registers each), and the wavefront launch it makes for a batch's larger pairs
    // one as well.
    anyseq_set_option(S->lane[1].ctx, "wave_ctas_per_sm", 1);
    anyseq_set_option(S->lane[0].ctx, "wave_ctas_per_sm", 1);
    anyseq_set_option(S->lane[0].ctx, "batch_ctas_per_sm", 2);
    for (int k = 0; k < 2; k++) S->lane[k].worker = std::thread(worker_main, S, k);
    *out = S;
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_server_submit(anyseq_server *S, const uint8_t *q, int64_t n, const uint8_t *s,
                                                int64_t m, uint64_t *ticket) {
    if (!S || !ticket) return anyseq::fail(ANYSEQ_ERR_ARG, "server and ticket must not be NULL");
    if (n < 0 || m < 0 || (n > 0 && !q) || (m > 0 && !s)) return anyseq::fail(ANYSEQ_ERR_ARG, "bad pair");
    if (n >= (1ll << 21) || m >= (1ll << 21)) return anyseq::fail(ANYSEQ_ERR_ARG, "pairs below 2^21 letters");
    if (S->cfg.mode != ANYSEQ_GLOBAL && !anyseq::key_range_ok(&S->sc, n < m ? n : m))
        return anyseq::fail(ANYSEQ_ERR_ARG, "local / semi-global scores of this pair may reach 2^21");
    Request *r = new Request();
    r->q.assign(q, q + n);
    r->s.assign(s, s + m);
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->worker_status != ANYSEQ_OK) {
        delete r;
        return anyseq::fail(S->worker_status, "the server's worker failed to start");
    }
    if (S->stop) {
        delete r;
        return anyseq::fail(ANYSEQ_ERR_ARG, "the server is shutting down");
    }
    const size_t bytes = (size_t)n + (size_t)m;
    if (S->held_bytes + bytes > S->cfg.mem_budget_bytes) {
        S->rejected += 1;
        delete r;
        return anyseq::fail(ANYSEQ_ERR_BUDGET, "request of %zu letters exceeds the server's budget (%zu held of %zu)",
                            bytes, S->held_bytes, S->cfg.mem_budget_bytes);
    }
    S->held_bytes += bytes;
    r->ticket = S->next_ticket++;
    r->t_submit = now_ns();
    S->live[r->ticket] = r;
    ServeLane &L = S->lane[is_long_pair(S, n, m) ? 1 : 0];
    L.queue.push_back(r);
    *ticket = r->ticket;
    L.cv_work.notify_one();
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_server_wait(anyseq_server *S, uint64_t ticket, int64_t timeout_us,
                                              anyseq_result_t *out, int64_t *latency_ns) {
    if (!S || !out) return anyseq::fail(ANYSEQ_ERR_ARG, "server and out must not be NULL");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return anyseq::fail(ANYSEQ_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0) {
        S->cv_done.wait(lock, ready);
    } else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
        return anyseq::fail(ANYSEQ_ERR_TIMEOUT, "ticket %llu not finished within %lld us", (unsigned long long)ticket,
                            (long long)timeout_us);
    }
    *out = r->res;
    if (latency_ns) *latency_ns = r->t_done - r->t_submit;
    const anyseq_status_t st = r->status;
    const std::string msg = r->error;
    S->live.erase(it);
    delete r;
    if (st != ANYSEQ_OK) return anyseq::fail(st, "%s", msg.c_str());
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_server_stat(anyseq_server *S, const char *key, double *value) {
    if (!S || !key || !value) return anyseq::fail(ANYSEQ_ERR_ARG, "server, key and value must not be NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    if (!strcmp(key, "completed")) *value = (double)S->completed;
    else if (!strcmp(key, "batches")) *value = (double)S->batches;
    else if (!strcmp(key, "long_pairs")) *value = (double)S->long_pairs;
    else if (!strcmp(key, "rejected")) *value = (double)S->rejected;
    else if (!strcmp(key, "queued")) *value = (double)(S->lane[0].queue.size() + S->lane[1].queue.size());
    else if (!strcmp(key, "held_bytes")) *value = (double)S->held_bytes;
    else if (!strcmp(key, "busy_ms")) *value = S->busy_ms;
    else return anyseq::fail(ANYSEQ_ERR_ARG, "unknown server statistic '%s'", key);
    return ANYSEQ_OK;
}

extern "C" anyseq_status_t anyseq_server_destroy(anyseq_server *S) {
    if (!S) return ANYSEQ_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        for (auto &L : S->lane) L.cv_work.notify_all();
    }
    for (auto &L : S->lane)
        if (L.worker.joinable()) L.worker.join();
    for (auto &kv : S->live) delete kv.second;
    anyseq_status_t st = ANYSEQ_OK;
    for (auto &L : S->lane) {
        if (L.stream) cudaStreamDestroy(L.stream);
        const anyseq_status_t d = anyseq_destroy(L.ctx);
        if (st == ANYSEQ_OK) st = d;
    }
    delete S;
    return st;
}
