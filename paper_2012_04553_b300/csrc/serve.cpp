// Serving loop: continuous batching of pattern-count requests against
// device-resident graphs.
//
// Requests (a graph and 1..n query patterns) are queued per graph.  Each
// graph has `workers_per_graph` worker threads, each with its own CUDA
// stream; a free worker takes every request queued for its graph (up to
// `max_batch_patterns` patterns), so requests that arrive while earlier
// batches are on the GPU join the next batch as soon as a worker and device
// memory are free, and batches of different graphs (and of the same graph on
// different workers) run concurrently on the device.  A batch is one pm_plan
// over the concatenated queries: morph selection deduplicates the matched
// (morphed) patterns shared by the batch's requests, and every request reads
// its own slice of the batch's counts.  Each matched pattern of a batch has
// its own deadline (pm_count_each), so a pattern that runs out of time fails
// only the requests whose queries need it.  A request queued longer than
// request_timeout_s is completed unrun with PM_ETIMEOUT (load shedding), and
// a batch's total deadline never outlasts its oldest request's.  Admission reserves an estimate of the
// batch's device memory against `hbm_budget_bytes`; a batch waits until the
// estimate fits.  Latency is measured from submission to completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "internal.hpp"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int graph = 0;
    std::vector<pm_pattern> queries;
    Clock::time_point submitted, finished;
    std::vector<uint64_t> counts;   // 2 words per query
    std::vector<int32_t> qstatus;   // per query
    pm_status status = PM_OK;
    bool done = false;
    int32_t matched_alone = 0;      // matched patterns if planned by itself
};

}  // namespace

struct pm_server {
    std::vector<const pm_graph *> graphs;
    pm_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::deque<uint64_t>> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<std::thread> workers;
    uint64_t next_id = 1;
    int64_t reserved = 0;
    bool stop = false;
    pm_server_stats stats{};
};

namespace {

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

// Device memory a batch may use: plan buffers, the deferral list (at most
// 2^26 entries of 12 bytes) and the 4-cycle wedge counters (one n-word array
// per SM).
int64_t batch_estimate(const pm_graph *g) {
    const int sms = pm::device_sm_count(g->device);
    return (int64_t(16) << 20) + (int64_t(12) << 26) + int64_t(4) * g->n * std::max(sms, 1);
}

void worker_loop(pm_server *s, int graph) {
    const pm_graph *g = s->graphs[graph];
    cudaSetDevice(g->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    const int64_t est = batch_estimate(g);
    for (;;) {
        std::vector<uint64_t> batch;
        Clock::time_point oldest{};
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->pending[graph].empty() &&
                                   (s->reserved == 0 || s->reserved + est <= s->cfg.hbm_budget_bytes));
            });
            if (s->stop) break;
            int npat = 0;
            bool shed = false;
            const auto now = Clock::now();
            while (!s->pending[graph].empty()) {
                const uint64_t id = s->pending[graph].front();
                Request &r = s->reqs[id];
                if (s->cfg.request_timeout_s > 0 && seconds(now - r.submitted) > s->cfg.request_timeout_s) {
                    // queued past its deadline: completed unrun
                    s->pending[graph].pop_front();
                    r.status = PM_ETIMEOUT;
                    r.counts.assign(2 * r.queries.size(), 0);
                    r.qstatus.assign(r.queries.size(), PM_ETIMEOUT);
                    r.finished = now;
                    r.done = true;
                    s->stats.matched_alone += r.matched_alone;
                    s->stats.timeouts++;
                    s->stats.shed++;
                    s->stats.requests_done++;
                    shed = true;
                    continue;
                }
                const int nq = int(r.queries.size());
                if (!batch.empty() && npat + nq > s->cfg.max_batch_patterns) break;
                if (batch.empty()) oldest = r.submitted;
                batch.push_back(id);
                npat += nq;
                s->pending[graph].pop_front();
            }
            if (shed) s->cv_done.notify_all();
            if (batch.empty()) continue;
            s->reserved += est;
        }
        // one plan for the whole batch
        std::vector<pm_pattern> all;
        std::vector<size_t> first;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint64_t id : batch) {
                first.push_back(all.size());
                const Request &r = s->reqs[id];
                all.insert(all.end(), r.queries.begin(), r.queries.end());
            }
        }
        std::vector<uint64_t> counts(2 * all.size(), 0);
        std::vector<int32_t> qstatus(all.size(), PM_OK);
        pm_query_plan *plan = nullptr;
        pm_status st = pm_plan(g, all.data(), int32_t(all.size()), PM_OP_COUNT,
                               pm_morph_mode(s->cfg.mode), &plan);
        int32_t matched = 0;
        if (st == PM_OK) {
            pm_plan_info info;
            pm_plan_get_info(plan, &info);
            matched = info.n_matched;
            pm_plan_select(plan, s->cfg.family);
            // a deadline per matched pattern: a heavy pattern fails only the
            // requests that need it
            double total = s->cfg.batch_total_s;
            if (s->cfg.request_timeout_s > 0) {
                // no longer than the oldest request has left
                const double left = std::max(0.05, s->cfg.request_timeout_s - seconds(Clock::now() - oldest));
                total = total > 0 ? std::min(total, left) : left;
            }
            st = pm_count_each(plan, stream, s->cfg.batch_timeout_s, total, counts.data(), qstatus.data());
            pm_free_plan(plan);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const auto now = Clock::now();
            for (size_t b = 0; b < batch.size(); b++) {
                Request &r = s->reqs[batch[b]];
                r.status = st;
                r.qstatus.assign(r.queries.size(), int32_t(st));
                if (st == PM_OK)
                    for (size_t qi = 0; qi < r.queries.size(); qi++) {
                        r.qstatus[qi] = qstatus[first[b] + qi];
                        if (qstatus[first[b] + qi] != PM_OK) r.status = pm_status(qstatus[first[b] + qi]);
                    }
                r.counts.assign(counts.begin() + 2 * first[b],
                                counts.begin() + 2 * (first[b] + r.queries.size()));
                r.finished = now;
                r.done = true;
                s->stats.matched_alone += r.matched_alone;
                if (r.status == PM_ETIMEOUT) s->stats.timeouts++;
                else if (r.status != PM_OK) s->stats.failures++;
            }
            s->stats.batches++;
            s->stats.requests_done += int64_t(batch.size());
            s->stats.patterns_done += int64_t(all.size());
            s->stats.matched_batched += matched;
            s->reserved -= est;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

pm_status pm_server_create(const pm_graph *const *graphs, int32_t n_graphs,
                           const pm_server_config *cfg, pm_server **out) {
    if (!graphs || n_graphs < 1 || !cfg || !out || cfg->workers_per_graph < 1 ||
        cfg->max_batch_patterns < 1 || cfg->hbm_budget_bytes <= 0) {
        pm::set_error("pm_server_create: bad argument");
        return PM_EINVAL;
    }
    for (int i = 0; i < n_graphs; i++)
        if (!graphs[i]) return PM_EINVAL;
    auto *s = new (std::nothrow) pm_server();
    if (!s) return PM_ENOMEM;
    s->graphs.assign(graphs, graphs + n_graphs);
    s->cfg = *cfg;
    s->pending.resize(n_graphs);
    for (int gi = 0; gi < n_graphs; gi++)
        for (int w = 0; w < cfg->workers_per_graph; w++) s->workers.emplace_back(worker_loop, s, gi);
    *out = s;
    return PM_OK;
}

pm_status pm_server_submit(pm_server *s, int32_t graph, const pm_pattern *queries, int32_t nq,
                           uint64_t *id) {
    if (!s || !queries || nq < 1 || !id || graph < 0 || graph >= int32_t(s->graphs.size())) {
        pm::set_error("pm_server_submit: bad argument");
        return PM_EINVAL;
    }
    // reject malformed patterns now rather than failing the whole batch later
    // validation and the request's own alternative-set size (no plan compilation)
    int32_t matched_alone = 0;
    pm_status st = pm::matched_set_size(s->graphs[graph], queries, nq, pm_morph_mode(s->cfg.mode),
                                        &matched_alone);
    if (st != PM_OK) return st;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const uint64_t rid = s->next_id++;
        Request &r = s->reqs[rid];
        r.graph = graph;
        r.queries.assign(queries, queries + nq);
        r.submitted = Clock::now();
        r.matched_alone = matched_alone;
        s->pending[graph].push_back(rid);
        s->stats.requests_submitted++;
        *id = rid;
    }
    s->cv_work.notify_all();
    return PM_OK;
}

pm_status pm_server_wait(pm_server *s, uint64_t id, double timeout_s, int32_t *done,
                         uint64_t *counts, double *latency_s, pm_status *request_status,
                         int32_t *query_status) {
    if (!s || !done) return PM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        pm::set_error("pm_server_wait: unknown request id");
        return PM_EINVAL;
    }
    auto ready = [&] { return s->reqs[id].done; };
    if (timeout_s > 0) s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    else if (timeout_s < 0) s->cv_done.wait(lk, ready);
    Request &r = s->reqs[id];
    *done = r.done ? 1 : 0;
    if (!r.done) return PM_OK;
    if (counts) std::copy(r.counts.begin(), r.counts.end(), counts);
    if (latency_s) *latency_s = seconds(r.finished - r.submitted);
    if (request_status) *request_status = r.status;
    if (query_status) std::copy(r.qstatus.begin(), r.qstatus.end(), query_status);
    s->reqs.erase(id);
    return PM_OK;
}

pm_status pm_server_get_stats(pm_server *s, pm_server_stats *out) {
    if (!s || !out) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return PM_OK;
}

void pm_server_destroy(pm_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
}

}  // extern "C"
