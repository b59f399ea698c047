// Serving loop over resident indexes with continuous batching.
//
// Requests (one query each: host tokens, an index, a k) are queued as they
// are submitted.  One worker thread owns the device side:
//   - it keeps up to max_inflight batches on the device at once, each on a
//     stream and workspace of its own (a "slot"), so batches overlap;
//   - whenever a slot is free and requests are waiting, it takes the oldest
//     waiting request's index and batches that index's waiting requests (up
//     to max_batch, in arrival order), admitting the batch only if the
//     slot's scratch for it (accumulators, tile candidates, dense vectors)
//     keeps all slots within memory_budget, else a smaller batch or, with
//     nothing to shrink, after a running batch completes;
//   - each batch is one bm25_retrieve_batch call (per-query k, rows k_max
//     wide) between a host-to-device copy of its queries and a device-to-host
//     copy of its results, all stream-ordered from pinned staging buffers;
//   - completed batches (polled with cudaEventQuery) hand each request its
//     row, so requests that arrived while others ran are admitted as soon as
//     a slot frees up.
// Batching changes no result beyond the order of FP32 additions: a query's
// top k is computed from its own columns only, whatever else is in its batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    int32_t index = 0;
    std::vector<int32_t> tokens;
    int32_t k = 0;
    Clock::time_point t_submit;
    std::vector<int32_t> ids;
    std::vector<float> scores;
    int status = BM25_PENDING;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bm25_workspace ws;
    // pinned host and device staging, grown on demand
    int32_t* h_tok = nullptr;
    int64_t* h_off = nullptr;
    int32_t* h_k = nullptr;
    int32_t* h_ids = nullptr;
    float* h_scores = nullptr;
    int32_t* d_tok = nullptr;
    int64_t* d_off = nullptr;
    int32_t* d_k = nullptr;
    int32_t* d_ids = nullptr;
    float* d_scores = nullptr;
    size_t cap_tok = 0, cap_q = 0, cap_out = 0;  // elements
    std::vector<std::shared_ptr<Request>> reqs;
    int32_t kmax = 0;
    bool busy = false;
};

}  // namespace

struct bm25_server {
    std::vector<const bm25_index*> indexes;
    bm25_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::deque<std::shared_ptr<Request>>> queues;
    std::unordered_map<int64_t, std::shared_ptr<Request>> tickets;
    int64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    // statistics since the last reset
    int64_t completed = 0, failed = 0, batches = 0, batched_queries = 0;
    std::vector<double> latency_us;
    bool any_submit = false, any_done = false;
    Clock::time_point first_submit, last_done;
};

using namespace bm25;

namespace {

size_t slot_bytes(const Slot& s)
{
    return workspace_bytes_held(&s.ws) +
           s.cap_tok * sizeof(int32_t) + s.cap_q * (sizeof(int64_t) + sizeof(int32_t)) +
           s.cap_out * (sizeof(int32_t) + sizeof(float));
}

template <typename T>
int grow_pair(T** h, T** d, size_t* cap, size_t need)
{
    if (need <= *cap && *h && *d)
        return BM25_OK;
    if (*h)
        cudaFreeHost(*h);
    if (*d)
        cudaFree(*d);
    *h = nullptr;
    *d = nullptr;
    *cap = 0;
    const size_t n = std::max<size_t>(need, 1);
    BM25_CUDA_TRY(cudaMallocHost((void**)h, n * sizeof(T)));
    BM25_CUDA_TRY(cudaMalloc((void**)d, n * sizeof(T)));
    *cap = n;
    return BM25_OK;
}

int slot_staging(Slot& s, size_t n_tok, size_t nq, size_t n_out)
{
    size_t ct = s.cap_tok, cq = s.cap_q, cq2 = s.cap_q, co = s.cap_out, co2 = s.cap_out;
    BM25_TRY(grow_pair(&s.h_tok, &s.d_tok, &ct, n_tok));
    BM25_TRY(grow_pair(&s.h_off, &s.d_off, &cq, nq + 1));
    BM25_TRY(grow_pair(&s.h_k, &s.d_k, &cq2, nq + 1));
    BM25_TRY(grow_pair(&s.h_ids, &s.d_ids, &co, n_out));
    BM25_TRY(grow_pair(&s.h_scores, &s.d_scores, &co2, n_out));
    s.cap_tok = ct;
    s.cap_q = std::min(cq, cq2);
    s.cap_out = std::min(co, co2);
    return BM25_OK;
}

void slot_free(Slot& s)
{
    if (s.stream)
        cudaStreamSynchronize(s.stream);
    workspace_release(&s.ws);
    for (void* p : {(void*)s.h_tok, (void*)s.h_off, (void*)s.h_k, (void*)s.h_ids,
                    (void*)s.h_scores})
        if (p)
            cudaFreeHost(p);
    for (void* p : {(void*)s.d_tok, (void*)s.d_off, (void*)s.d_k, (void*)s.d_ids,
                    (void*)s.d_scores})
        if (p)
            cudaFree(p);
    if (s.done)
        cudaEventDestroy(s.done);
    if (s.stream)
        cudaStreamDestroy(s.stream);
    s = Slot();
}

Plan plan_of_index(const bm25_index* ix)
{
    std::lock_guard<std::mutex> g(const_cast<bm25_index*>(ix)->mu);
    return ix->plan;
}

// Finishes a completed slot's batch (lock held).
void complete(bm25_server* sv, Slot& s, int rc)
{
    const auto now = Clock::now();
    for (size_t i = 0; i < s.reqs.size(); i++) {
        Request& r = *s.reqs[i];
        if (rc == BM25_OK) {
            r.ids.assign(s.h_ids + i * s.kmax, s.h_ids + i * s.kmax + r.k);
            r.scores.assign(s.h_scores + i * s.kmax, s.h_scores + i * s.kmax + r.k);
            r.status = BM25_OK;
            sv->completed++;
            sv->latency_us.push_back(
                std::chrono::duration<double, std::micro>(now - r.t_submit).count());
            sv->any_done = true;
            sv->last_done = now;
        } else {
            r.status = rc;
            sv->failed++;
        }
    }
    s.reqs.clear();
    s.busy = false;
}

// Launches one batch on a free slot (lock held; the launches are
// asynchronous).  Returns the number of requests taken from the queue (0:
// not admitted now).
int dispatch(bm25_server* sv, Slot& s, int32_t qi, std::deque<std::shared_ptr<Request>>& q,
             bool others_busy)
{
    const bm25_index* ix = sv->indexes[qi];
    const Plan plan = plan_of_index(ix);
    size_t held_others = 0;
    for (const Slot& o : sv->slots)
        if (&o != &s)
            held_others += slot_bytes(o);
    int32_t nb = (int32_t)std::min<size_t>(q.size(), (size_t)sv->cfg.max_batch_queries);
    int32_t kmax = 1;
    int64_t n_tok = 0;
    size_t need = 0;
    for (;;) {  // the largest prefix of the queue that fits the budget
        kmax = 1;
        n_tok = 0;
        for (int32_t i = 0; i < nb; i++) {
            kmax = std::max(kmax, q[i]->k);
            n_tok += (int64_t)q[i]->tokens.size();
        }
        size_t ws_bytes = 0;
        BM25_TRY(workspace_bytes_for(ix, nb, n_tok, kmax, plan, &ws_bytes));
        need = std::max(ws_bytes, workspace_bytes_held(&s.ws)) +
               (size_t)n_tok * 4 + (size_t)(nb + 1) * 12 + (size_t)nb * kmax * 8;
        if (held_others + need <= (size_t)sv->cfg.memory_budget || nb == 1)
            break;
        nb = std::max(1, nb / 2);
    }
    if (held_others + need > (size_t)sv->cfg.memory_budget) {
        // idle slots give their scratch back first (this one included)
        held_others = 0;
        for (Slot& o : sv->slots) {
            if (!o.busy) {
                workspace_release(&o.ws);
                o.ws.device = sv->device;
            }
            if (&o != &s)
                held_others += slot_bytes(o);
        }
        size_t ws_bytes = 0;
        BM25_TRY(workspace_bytes_for(ix, nb, n_tok, kmax, plan, &ws_bytes));
        need = ws_bytes + (size_t)n_tok * 4 + (size_t)(nb + 1) * 12 + (size_t)nb * kmax * 8;
        if (held_others + need > (size_t)sv->cfg.memory_budget) {
            if (others_busy)
                return 0;  // wait for a running batch to free its scratch
            std::shared_ptr<Request> r = q.front();
            q.pop_front();
            r->status = set_error(BM25_E_OOM, "a single query needs more scratch than the "
                                              "server's memory budget");
            sv->failed++;
            return 1;
        }
    }
    BM25_TRY(slot_staging(s, (size_t)n_tok, (size_t)nb, (size_t)nb * kmax));
    s.reqs.assign(q.begin(), q.begin() + nb);
    q.erase(q.begin(), q.begin() + nb);
    int64_t o = 0;
    for (int32_t i = 0; i < nb; i++) {
        const Request& r = *s.reqs[i];
        s.h_off[i] = o;
        s.h_k[i] = r.k;
        std::copy(r.tokens.begin(), r.tokens.end(), s.h_tok + o);
        o += (int64_t)r.tokens.size();
    }
    s.h_off[nb] = o;
    s.kmax = kmax;
    cudaStream_t st = s.stream;
    int rc = BM25_OK;
    if (n_tok > 0 && cudaMemcpyAsync(s.d_tok, s.h_tok, sizeof(int32_t) * n_tok,
                                     cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "query copy failed");
    if (rc == BM25_OK &&
        (cudaMemcpyAsync(s.d_off, s.h_off, sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                         st) != cudaSuccess ||
         cudaMemcpyAsync(s.d_k, s.h_k, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st) !=
             cudaSuccess))
        rc = set_error(BM25_E_CUDA, "query copy failed");
    if (rc == BM25_OK)
        rc = retrieve_device(ix, &s.ws, s.d_tok, s.d_off, nb, n_tok, s.d_k, kmax, s.d_ids,
                             s.d_scores, plan, st);
    if (rc == BM25_OK &&
        (cudaMemcpyAsync(s.h_ids, s.d_ids, sizeof(int32_t) * nb * kmax, cudaMemcpyDeviceToHost,
                         st) != cudaSuccess ||
         cudaMemcpyAsync(s.h_scores, s.d_scores, sizeof(float) * nb * kmax,
                         cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = set_error(BM25_E_CUDA, "result copy failed");
    if (rc == BM25_OK && cudaEventRecord(s.done, st) != cudaSuccess)
        rc = set_error(BM25_E_CUDA, "event record failed");
    sv->batches++;
    sv->batched_queries += nb;
    if (rc != BM25_OK) {
        cudaStreamSynchronize(st);
        complete(sv, s, rc);
        return nb;
    }
    s.busy = true;
    return nb;
}

void worker_main(bm25_server* sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // completions
        bool any_busy = false;
        for (Slot& s : sv->slots) {
            if (!s.busy)
                continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) {
                complete(sv, s, BM25_OK);
                sv->cv_done.notify_all();
            } else if (e != cudaErrorNotReady) {
                complete(sv, s, set_error(BM25_E_CUDA, "batch failed: %s", cudaGetErrorString(e)));
                sv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (sv->stop && !any_busy)
            break;
        // dispatch: oldest waiting request first
        bool progressed = false;
        while (!sv->stop) {
            Slot* free_slot = nullptr;
            for (Slot& s : sv->slots)
                if (!s.busy) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot)
                break;
            int32_t qi = -1;
            for (int32_t i = 0; i < (int32_t)sv->queues.size(); i++)
                if (!sv->queues[i].empty() &&
                    (qi < 0 || sv->queues[i].front()->ticket < sv->queues[qi].front()->ticket))
                    qi = i;
            if (qi < 0)
                break;
            bool others = false;
            for (Slot& s : sv->slots)
                others |= s.busy;
            const int taken = dispatch(sv, *free_slot, qi, sv->queues[qi], others);
            if (taken < 0) {  // failed before taking requests: fail the oldest one
                std::shared_ptr<Request> r = sv->queues[qi].front();
                sv->queues[qi].pop_front();
                r->status = taken;
                sv->failed++;
                sv->cv_done.notify_all();
                progressed = true;
                continue;
            }
            if (taken == 0)
                break;
            progressed = true;
            any_busy |= free_slot->busy;
            if (!free_slot->busy)
                sv->cv_done.notify_all();  // failed without running
        }
        if (sv->stop && !any_busy)
            break;
        if (!any_busy && !progressed) {
            bool waiting = false;
            for (auto& q : sv->queues)
                waiting |= !q.empty();
            if (!waiting)
                sv->cv_work.wait(lk);  // idle until a submit or destroy
        } else if (any_busy) {
            // a batch is running: look again shortly (a submit wakes us earlier)
            sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
    // fail whatever is still queued
    for (auto& q : sv->queues)
        for (auto& r : q) {
            r->status = BM25_E_INVALID;
            sv->failed++;
        }
    for (auto& q : sv->queues)
        q.clear();
    sv->cv_done.notify_all();
}

}  // namespace

extern "C" {

int bm25_server_create(const bm25_index* const* indexes, int32_t n_indexes,
                       const bm25_server_config* cfg, bm25_server** out)
{
    clear_error();
    if (!out || !indexes || n_indexes < 1)
        return set_error(BM25_E_INVALID, "need at least one index");
    *out = nullptr;
    bm25_server_config c;
    c.max_batch_queries = 2048;
    c.max_inflight = 3;
    c.k_max = 1000;
    c.reserved = 0;
    c.memory_budget = int64_t(4) << 30;
    if (cfg) {
        if (cfg->max_batch_queries) c.max_batch_queries = cfg->max_batch_queries;
        if (cfg->max_inflight) c.max_inflight = cfg->max_inflight;
        if (cfg->k_max) c.k_max = cfg->k_max;
        if (cfg->memory_budget) c.memory_budget = cfg->memory_budget;
    }
    if (c.max_batch_queries < 1 || c.max_inflight < 1 || c.max_inflight > 16 || c.k_max < 1 ||
        c.k_max > BM25_MAX_K || c.memory_budget < 1)
        return set_error(BM25_E_INVALID, "bad server configuration");
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    for (int32_t i = 0; i < n_indexes; i++)
        if (!indexes[i] || indexes[i]->device != dev)
            return set_error(BM25_E_INVALID, "index %d is NULL or on another device", i);
    bm25_server* sv = new bm25_server();
    sv->indexes.assign(indexes, indexes + n_indexes);
    sv->cfg = c;
    sv->device = dev;
    sv->queues.resize(n_indexes);
    sv->slots.resize(c.max_inflight);
    int rc = BM25_OK;
    for (Slot& s : sv->slots) {
        s.ws.device = dev;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            rc = set_error(BM25_E_CUDA, "stream / event creation failed");
            break;
        }
    }
    if (rc != BM25_OK) {
        for (Slot& s : sv->slots)
            slot_free(s);
        delete sv;
        return rc;
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return BM25_OK;
}

int bm25_server_submit(bm25_server* sv, int32_t index_id, const int32_t* tokens,
                       int32_t n_tokens, int32_t k, int64_t* ticket)
{
    clear_error();
    if (!sv || !ticket || n_tokens < 0 || (n_tokens > 0 && !tokens))
        return set_error(BM25_E_INVALID, "bad argument");
    if (index_id < 0 || index_id >= (int32_t)sv->indexes.size())
        return set_error(BM25_E_INVALID, "index id %d out of range", index_id);
    if (k < 1 || k > sv->cfg.k_max)
        return set_error(BM25_E_INVALID, "k = %d outside [1, %d]", k, sv->cfg.k_max);
    const int32_t vocab = sv->indexes[index_id]->vocab;
    for (int32_t i = 0; i < n_tokens; i++)
        if (tokens[i] < 0 || tokens[i] >= vocab)
            return set_error(BM25_E_TOKEN_RANGE, "token %d outside [0, %d)", tokens[i], vocab);
    auto r = std::make_shared<Request>();
    r->index = index_id;
    r->tokens.assign(tokens, tokens + n_tokens);
    r->k = k;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->stop)
            return set_error(BM25_E_INVALID, "server is shutting down");
        r->ticket = sv->next_ticket++;
        r->t_submit = Clock::now();
        if (!sv->any_submit) {
            sv->any_submit = true;
            sv->first_submit = r->t_submit;
        }
        sv->tickets[r->ticket] = r;
        sv->queues[index_id].push_back(r);
        *ticket = r->ticket;
    }
    sv->cv_work.notify_one();
    return BM25_OK;
}

int bm25_server_replay(bm25_server* sv, int32_t n, const int32_t* index_ids,
                       const int32_t* tokens, const int64_t* offsets, const int32_t* ks,
                       const double* arrival_s, int64_t* tickets)
{
    clear_error();
    if (!sv || n < 0 || (n > 0 && (!index_ids || !offsets || !ks || !arrival_s || !tickets)))
        return set_error(BM25_E_INVALID, "bad argument");
    const auto t0 = Clock::now();
    for (int32_t i = 0; i < n; i++) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                  std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        const int64_t a = offsets[i], b = offsets[i + 1];
        BM25_TRY(bm25_server_submit(sv, index_ids[i], tokens ? tokens + a : nullptr,
                                    (int32_t)(b - a), ks[i], &tickets[i]));
    }
    return BM25_OK;
}

int bm25_replay_plain(const bm25_index* const* indexes, int32_t n_indexes, int32_t n,
                      const int32_t* index_ids, const int32_t* tokens, const int64_t* offsets,
                      const int32_t* ks, const double* arrival_s, double* latency_us,
                      void* cuda_stream)
{
    clear_error();
    if (!indexes || n_indexes < 1 || n < 0 ||
        (n > 0 && (!index_ids || !offsets || !ks || !arrival_s || !latency_us)))
        return set_error(BM25_E_INVALID, "bad argument");
    int32_t kmax = 1;
    for (int32_t i = 0; i < n; i++)
        kmax = std::max(kmax, ks[i]);
    std::vector<int32_t> ids((size_t)kmax);
    std::vector<float> scores((size_t)kmax);
    const auto t0 = Clock::now();
    for (int32_t i = 0; i < n; i++) {
        if (index_ids[i] < 0 || index_ids[i] >= n_indexes)
            return set_error(BM25_E_INVALID, "index id %d out of range", index_ids[i]);
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                  std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        const int64_t off[2] = {0, offsets[i + 1] - offsets[i]};
        BM25_TRY(bm25_retrieve_host(indexes[index_ids[i]], tokens ? tokens + offsets[i] : nullptr,
                                    off, 1, ks[i], ids.data(), scores.data(), cuda_stream));
        latency_us[i] = std::chrono::duration<double, std::micro>(Clock::now() - due).count();
    }
    return BM25_OK;
}

int bm25_server_poll(bm25_server* sv, int64_t ticket, int32_t* ids, float* scores,
                     int32_t timeout_us)
{
    clear_error();
    if (!sv)
        return set_error(BM25_E_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end())
        return set_error(BM25_E_INVALID, "unknown ticket %lld", (long long)ticket);
    std::shared_ptr<Request> r = it->second;
    if (r->status == BM25_PENDING && timeout_us != 0) {
        auto pred = [&] { return r->status != BM25_PENDING; };
        if (timeout_us < 0)
            sv->cv_done.wait(lk, pred);
        else
            sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    }
    if (r->status == BM25_PENDING)
        return BM25_PENDING;
    sv->tickets.erase(ticket);
    if (r->status != BM25_OK)
        return set_error(r->status, "request failed");
    if (ids)
        std::copy(r->ids.begin(), r->ids.end(), ids);
    if (scores)
        std::copy(r->scores.begin(), r->scores.end(), scores);
    return BM25_OK;
}

int bm25_server_stats_get(bm25_server* sv, int reset, bm25_server_stats* out)
{
    clear_error();
    if (!sv || !out)
        return set_error(BM25_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> g(sv->mu);
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->batches = sv->batches;
    out->batched_queries = sv->batched_queries;
    std::vector<double> l = sv->latency_us;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (double)(l.size() - 1) + 0.5))];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = l.empty() ? 0.0 : l.back();
    size_t held = 0;
    for (const Slot& s : sv->slots)
        held += slot_bytes(s);
    out->bytes_held = (int64_t)held;
    out->span_us = (sv->any_submit && sv->any_done && sv->last_done > sv->first_submit)
                       ? std::chrono::duration<double, std::micro>(sv->last_done -
                                                                   sv->first_submit).count()
                       : 0.0;
    if (reset) {
        sv->completed = sv->failed = sv->batches = sv->batched_queries = 0;
        sv->latency_us.clear();
        sv->any_submit = sv->any_done = false;
    }
    return BM25_OK;
}

void bm25_server_destroy(bm25_server* sv)
{
    if (!sv)
        return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable())
        sv->worker.join();
    for (Slot& s : sv->slots)
        slot_free(s);
    delete sv;
}

}  // extern "C"
