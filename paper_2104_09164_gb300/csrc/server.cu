// server.cu -- continuous-batching server for encrypted inference requests.
//
// Requests (ciphertexts of the end-user, coefficient domain, host memory) arrive at any
// time.  hear_server_submit copies them once, straight into pinned staging buffers that
// the server owns (checking every residue on the way), so the batch upload reads pinned
// memory; a full staging arena or queue refuses the request with HEAR_E_BUSY.  A worker
// thread admits pending requests in arrival order while the ciphertexts in flight fit the
// HBM budget, packs up to max_batch ciphertexts into one batch and runs it on a free slot:
// each slot owns a CUDA stream and device buffers, so up to n_slots batches overlap on the
// device (copies of one batch overlap the evaluation of another).  A batch is split into
// power-of-two sub-batches, each the replay of a captured CUDA graph of the whole network.
// Results are copied by the device into pinned result buffers, and from there once into
// the caller's array by hear_server_poll / hear_server_wait.  The evaluation keys and the
// encoded model stay resident.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include "ckks.h"

namespace hear {
void set_last_error(const std::string &msg);
}  // namespace hear

using namespace hear;
using Clock = std::chrono::steady_clock;

namespace {

// pinned host buffers of `words` words each, handed out by index
struct Arena {
    uint64_t *base = nullptr;
    uint64_t words = 0;
    std::vector<uint32_t> free;
    uint64_t *at(uint32_t i) const { return base + (uint64_t)i * words; }
};

struct Request {
    uint64_t id = 0;
    uint32_t n_ct = 0, n_clips = 0;
    double scale = 0;
    std::vector<uint32_t> in_bufs, out_bufs;   // staging buffers (one per ciphertext)
    Clock::time_point t_submit, t_done;
    int state = 0;                    // 0 pending, 1 running, 2 done, 3 failed
    hear_status status = HEAR_OK;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<std::shared_ptr<Request>> reqs;
    uint32_t n_ct = 0;
    bool busy = false;
};

}  // namespace

struct hear_server {
    const hear_model *m = nullptr;
    const hear_eval_keys *evk = nullptr;
    hear_server_config cfg{};
    uint32_t lin = 0, lout = 0;
    uint64_t in_words = 0, out_words = 0;  // per ciphertext
    uint64_t ct_bytes = 0;                  // device bytes charged per in-flight ciphertext
    std::mutex mu;
    std::condition_variable cv;            // worker: new work or a finished slot
    std::condition_variable cv_done;       // waiters: a request finished or failed
    std::deque<std::shared_ptr<Request>> pending;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::vector<Slot> slots;
    Arena in_arena, out_arena;
    uint64_t next_id = 1, in_flight_cts = 0, max_in_flight_cts = 0;
    uint64_t done_reqs = 0, done_cts = 0, done_clips = 0, batches = 0, busy_refusals = 0;
    std::vector<double> lat_ms;
    bool stop = false, paused = false;
    hear_status fault = HEAR_OK;
    std::string fault_msg;
    std::thread worker;
};

namespace {

// run the batch of slot s on its stream: the ciphertexts, in request order, go in power-of-
// two sub-batches through captured graphs that take and give the coefficient domain (the
// NTT conversions are graph nodes); each sub-batch is uploaded from the requests' pinned
// staging buffers straight into the graph's input and downloaded from its output into their
// pinned result buffers
void launch(hear_server *S, Slot &s, uint32_t slot_index) {
    const hear_model *m = S->m;
    std::vector<std::pair<uint32_t, uint32_t>> io;      // (staging buffer, result buffer) per ciphertext
    for (auto &r : s.reqs)
        for (size_t i = 0; i < r->in_bufs.size(); i++) io.emplace_back(r->in_bufs[i], r->out_bufs[i]);
    uint32_t done = 0;
    for (uint32_t b = 1u << 31; b; b >>= 1) {
        while (S->cfg.max_batch >= b && s.n_ct - done >= b) {
            hear_model::Plan *p;
            {
                std::lock_guard<std::mutex> g(m->plan_mu);
                p = graph_plan(m, S->evk, 0, m->layers.size(), b, s.reqs[0]->scale, s.st, 1 + slot_index, true);
            }
            for (uint32_t i = 0; i < b; i++)
                HEAR_CHECK_CUDA(cudaMemcpyAsync(p->X.u64() + (uint64_t)i * S->in_words, S->in_arena.at(io[done + i].first),
                                                S->in_words * 8, cudaMemcpyHostToDevice, s.st));
            HEAR_CHECK_CUDA(cudaGraphLaunch(p->exec, s.st));
            g_launches += p->launches;
            for (uint32_t i = 0; i < b; i++)
                HEAR_CHECK_CUDA(cudaMemcpyAsync(S->out_arena.at(io[done + i].second), p->Y.u64() + (uint64_t)i * S->out_words,
                                                S->out_words * 8, cudaMemcpyDeviceToHost, s.st));
            done += b;
        }
    }
    HEAR_CHECK_CUDA(cudaEventRecord(s.done, s.st));
    s.busy = true;
}

void release(Arena &a, std::vector<uint32_t> &bufs) {
    a.free.insert(a.free.end(), bufs.begin(), bufs.end());
    bufs.clear();
}

// called with S->mu held once the slot's event has completed
void finish(hear_server *S, Slot &s) {
    const auto now = Clock::now();
    for (auto &r : s.reqs) {
        r->t_done = now;
        r->state = 2;
        release(S->in_arena, r->in_bufs);    // the upload has completed
        S->done_reqs++;
        S->done_cts += r->n_ct;
        S->done_clips += r->n_clips;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
    }
    S->in_flight_cts -= s.n_ct;
    s.reqs.clear();
    s.n_ct = 0;
    s.busy = false;
    S->batches++;
}

// every request in flight or queued fails with `code`; their buffers return to the arenas
void fail_all(hear_server *S, hear_status code, const std::string &msg) {
    S->fault = code;
    S->fault_msg = msg;
    auto drop = [&](const std::shared_ptr<Request> &r) {
        r->state = 3;
        r->status = code;
        release(S->in_arena, r->in_bufs);
        release(S->out_arena, r->out_bufs);
    };
    for (auto &s : S->slots) {
        if (s.busy && s.st) cudaStreamSynchronize(s.st);   // no copy may still target the buffers
        for (auto &r : s.reqs) drop(r);
        s.reqs.clear();
        s.n_ct = 0;
        s.busy = false;
    }
    for (auto &r : S->pending) drop(r);
    S->pending.clear();
    S->in_flight_cts = 0;
}

void worker_loop(hear_server *S) {
    hear_context *c = S->m->ctx;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progressed = false;
        try {
            bool finished = false;
            for (auto &s : S->slots) {
                if (!s.busy) continue;
                const cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaSuccess) {
                    finish(S, s);
                    finished = true;
                } else if (q != cudaErrorNotReady) {
                    (void)cudaGetLastError();
                    throw Error(HEAR_E_CUDA, std::string("batch failed: ") + cudaGetErrorString(q));
                }
            }
            if (finished) {
                progressed = true;
                S->cv_done.notify_all();
            }
            for (uint32_t si = 0; si < S->slots.size() && !S->pending.empty() && !S->paused; si++) {
                Slot &s = S->slots[si];
                if (s.busy) continue;
                // admission in arrival order: batch size, HBM budget, result buffers
                while (!S->pending.empty()) {
                    auto &r = S->pending.front();
                    const uint64_t n = r->n_ct;
                    const bool fits_batch = s.n_ct + n <= S->cfg.max_batch;
                    const bool fits_hbm = (S->in_flight_cts + n) * S->ct_bytes <= S->cfg.hbm_budget_bytes;
                    const bool same_scale = s.reqs.empty() || s.reqs[0]->scale == r->scale;
                    const bool fits_out = S->out_arena.free.size() >= n;
                    if (!fits_batch || !fits_hbm || !same_scale || !fits_out) break;
                    for (uint64_t i = 0; i < n; i++) {
                        r->out_bufs.push_back(S->out_arena.free.back());
                        S->out_arena.free.pop_back();
                    }
                    r->state = 1;
                    s.reqs.push_back(r);
                    s.n_ct += (uint32_t)n;
                    S->in_flight_cts += n;
                    S->pending.pop_front();
                }
                if (s.reqs.empty()) break;   // the head of the queue does not fit right now
                S->max_in_flight_cts = std::max(S->max_in_flight_cts, S->in_flight_cts);
                lk.unlock();
                try {
                    launch(S, s, si);
                } catch (...) {
                    lk.lock();
                    throw;
                }
                lk.lock();
                progressed = true;
            }
        } catch (const Error &e) {
            fail_all(S, e.code, e.what());
            if (e.code == HEAR_E_CUDA) c->poisoned = true;
            S->cv_done.notify_all();
        }
        if (!progressed) S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

hear_status fail(hear_status code, const std::string &m) {
    set_last_error(m);
    return code;
}

// hands a finished request's result to the caller (lk held on entry and exit); a failed
// request reports its error; both release the id
hear_status deliver(hear_server *S, std::unique_lock<std::mutex> &lk,
                    std::map<uint64_t, std::shared_ptr<Request>>::iterator it, uint64_t *out, size_t cap,
                    size_t *n, int *done) {
    std::shared_ptr<Request> r = it->second;
    if (done) *done = 0;
    if (r->state == 3) {
        S->reqs.erase(it);
        return fail(r->status, "request failed: " + S->fault_msg);
    }
    if (r->state != 2) return HEAR_OK;
    const uint64_t words = (uint64_t)r->n_ct * S->out_words;
    if (n) *n = words;
    if (!out || cap < words) return fail(HEAR_E_INVAL, "output capacity too small");
    S->reqs.erase(it);      // the result buffers now belong to this call alone
    lk.unlock();
    for (uint32_t i = 0; i < r->n_ct; i++)
        std::memcpy(out + (uint64_t)i * S->out_words, S->out_arena.at(r->out_bufs[i]), S->out_words * 8);
    lk.lock();
    release(S->out_arena, r->out_bufs);
    S->cv.notify_all();     // result buffers freed: the worker may admit more
    if (done) *done = 1;
    return HEAR_OK;
}

void free_server(hear_server *S) {
    for (auto &s : S->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.done) cudaEventDestroy(s.done);
        if (s.st) cudaStreamDestroy(s.st);
    }
    if (S->in_arena.base) cudaFreeHost(S->in_arena.base);
    if (S->out_arena.base) cudaFreeHost(S->out_arena.base);
    S->in_arena.base = S->out_arena.base = nullptr;
}

}  // namespace

extern "C" {

hear_status hear_server_create(const hear_model *m, const hear_eval_keys *evk, const hear_server_config *cfg,
                               hear_server **out) {
    if (!m || !evk || !cfg || !out) return fail(HEAR_E_INVAL, "null argument");
    if (evk->ctx != m->ctx) return fail(HEAR_E_STATE, "keys from another context");
    if (cfg->max_batch < 1 || cfg->n_slots < 1 || cfg->n_slots > 8)
        return fail(HEAR_E_INVAL, "need max_batch >= 1 and 1 <= n_slots <= 8");
    const uint32_t staging = cfg->staging_cts ? cfg->staging_cts : std::max(4 * cfg->n_slots * cfg->max_batch, 64u);
    if (staging < cfg->max_batch) return fail(HEAR_E_INVAL, "staging_cts must hold a request of max_batch ciphertexts");
    hear_context *c = m->ctx;
    if (c->poisoned) return fail(HEAR_E_CUDA, "context is poisoned by an earlier CUDA error");
    auto S = std::make_unique<hear_server>();
    S->m = m;
    S->evk = evk;
    S->cfg = *cfg;
    S->cfg.staging_cts = staging;
    S->lin = m->layers.front().level_in;
    S->lout = m->layers.back().level_out;
    S->in_words = 2ull * (S->lin + 1) * c->n;
    S->out_words = 2ull * (S->lout + 1) * c->n;
    try {
        HEAR_CHECK_CUDA(cudaSetDevice(c->device));
        // device bytes charged per in-flight ciphertext: its share of the pool's high-water
        // mark over one single-ciphertext evaluation (work buffers), plus input and output
        uint64_t zero = 0, high = 0, base = 0;
        HEAR_CHECK_CUDA(cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &base));
        HEAR_CHECK_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrUsedMemHigh, &zero));
        {
            DevBuf x(S->in_words * 8, c->stream);
            HEAR_CHECK_CUDA(cudaMemsetAsync(x.p, 0, S->in_words * 8, c->stream));
            uint32_t lo;
            double so;
            DevBuf y = evaluate_batch(m, evk, 0, m->layers.size(), x.u64(), 1, &lo, c->default_scale, &so, c->stream);
            HEAR_CHECK_CUDA(cudaStreamSynchronize(c->stream));
        }
        HEAR_CHECK_CUDA(cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemHigh, &high));
        S->ct_bytes = (high > base ? high - base : 0) + 8 * (S->in_words + S->out_words) * 2;
        for (Arena *a : {&S->in_arena, &S->out_arena}) {
            a->words = a == &S->in_arena ? S->in_words : S->out_words;
            HEAR_CHECK_CUDA(cudaHostAlloc((void **)&a->base, (size_t)staging * a->words * 8, cudaHostAllocDefault));
            for (uint32_t i = staging; i-- > 0;) a->free.push_back(i);
        }
        S->slots.resize(cfg->n_slots);
        for (auto &s : S->slots) {
            HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
            HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
        }
    } catch (const Error &e) {
        free_server(S.get());
        return fail(e.code, e.what());
    }
    S->worker = std::thread(worker_loop, S.get());
    *out = S.release();
    return HEAR_OK;
}

hear_status hear_server_submit(hear_server *S, const uint64_t *words, size_t n_ct, uint32_t n_clips, double scale,
                               uint64_t *request_id) {
    if (!S || !words || !request_id || n_ct == 0) return fail(HEAR_E_INVAL, "bad argument");
    if (n_ct > S->cfg.max_batch) return fail(HEAR_E_INVAL, "request larger than max_batch ciphertexts");
    if (n_ct * S->ct_bytes > S->cfg.hbm_budget_bytes)
        return fail(HEAR_E_NOMEM, "request larger than the HBM budget");
    auto r = std::make_shared<Request>();
    r->n_ct = (uint32_t)n_ct;
    r->n_clips = n_clips;
    r->scale = scale;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->fault != HEAR_OK) return fail(S->fault, "server stopped after an error: " + S->fault_msg);
        if (S->cfg.max_pending && S->pending.size() >= S->cfg.max_pending) {
            S->busy_refusals++;
            return fail(HEAR_E_BUSY, "request queue full (max_pending)");
        }
        if (S->in_arena.free.size() < n_ct) {
            S->busy_refusals++;
            return fail(HEAR_E_BUSY, "staging buffers full (staging_cts)");
        }
        for (size_t i = 0; i < n_ct; i++) {
            r->in_bufs.push_back(S->in_arena.free.back());
            S->in_arena.free.pop_back();
        }
    }
    // one copy into the reserved pinned buffers, every residue checked against its prime
    const hear_context *c = S->m->ctx;
    const uint32_t L1 = S->lin + 1;
    bool bad = false;
    for (size_t i = 0; i < n_ct && !bad; i++) {
        uint64_t *dst = S->in_arena.at(r->in_bufs[i]);
        const uint64_t *src = words + i * S->in_words;
        for (uint32_t pl = 0; pl < 2 * L1 && !bad; pl++) {
            const uint64_t q = c->primes[pl % L1];
            const uint64_t *sp = src + (uint64_t)pl * c->n;
            uint64_t *dp = dst + (uint64_t)pl * c->n;
            uint64_t over = 0;
            for (uint32_t k = 0; k < c->n; k++) {
                const uint64_t v = sp[k];
                over |= (uint64_t)(v >= q);
                dp[k] = v;
            }
            bad = over != 0;
        }
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (bad) {
        release(S->in_arena, r->in_bufs);
        return fail(HEAR_E_FORMAT, "residue not reduced");
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    *request_id = r->id;
    S->cv.notify_all();
    return HEAR_OK;
}

hear_status hear_server_poll(hear_server *S, uint64_t request_id, uint64_t *out, size_t cap, size_t *n, int *done) {
    if (!S || !done) return fail(HEAR_E_INVAL, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return fail(HEAR_E_INVAL, "unknown request id");
    return deliver(S, lk, it, out, cap, n, done);
}

hear_status hear_server_wait(hear_server *S, uint64_t request_id, uint32_t timeout_ms, uint64_t *out, size_t cap,
                             size_t *n) {
    if (!S) return fail(HEAR_E_INVAL, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return fail(HEAR_E_INVAL, "unknown request id");
    std::shared_ptr<Request> r = it->second;
    const bool ready = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                           [&] { return r->state >= 2 || S->stop; });
    if (!ready || r->state < 2)
        return fail(HEAR_E_TIMEOUT, "request " + std::to_string(request_id) + " not finished within " +
                                        std::to_string(timeout_ms) + " ms (it stays queued)");
    it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return fail(HEAR_E_INVAL, "request was read by another call");
    int done = 0;
    return deliver(S, lk, it, out, cap, n, &done);
}

hear_status hear_server_pause(hear_server *S, int paused) {
    if (!S) return fail(HEAR_E_INVAL, "null argument");
    std::lock_guard<std::mutex> g(S->mu);
    S->paused = paused != 0;
    S->cv.notify_all();
    return HEAR_OK;
}

hear_status hear_server_stats(hear_server *S, hear_server_counters *st) {
    if (!S || !st) return fail(HEAR_E_INVAL, "null argument");
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->requests_done = S->done_reqs;
    st->ciphertexts_done = S->done_cts;
    st->clips_done = S->done_clips;
    st->batches = S->batches;
    st->pending = S->pending.size();
    st->max_in_flight_ciphertexts = S->max_in_flight_cts;
    st->bytes_per_ciphertext = S->ct_bytes;
    st->busy_refusals = S->busy_refusals;
    if (!S->lat_ms.empty()) {
        std::vector<double> l = S->lat_ms;
        std::sort(l.begin(), l.end());
        st->p50_ms = l[l.size() / 2];
        st->p99_ms = l[std::min(l.size() - 1, (size_t)(0.99 * l.size()))];
        double sum = 0;
        for (double v : l) sum += v;
        st->mean_ms = sum / l.size();
    }
    return HEAR_OK;
}

void hear_server_destroy(hear_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    S->cv_done.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->m->ctx->device);
    free_server(S);
    delete S;
}

}  // extern "C"
