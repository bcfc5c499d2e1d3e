// server.cu -- continuous-batching server for encrypted inference requests.
//
// Requests (ciphertexts of the end-user, coefficient domain, host memory) arrive at any
// time.  A worker thread admits pending requests in arrival order while the ciphertexts in
// flight fit the HBM budget, packs up to max_batch ciphertexts into one batch and runs it on
// a free slot: each slot owns a CUDA stream, pinned staging buffers and device buffers, so
// up to n_slots batches overlap on the device (copies of one batch overlap the evaluation of
// another).  A batch is split into power-of-two sub-batches, each the replay of a captured
// CUDA graph of the whole network.  The evaluation keys and the encoded model stay resident.
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

struct Request {
    uint64_t id = 0;
    uint32_t n_ct = 0, n_clips = 0;
    double scale = 0;
    std::vector<uint64_t> in, out;
    Clock::time_point t_submit, t_done;
    int state = 0;                    // 0 pending, 1 running, 2 done, 3 failed
    hear_status status = HEAR_OK;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf x, y;                      // device batch in (coefficient domain -> NTT), out
    uint64_t *h_in = nullptr, *h_out = nullptr;   // pinned staging
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
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::vector<Slot> slots;
    uint64_t next_id = 1, in_flight_cts = 0, max_in_flight_cts = 0;
    uint64_t done_reqs = 0, done_cts = 0, done_clips = 0, batches = 0;
    std::vector<double> lat_ms;
    Clock::time_point t0;
    bool t0_set = false, stop = false;
    hear_status fault = HEAR_OK;
    std::string fault_msg;
    std::thread worker;
};

namespace {

// evaluate the n_ct ciphertexts of slot s (already in s.x, NTT domain) into s.y
void run_batch(hear_server *S, Slot &s, uint32_t slot_index) {
    const hear_model *m = S->m;
    hear_context *c = m->ctx;
    const uint64_t ctw_in = S->in_words, ctw_out = S->out_words;
    uint32_t done = 0;
    for (uint32_t b = 1u << 31; b; b >>= 1) {
        while (S->cfg.max_batch >= b && s.n_ct - done >= b) {
            hear_model::Plan *p;
            {
                std::lock_guard<std::mutex> g(m->plan_mu);
                p = graph_plan(m, S->evk, 0, m->layers.size(), b, s.reqs[0]->scale, s.st, 1 + slot_index);
            }
            HEAR_CHECK_CUDA(cudaMemcpyAsync(p->X.p, s.x.u64() + done * ctw_in, b * ctw_in * 8,
                                            cudaMemcpyDeviceToDevice, s.st));
            HEAR_CHECK_CUDA(cudaGraphLaunch(p->exec, s.st));
            g_launches += p->launches;
            HEAR_CHECK_CUDA(cudaMemcpyAsync(s.y.u64() + done * ctw_out, p->Y.p, b * ctw_out * 8,
                                            cudaMemcpyDeviceToDevice, s.st));
            done += b;
        }
    }
}

void launch(hear_server *S, Slot &s, uint32_t slot_index) {
    hear_context *c = S->m->ctx;
    uint64_t off = 0;
    for (auto &r : s.reqs) {
        std::memcpy(s.h_in + off, r->in.data(), r->in.size() * 8);
        off += r->in.size();
    }
    HEAR_CHECK_CUDA(cudaMemcpyAsync(s.x.p, s.h_in, off * 8, cudaMemcpyHostToDevice, s.st));
    ntt_forward(c, s.x.u64(), s.n_ct * 2 * (S->lin + 1), map_q(S->lin, c->n_q), s.st);
    run_batch(S, s, slot_index);
    ntt_inverse(c, s.y.u64(), s.n_ct * 2 * (S->lout + 1), map_q(S->lout, c->n_q), s.st);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(s.h_out, s.y.p, s.n_ct * S->out_words * 8, cudaMemcpyDeviceToHost, s.st));
    HEAR_CHECK_CUDA(cudaEventRecord(s.done, s.st));
    s.busy = true;
}

// copies the results of a finished slot out of its pinned buffer; called without S->mu
// (the requests stay in state 1 and the slot busy until finish() runs)
void collect(hear_server *S, Slot &s) {
    uint64_t off = 0;
    for (auto &r : s.reqs) {
        r->out.assign(s.h_out + off, s.h_out + off + (uint64_t)r->n_ct * S->out_words);
        off += (uint64_t)r->n_ct * S->out_words;
    }
}

// called with S->mu held, after collect()
void finish(hear_server *S, Slot &s) {
    const auto now = Clock::now();
    for (auto &r : s.reqs) {
        r->t_done = now;
        r->state = 2;
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

void worker_loop(hear_server *S) {
    hear_context *c = S->m->ctx;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progressed = false;
        try {
            for (auto &s : S->slots)
                if (s.busy && cudaEventQuery(s.done) == cudaSuccess) {
                    lk.unlock();
                    collect(S, s);
                    lk.lock();
                    finish(S, s);
                    progressed = true;
                }
            for (uint32_t si = 0; si < S->slots.size() && !S->pending.empty(); si++) {
                Slot &s = S->slots[si];
                if (s.busy) continue;
                // admission in arrival order: batch size and HBM budget
                while (!S->pending.empty()) {
                    auto &r = S->pending.front();
                    const uint64_t n = r->n_ct;
                    const bool fits_batch = s.n_ct + n <= S->cfg.max_batch;
                    const bool fits_hbm = (S->in_flight_cts + n) * S->ct_bytes <= S->cfg.hbm_budget_bytes;
                    const bool same_scale = s.reqs.empty() || s.reqs[0]->scale == r->scale;
                    if (!fits_batch || !fits_hbm || !same_scale) break;
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
            S->fault = e.code;
            S->fault_msg = e.what();
            for (auto &s : S->slots) {
                for (auto &r : s.reqs) {
                    r->state = 3;
                    r->status = e.code;
                }
                s.reqs.clear();
                s.busy = false;
            }
            for (auto &r : S->pending) {
                r->state = 3;
                r->status = e.code;
            }
            S->pending.clear();
            if (e.code == HEAR_E_CUDA) c->poisoned = true;
        }
        S->cv.notify_all();
        if (!progressed) S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

hear_status fail(hear_status code, const std::string &m) {
    set_last_error(m);
    return code;
}

}  // namespace

extern "C" {

hear_status hear_server_create(const hear_model *m, const hear_eval_keys *evk, const hear_server_config *cfg,
                               hear_server **out) {
    if (!m || !evk || !cfg || !out) return fail(HEAR_E_INVAL, "null argument");
    if (evk->ctx != m->ctx) return fail(HEAR_E_STATE, "keys from another context");
    if (cfg->max_batch < 1 || cfg->n_slots < 1 || cfg->n_slots > 8)
        return fail(HEAR_E_INVAL, "need max_batch >= 1 and 1 <= n_slots <= 8");
    hear_context *c = m->ctx;
    if (c->poisoned) return fail(HEAR_E_CUDA, "context is poisoned by an earlier CUDA error");
    auto S = std::make_unique<hear_server>();
    S->m = m;
    S->evk = evk;
    S->cfg = *cfg;
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
        S->slots.resize(cfg->n_slots);
        for (auto &s : S->slots) {
            HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
            HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
            s.x = DevBuf((size_t)cfg->max_batch * S->in_words * 8, nullptr);
            s.y = DevBuf((size_t)cfg->max_batch * S->out_words * 8, nullptr);
            HEAR_CHECK_CUDA(cudaHostAlloc(&s.h_in, (size_t)cfg->max_batch * S->in_words * 8, cudaHostAllocDefault));
            HEAR_CHECK_CUDA(cudaHostAlloc(&s.h_out, (size_t)cfg->max_batch * S->out_words * 8, cudaHostAllocDefault));
        }
    } catch (const Error &e) {
        for (auto &s : S->slots) {
            if (s.h_in) cudaFreeHost(s.h_in);
            if (s.h_out) cudaFreeHost(s.h_out);
            if (s.st) cudaStreamDestroy(s.st);
            if (s.done) cudaEventDestroy(s.done);
        }
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
    const hear_context *c = S->m->ctx;
    r->in.assign(words, words + n_ct * S->in_words);
    for (uint64_t i = 0; i < n_ct * 2 * (S->lin + 1); i++) {
        const uint64_t q = c->primes[i % (S->lin + 1)];
        const uint64_t *w = r->in.data() + i * c->n;
        for (uint32_t k = 0; k < c->n; k++)
            if (w[k] >= q) return fail(HEAR_E_FORMAT, "residue not reduced");
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fault != HEAR_OK) return fail(S->fault, "server stopped after an error: " + S->fault_msg);
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    if (!S->t0_set) {
        S->t0 = r->t_submit;
        S->t0_set = true;
    }
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    *request_id = r->id;
    S->cv.notify_all();
    return HEAR_OK;
}

hear_status hear_server_poll(hear_server *S, uint64_t request_id, uint64_t *out, size_t cap, size_t *n, int *done) {
    if (!S || !done) return fail(HEAR_E_INVAL, "null argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return fail(HEAR_E_INVAL, "unknown request id");
    Request &r = *it->second;
    *done = 0;
    if (r.state == 3) {
        S->reqs.erase(it);
        return fail(r.status, "request failed: " + S->fault_msg);
    }
    if (r.state != 2) return HEAR_OK;
    if (n) *n = r.out.size();
    if (!out || cap < r.out.size()) return fail(HEAR_E_INVAL, "output capacity too small");
    std::copy(r.out.begin(), r.out.end(), out);
    *done = 1;
    S->reqs.erase(it);
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
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->m->ctx->device);
    for (auto &s : S->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.h_in) cudaFreeHost(s.h_in);
        if (s.h_out) cudaFreeHost(s.h_out);
        if (s.done) cudaEventDestroy(s.done);
        if (s.st) cudaStreamDestroy(s.st);
    }
    delete S;
}

}  // extern "C"
