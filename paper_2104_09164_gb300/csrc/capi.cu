// capi.cu -- the extern "C" boundary (include/hear.h): argument checks, error capture,
// handle management.  No C++ exception crosses it.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include "ckks.h"
#include "simd.h"

using namespace hear;

namespace {
thread_local std::string g_last_error;

hear_status fail(hear_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

template <class F>
hear_status guard(hear_context *ctx, F &&f) {
    if (ctx && ctx->poisoned) return fail(HEAR_E_CUDA, "context is poisoned by an earlier CUDA error");
    try {
        if (ctx) HEAR_CHECK_CUDA(cudaSetDevice(ctx->device));
        AllocScope alloc_scope(ctx ? &ctx->allocator : nullptr);
        f();
        return HEAR_OK;
    } catch (const Error &e) {
        if (e.code == HEAR_E_CUDA && ctx) ctx->poisoned = true;
        return fail(e.code, e.what());
    } catch (const std::bad_alloc &) {
        return fail(HEAR_E_NOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(HEAR_E_INVAL, e.what());
    } catch (...) {
        return fail(HEAR_E_INVAL, "unknown error");
    }
}

cudaStream_t stream_of(hear_context *c, void *s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

// Whole evaluations replay a captured CUDA graph unless the stage profiler is on (it brackets
// each launch with events) or HEAR_NO_GRAPH is set in the environment.
bool use_graphs(const hear_context *c) {
    static const bool off = [] {
        const char *v = std::getenv("HEAR_NO_GRAPH");
        return v && *v && *v != '0';
    }();
    return !off && !c->prof.on;
}

template <class T>
hear_status copy_out(const std::vector<T> &v, T *out, size_t cap, size_t *n) {
    if (n) *n = v.size();
    if (!out || cap < v.size()) return fail(HEAR_E_INVAL, "output capacity too small");
    std::copy(v.begin(), v.end(), out);
    return HEAR_OK;
}

// ciphertext memory comes from the stream-ordered pool of the stream the ciphertext is
// produced on and is returned to it when the handle is destroyed
hear_ciphertext *new_ct(hear_context *c, uint32_t level, uint32_t n_poly, double scale, cudaStream_t st) {
    auto ct = new hear_ciphertext();
    ct->ctx = c;
    ct->level = level;
    ct->n_poly = n_poly;
    ct->scale = scale;
    try {
        ct->d = DevBuf((size_t)n_poly * (level + 1) * c->n * 8, st);
    } catch (...) {
        delete ct;
        throw;
    }
    return ct;
}

// coefficient-domain host words -> NTT-domain device batch (n_polys polynomials at level)
void to_device_ntt(hear_context *c, const uint64_t *words, uint32_t level, uint32_t n_polys, uint64_t *d,
                   cudaStream_t st) {
    const size_t words_n = (size_t)n_polys * (level + 1) * c->n;
    HEAR_CHECK_CUDA(cudaMemcpyAsync(d, words, words_n * 8, cudaMemcpyHostToDevice, st));
    ntt_forward(c, d, n_polys * (level + 1), map_q(level, c->n_q), st);
}
}  // namespace

namespace hear {
// lets other translation units report through hear_last_error()
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace hear

extern "C" {

const char *hear_last_error(void) { return g_last_error.c_str(); }

hear_status hear_context_create(const hear_params_desc *params, int cuda_device, hear_context **out) {
    if (!out || !params) return fail(HEAR_E_INVAL, "null argument");
    auto c = new hear_context();
    hear_status s = guard(nullptr, [&] {
        build_context(c, params, cuda_device);
        ks_bulk_setup();
        simd_setup();
        // pick the NTT launch variant per launch size by timing them (HEAR_NTT_TUNE=0 keeps
        // the fixed rule); every variant computes the same residues
        const char *t = std::getenv("HEAR_NTT_TABLE");
        const char *v = std::getenv("HEAR_NTT_TUNE");
        if (t && *t) {
            // a pinned table: 32 digits, forward buckets then inverse buckets
            HEAR_REQUIRE(std::strlen(t) == 2 * (size_t)kNttBuckets, HEAR_E_INVAL, "HEAR_NTT_TABLE needs 32 digits");
            for (int i = 0; i < 2 * kNttBuckets; i++) {
                HEAR_REQUIRE(t[i] >= '0' && t[i] < '0' + kNttVariants, HEAR_E_INVAL, "bad HEAR_NTT_TABLE digit");
                c->ntt_choice[i / kNttBuckets][i % kNttBuckets] = (uint8_t)(t[i] - '0');
            }
        } else if (!(v && *v == '0')) {
            ntt_tune(c, 1024, 8, nullptr);
        }
        // a pinned table of key-switch / inner-sum launch forms (24 digits), e.g. to profile
        // the forms a tuned run used; every form computes the same residues
        const char *kt = std::getenv("HEAR_KS_TABLE");
        if (kt && *kt) {
            HEAR_REQUIRE(std::strlen(kt) == (size_t)kKsTables * kKsBuckets, HEAR_E_INVAL, "HEAR_KS_TABLE needs 24 digits");
            for (int i = 0; i < kKsTables * kKsBuckets; i++) {
                HEAR_REQUIRE(kt[i] >= '0' && kt[i] < '0' + kKsVariants[i / kKsBuckets], HEAR_E_INVAL,
                             "bad HEAR_KS_TABLE digit");
                c->ks_choice[i / kKsBuckets][i % kKsBuckets] = (uint8_t)(kt[i] - '0');
            }
        }
    });
    if (s != HEAR_OK) {
        delete c;
        return s;
    }
    *out = c;
    return HEAR_OK;
}

void hear_context_destroy(hear_context *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    forget_encoder(ctx);
    ctx->levels.clear();
    ctx->d_primes.reset();
    ctx->d_tw.reset();
    ctx->d_cdt.reset();
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

hear_status hear_set_allocator(hear_context *ctx, void *(*alloc)(size_t, void *, void *),
                               void (*free_fn)(void *, void *, void *), void *user) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    if (!alloc != !free_fn) return fail(HEAR_E_INVAL, "give both allocator functions or neither");
    ctx->allocator.alloc = alloc;
    ctx->allocator.free = free_fn;
    ctx->allocator.user = user;
    return HEAR_OK;
}

hear_status hear_context_primes(const hear_context *ctx, uint64_t *out, size_t cap, size_t *n) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    return copy_out(ctx->primes, out, cap, n);
}

hear_status hear_context_cdt(const hear_context *ctx, uint64_t *out, size_t cap, size_t *n) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    return copy_out(ctx->cdt, out, cap, n);
}

hear_status hear_keygen(hear_context *ctx, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                        hear_secret_key **sk, hear_public_key **pk, hear_eval_keys **evk) {
    if (!ctx || !sk || !pk || !evk || (n_steps && !rot_steps)) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { keygen(ctx, seed, rot_steps, n_steps, sk, pk, evk); });
}

void hear_secret_key_destroy(hear_secret_key *k) {
    if (k) cudaSetDevice(k->ctx->device);
    delete k;
}
void hear_public_key_destroy(hear_public_key *k) {
    if (k) cudaSetDevice(k->ctx->device);
    delete k;
}
void hear_eval_keys_destroy(hear_eval_keys *k) {
    if (k) cudaSetDevice(k->ctx->device);
    delete k;
}

hear_status hear_secret_key_export(const hear_secret_key *sk, int8_t *out, size_t cap, size_t *n) {
    if (!sk) return fail(HEAR_E_INVAL, "null key");
    return copy_out(sk->s, out, cap, n);
}

hear_status hear_public_key_export(const hear_public_key *pk, uint64_t *out, size_t cap, size_t *n) {
    if (!pk) return fail(HEAR_E_INVAL, "null key");
    hear_context *c = pk->ctx;
    const size_t words = 2ull * c->n_q * c->n;
    if (n) *n = words;
    if (!out || cap < words) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = c->stream;
        DevBuf t(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(t.p, pk->pk_mont.p, words * 8, cudaMemcpyDeviceToDevice, st));
        LimbMap m = map_q(c->L, c->n_q);
        from_mont(c, t.u64(), 2 * c->n_q, m, st);
        ntt_inverse(c, t.u64(), 2 * c->n_q, m, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_eval_key_export(const hear_eval_keys *evk, uint32_t galois, uint64_t *out, size_t cap, size_t *n) {
    if (!evk) return fail(HEAR_E_INVAL, "null key");
    hear_context *c = evk->ctx;
    const uint64_t *k = evk->key(galois);
    if (!k) return fail(HEAR_E_NOKEY, "no key for this galois element");
    const size_t words = (size_t)c->dnum_max() * 2 * c->nqp() * c->n;
    if (n) *n = words;
    if (!out || cap < words) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = c->stream;
        DevBuf t(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(t.p, k, words * 8, cudaMemcpyDeviceToDevice, st));
        LimbMap m;
        m.per_group = c->nqp();
        m.q_count = c->n_q;
        m.n_q = c->n_q;
        const uint32_t limbs = c->dnum_max() * 2 * c->nqp();
        if (galois != 1) {
            // rotation keys are stored sigma_g^{-1}-permuted; undo it
            DevBuf u(words * 8, st);
            automorphism(c, c->nqp() - 1, c->dnum_max() * 2, galois, t.u64(), u.u64(), st);
            HEAR_CHECK_CUDA(cudaMemcpyAsync(t.p, u.p, words * 8, cudaMemcpyDeviceToDevice, st));
        }
        from_mont(c, t.u64(), limbs, m, st);
        ntt_inverse(c, t.u64(), limbs, m, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_encode(const hear_context *ctx, const double *z, size_t n_slots, double scale, int64_t *m_out,
                        size_t cap, size_t *n) {
    if (!ctx || !z || !m_out) return fail(HEAR_E_INVAL, "null argument");
    if (n) *n = ctx->n;
    if (n_slots != ctx->n / 2) return fail(HEAR_E_INVAL, "n_slots must be N/2");
    if (cap < ctx->n) return fail(HEAR_E_INVAL, "output capacity too small");
    hear_context *c = const_cast<hear_context *>(ctx);
    return guard(c, [&] { encode_dd(*encoder(c), z, scale, m_out); });
}

hear_status hear_encrypt(hear_context *ctx, const hear_public_key *pk, const double *z, size_t n_slots, double scale,
                         uint64_t seed, uint64_t ct_id, hear_ciphertext **out, void *stream) {
    if (!ctx || !pk || !z || !out) return fail(HEAR_E_INVAL, "null argument");
    if (pk->ctx != ctx) return fail(HEAR_E_STATE, "key from another context");
    if (n_slots != ctx->n / 2) return fail(HEAR_E_INVAL, "n_slots must be N/2");
    return guard(ctx, [&] {
        double sc = scale > 0 ? scale : ctx->default_scale;
        *out = encrypt_slots(ctx, pk, z, sc, seed, ct_id, stream_of(ctx, stream));
    });
}

hear_status hear_encrypt_clips(hear_context *ctx, const hear_public_key *pk, const double *clips, size_t n_clips,
                               size_t clip_dim, uint64_t seed, uint64_t ct_id, hear_ciphertext **out, void *stream) {
    if (!ctx || !pk || !clips || !out) return fail(HEAR_E_INVAL, "null argument");
    const size_t slots = ctx->n / 2;
    if (!clip_dim || (clip_dim & (clip_dim - 1)) || clip_dim > slots)
        return fail(HEAR_E_INVAL, "clip_dim must be a power of two <= N/2");
    const size_t k = slots / clip_dim;
    if (n_clips < 1 || n_clips > k) return fail(HEAR_E_INVAL, "n_clips must be in [1, N/2 / clip_dim]");
    std::vector<double> z(slots);
    for (size_t c = 0; c < k; c++)
        for (size_t p = 0; p < clip_dim; p++) z[p * k + c] = clips[(c % n_clips) * clip_dim + p];
    return hear_encrypt(ctx, pk, z.data(), slots, 0.0, seed, ct_id, out, stream);
}

hear_status hear_decrypt(hear_context *ctx, const hear_secret_key *sk, const hear_ciphertext *ct, double *out,
                         size_t cap, size_t *n) {
    if (!ctx || !sk || !ct) return fail(HEAR_E_INVAL, "null argument");
    if (n) *n = ctx->n / 2;
    if (!out || cap < ctx->n / 2) return fail(HEAR_E_INVAL, "output capacity too small");
    if (ct->n_poly != 2) return fail(HEAR_E_STATE, "decrypt needs a 2-polynomial ciphertext");
    return guard(ctx, [&] { decrypt_slots(ctx, sk, ct, out); });
}

void hear_ciphertext_destroy(hear_ciphertext *ct) {
    if (ct) cudaSetDevice(ct->ctx->device);
    delete ct;
}

hear_status hear_ciphertext_info(const hear_ciphertext *ct, uint32_t *level, uint32_t *n_poly, double *scale) {
    if (!ct) return fail(HEAR_E_INVAL, "null ciphertext");
    if (level) *level = ct->level;
    if (n_poly) *n_poly = ct->n_poly;
    if (scale) *scale = ct->scale;
    return HEAR_OK;
}

hear_status hear_ciphertext_export(const hear_ciphertext *ct, uint64_t *out, size_t cap, size_t *n) {
    if (!ct) return fail(HEAR_E_INVAL, "null ciphertext");
    hear_context *c = ct->ctx;
    const size_t words = (size_t)ct->n_poly * (ct->level + 1) * c->n;
    if (n) *n = words;
    if (!out || cap < words) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = c->stream;
        DevBuf t(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(t.p, ct->d.p, words * 8, cudaMemcpyDeviceToDevice, st));
        ntt_inverse(c, t.u64(), ct->n_poly * (ct->level + 1), map_q(ct->level, c->n_q), st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_ciphertext_import(hear_context *ctx, const uint64_t *words, size_t n_words, uint32_t level,
                                   uint32_t n_poly, double scale, hear_ciphertext **out, void *stream) {
    if (!ctx || !words || !out) return fail(HEAR_E_INVAL, "null argument");
    if (level > ctx->L || n_poly < 2 || n_poly > 3) return fail(HEAR_E_FORMAT, "bad level or polynomial count");
    if (n_words != (size_t)n_poly * (level + 1) * ctx->n) return fail(HEAR_E_FORMAT, "word count mismatch");
    return guard(ctx, [&] {
        for (size_t i = 0; i < (size_t)n_poly * (level + 1); i++) {
            uint64_t q = ctx->primes[i % (level + 1)];
            const uint64_t *w = words + i * ctx->n;
            for (uint32_t k = 0; k < ctx->n; k++)
                HEAR_REQUIRE(w[k] < q, HEAR_E_FORMAT, "residue not reduced");
        }
        hear_ciphertext *ct = new_ct(ctx, level, n_poly, scale, stream_of(ctx, stream));
        try {
            to_device_ntt(ctx, words, level, n_poly, ct->d.u64(), stream_of(ctx, stream));
        } catch (...) {
            delete ct;
            throw;
        }
        *out = ct;
    });
}

hear_status hear_rotate_hoisted(const hear_eval_keys *evk, const hear_ciphertext *ct, const int32_t *steps,
                                size_t n_steps, hear_ciphertext **out, void *stream) {
    if (!evk || !ct || !out || (n_steps && !steps)) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = ct->ctx;
    if (evk->ctx != c) return fail(HEAR_E_STATE, "key from another context");
    if (ct->n_poly != 2) return fail(HEAR_E_STATE, "rotation needs a 2-polynomial ciphertext");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        std::vector<Rot> rots;
        for (size_t i = 0; i < n_steps; i++) {
            uint32_t g = galois_of(c, steps[i]);
            const uint64_t *k = evk->key(g);
            HEAR_REQUIRE(k, HEAR_E_NOKEY, "missing rotation key for step " + std::to_string(steps[i]));
            rots.push_back(Rot{k, g});
        }
        const uint64_t ctw = 2ull * (ct->level + 1) * c->n;
        DevBuf all((size_t)n_steps * ctw * 8, st);
        rotate_hoisted(c, ct->level, 1, ct->d.u64(), rots, all.u64(), st);
        std::vector<std::unique_ptr<hear_ciphertext>> res;
        for (size_t i = 0; i < n_steps; i++) {
            res.emplace_back(new_ct(c, ct->level, 2, ct->scale, st));
            HEAR_CHECK_CUDA(cudaMemcpyAsync(res.back()->d.p, all.u64() + i * ctw, ctw * 8, cudaMemcpyDeviceToDevice, st));
        }
        for (size_t i = 0; i < n_steps; i++) out[i] = res[i].release();
    });
}

hear_status hear_rotate(const hear_eval_keys *evk, const hear_ciphertext *ct, int32_t step, hear_ciphertext **out,
                        void *stream) {
    return hear_rotate_hoisted(evk, ct, &step, 1, out, stream);
}

hear_status hear_rescale(const hear_ciphertext *ct, hear_ciphertext **out, void *stream) {
    if (!ct || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = ct->ctx;
    if (ct->level == 0) return fail(HEAR_E_LEVEL, "ciphertext at level 0 cannot be rescaled");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        const size_t words = (size_t)ct->n_poly * (ct->level + 1) * c->n;
        DevBuf in(words * 8, st), tmp((size_t)ct->n_poly * ct->level * c->n * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(in.p, ct->d.p, words * 8, cudaMemcpyDeviceToDevice, st));
        std::unique_ptr<hear_ciphertext> r(
            new_ct(c, ct->level - 1, ct->n_poly, ct->scale / (double)c->primes[ct->level], st));
        rescale(c, ct->level, ct->n_poly, in.u64(), r->d.u64(), tmp.u64(), st);
        *out = r.release();
    });
}

hear_status hear_ciphertext_drop_level(const hear_ciphertext *ct, uint32_t level, hear_ciphertext **out,
                                       void *stream) {
    if (!ct || !out) return fail(HEAR_E_INVAL, "null argument");
    if (level > ct->level) return fail(HEAR_E_LEVEL, "cannot raise the level of a ciphertext");
    hear_context *c = ct->ctx;
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        std::unique_ptr<hear_ciphertext> r(new_ct(c, level, ct->n_poly, ct->scale, st));
        HEAR_CHECK_CUDA(cudaMemcpy2DAsync(r->d.p, (size_t)(level + 1) * c->n * 8, ct->d.p,
                                          (size_t)(ct->level + 1) * c->n * 8, (size_t)(level + 1) * c->n * 8,
                                          ct->n_poly, cudaMemcpyDeviceToDevice, st));
        *out = r.release();
    });
}

hear_status hear_add(const hear_ciphertext *a, const hear_ciphertext *b, hear_ciphertext **out, void *stream) {
    if (!a || !b || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = a->ctx;
    if (b->ctx != c) return fail(HEAR_E_STATE, "operands from different contexts");
    if (a->level != b->level || a->n_poly != b->n_poly) return fail(HEAR_E_SCALE, "operands at different levels");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        std::unique_ptr<hear_ciphertext> r(new_ct(c, a->level, a->n_poly, a->scale, st));
        add_ct(c, a->level, a->n_poly, a->d.u64(), b->d.u64(), r->d.u64(), st);
        *out = r.release();
    });
}

hear_status hear_mulplain(const hear_ciphertext *ct, const double *z, size_t n_slots, double pt_scale,
                          hear_ciphertext **out, void *stream) {
    if (!ct || !z || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = ct->ctx;
    if (n_slots != c->n / 2) return fail(HEAR_E_INVAL, "n_slots must be N/2");
    if (ct->n_poly != 2) return fail(HEAR_E_STATE, "MultPlain needs a 2-polynomial ciphertext");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        DevBuf pt = encode_plain(c, z, pt_scale, ct->level, st);
        std::unique_ptr<hear_ciphertext> r(new_ct(c, ct->level, 2, ct->scale * pt_scale, st));
        mulplain(c, ct->level, 1, ct->d.u64(), pt.u64(), r->d.u64(), st);
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
        *out = r.release();
    });
}

hear_status hear_multiply_relin(const hear_eval_keys *evk, const hear_ciphertext *a, const hear_ciphertext *b,
                                hear_ciphertext **out, void *stream) {
    if (!evk || !a || !b || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = a->ctx;
    if (b->ctx != c || evk->ctx != c) return fail(HEAR_E_STATE, "operands from different contexts");
    if (a->level != b->level || a->n_poly != 2 || b->n_poly != 2) return fail(HEAR_E_SCALE, "operand mismatch");
    const uint64_t *rk = evk->key(1);
    if (!rk) return fail(HEAR_E_NOKEY, "missing relinearisation key");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        std::unique_ptr<hear_ciphertext> r(new_ct(c, a->level, 2, a->scale * b->scale, st));
        mul_relin(c, a->level, 1, a->d.u64(), b->d.u64(), rk, r->d.u64(), st);
        *out = r.release();
    });
}

hear_status hear_model_create(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers, uint32_t clip_dim,
                              hear_model **out) {
    if (!ctx || !layers || !out) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *out = model_create(ctx, layers, n_layers, clip_dim, ctx->L, kDefaultRotsumRadix); });
}

hear_status hear_model_create_at_level(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                                       uint32_t clip_dim, uint32_t level, hear_model **out) {
    if (!ctx || !layers || !out) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *out = model_create(ctx, layers, n_layers, clip_dim, level, kDefaultRotsumRadix); });
}

hear_status hear_model_create_ex(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers, uint32_t clip_dim,
                                const hear_model_opts *opts, hear_model **out) {
    if (!ctx || !layers || !out) return fail(HEAR_E_INVAL, "null argument");
    const uint32_t level = opts && opts->level ? opts->level : ctx->L;
    const uint32_t radix = opts && opts->rotsum_radix ? opts->rotsum_radix : kDefaultRotsumRadix;
    const uint32_t n1 = opts ? opts->fc_n1 : 0;
    const bool dh = opts && opts->hoist_moddown;
    const bool hs = opts && opts->hoist_sums;
    if (n1 && (n1 & (n1 - 1))) return fail(HEAR_E_INVAL, "fc_n1 must be a power of two");
    return guard(ctx, [&] { *out = model_create(ctx, layers, n_layers, clip_dim, level, radix, n1, dh, hs); });
}

hear_status hear_model_levels(const hear_model *m, uint32_t *level_in, uint32_t *level_out) {
    if (!m || m->layers.empty()) return fail(HEAR_E_INVAL, "null model");
    if (level_in) *level_in = m->layers.front().level_in;
    if (level_out) *level_out = m->layers.back().level_out;
    return HEAR_OK;
}

void hear_model_destroy(hear_model *m) {
    if (m) cudaSetDevice(m->ctx->device);
    delete m;
}

hear_status hear_model_rotations(const hear_model *m, int32_t *steps, size_t cap, size_t *n) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    return copy_out(m->rotations, steps, cap, n);
}

hear_status hear_model_output_positions(const hear_model *m, uint32_t *pos, size_t cap, size_t *n) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    return copy_out(m->out_pos, pos, cap, n);
}

static hear_status evaluate_range(const hear_model *m, size_t l0, size_t l1, const hear_eval_keys *evk,
                                  hear_ciphertext *const *in, size_t n_ct, hear_ciphertext **out, void *stream) {
    if (!m || !evk || !in || !out || n_ct == 0) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = m->ctx;
    if (evk->ctx != c) return fail(HEAR_E_STATE, "keys from another context");
    const uint32_t lin = m->layers[l0].level_in;
    for (size_t i = 0; i < n_ct; i++) {
        if (!in[i] || in[i]->ctx != c) return fail(HEAR_E_STATE, "ciphertext from another context");
        if (in[i]->level != lin || in[i]->n_poly != 2) return fail(HEAR_E_LEVEL, "input not at the layer's level");
        if (in[i]->scale != in[0]->scale) return fail(HEAR_E_SCALE, "inputs at different scales");
    }
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        const uint64_t ctw = 2ull * (lin + 1) * c->n;
        if (use_graphs(c)) {
            std::lock_guard<std::mutex> g(m->plan_mu);
            hear_model::Plan *p = graph_plan(m, evk, l0, l1, (uint32_t)n_ct, in[0]->scale, st);
            HEAR_CHECK_CUDA(cudaStreamWaitEvent(st, p->done, 0));
            for (size_t i = 0; i < n_ct; i++)
                HEAR_CHECK_CUDA(cudaMemcpyAsync(p->X.u64() + i * ctw, in[i]->d.p, ctw * 8, cudaMemcpyDeviceToDevice, st));
            HEAR_CHECK_CUDA(cudaGraphLaunch(p->exec, st));
            g_launches += p->launches;
            const uint64_t otw = 2ull * (p->level_out + 1) * c->n;
            std::vector<std::unique_ptr<hear_ciphertext>> res;
            for (size_t i = 0; i < n_ct; i++) {
                res.emplace_back(new_ct(c, p->level_out, 2, p->scale_out, st));
                HEAR_CHECK_CUDA(
                    cudaMemcpyAsync(res.back()->d.p, p->Y.u64() + i * otw, otw * 8, cudaMemcpyDeviceToDevice, st));
            }
            HEAR_CHECK_CUDA(cudaEventRecord(p->done, st));
            for (size_t i = 0; i < n_ct; i++) out[i] = res[i].release();
            return;
        }
        DevBuf X((size_t)n_ct * ctw * 8, st);
        for (size_t i = 0; i < n_ct; i++)
            HEAR_CHECK_CUDA(cudaMemcpyAsync(X.u64() + i * ctw, in[i]->d.p, ctw * 8, cudaMemcpyDeviceToDevice, st));
        uint32_t lout;
        double sout;
        DevBuf Y = evaluate_batch(m, evk, l0, l1, X.u64(), (uint32_t)n_ct, &lout, in[0]->scale, &sout, st);
        const uint64_t otw = 2ull * (lout + 1) * c->n;
        std::vector<std::unique_ptr<hear_ciphertext>> res;
        for (size_t i = 0; i < n_ct; i++) {
            res.emplace_back(new_ct(c, lout, 2, sout, st));
            HEAR_CHECK_CUDA(cudaMemcpyAsync(res.back()->d.p, Y.u64() + i * otw, otw * 8, cudaMemcpyDeviceToDevice, st));
        }
        for (size_t i = 0; i < n_ct; i++) out[i] = res[i].release();
    });
}

hear_status hear_evaluate(const hear_model *m, const hear_eval_keys *evk, hear_ciphertext *const *in, size_t n_ct,
                          hear_ciphertext **out, void *stream) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    return evaluate_range(m, 0, m->layers.size(), evk, in, n_ct, out, stream);
}

hear_status hear_multi_create(const hear_model *const *models, const hear_eval_keys *const *evks, size_t n_jobs,
                              const uint32_t *n_ct, const double *scales, hear_multi **out) {
    if (!models || !evks || !n_ct || !scales || !out || n_jobs == 0) return fail(HEAR_E_INVAL, "null argument");
    for (size_t i = 0; i < n_jobs; i++) {
        if (!models[i] || !evks[i]) return fail(HEAR_E_INVAL, "null model or keys");
        if (evks[i]->ctx != models[i]->ctx) return fail(HEAR_E_STATE, "keys from another context");
        if (models[i]->ctx->device != models[0]->ctx->device) return fail(HEAR_E_INVAL, "jobs on different devices");
        if (n_ct[i] == 0 || !(scales[i] > 0)) return fail(HEAR_E_INVAL, "empty job or bad scale");
    }
    hear_context *c = models[0]->ctx;
    return guard(c, [&] { *out = multi_create(models, evks, n_jobs, n_ct, scales, c->stream); });
}

hear_status hear_multi_evaluate(hear_multi *mu, hear_ciphertext *const *in, hear_ciphertext **out, void *stream) {
    if (!mu || !in || !out) return fail(HEAR_E_INVAL, "null argument");
    size_t k = 0;
    for (size_t j = 0; j < mu->models.size(); j++)
        for (uint32_t i = 0; i < mu->n_ct[j]; i++, k++) {
            const hear_ciphertext *ct = in[k];
            if (!ct || ct->ctx != mu->models[j]->ctx) return fail(HEAR_E_STATE, "ciphertext from another context");
            if (ct->level != mu->level_in[j] || ct->n_poly != 2) return fail(HEAR_E_LEVEL, "input not at the job's level");
            if (ct->scale != mu->scale_in[j]) return fail(HEAR_E_SCALE, "input not at the job's scale");
        }
    hear_context *c0 = mu->models[0]->ctx;
    return guard(c0, [&] {
        cudaStream_t st = stream_of(c0, stream);
        HEAR_CHECK_CUDA(cudaStreamWaitEvent(st, mu->done, 0));
        size_t kk = 0;
        for (size_t j = 0; j < mu->models.size(); j++) {
            const uint64_t ctw = 2ull * (mu->level_in[j] + 1) * mu->models[j]->ctx->n;
            for (uint32_t i = 0; i < mu->n_ct[j]; i++, kk++)
                HEAR_CHECK_CUDA(cudaMemcpyAsync(mu->X[j].u64() + i * ctw, in[kk]->d.p, ctw * 8, cudaMemcpyDeviceToDevice, st));
        }
        HEAR_CHECK_CUDA(cudaGraphLaunch(mu->exec, st));
        g_launches += mu->launches;
        std::vector<std::unique_ptr<hear_ciphertext>> res;
        for (size_t j = 0; j < mu->models.size(); j++) {
            hear_context *c = mu->models[j]->ctx;
            const uint64_t otw = 2ull * (mu->level_out[j] + 1) * c->n;
            for (uint32_t i = 0; i < mu->n_ct[j]; i++) {
                res.emplace_back(new_ct(c, mu->level_out[j], 2, mu->scale_out[j], st));
                HEAR_CHECK_CUDA(cudaMemcpyAsync(res.back()->d.p, mu->Y[j].u64() + i * otw, otw * 8,
                                                cudaMemcpyDeviceToDevice, st));
            }
        }
        HEAR_CHECK_CUDA(cudaEventRecord(mu->done, st));
        for (size_t i = 0; i < res.size(); i++) out[i] = res[i].release();
    });
}

void hear_multi_destroy(hear_multi *mu) { delete mu; }

hear_status hear_evaluate_layer(const hear_model *m, size_t layer, const hear_eval_keys *evk,
                                hear_ciphertext *const *in, size_t n_ct, hear_ciphertext **out, void *stream) {
    if (!m || layer >= m->layers.size()) return fail(HEAR_E_INVAL, "bad layer index");
    return evaluate_range(m, layer, layer + 1, evk, in, n_ct, out, stream);
}

hear_status hear_evaluate_host(const hear_model *m, const hear_eval_keys *evk, const uint64_t *in_words, size_t n_ct,
                               double scale, uint64_t *out_words, size_t cap, size_t *n, uint32_t *level_out,
                               double *scale_out, void *stream) {
    if (!m || !evk || !in_words || n_ct == 0) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = m->ctx;
    const uint32_t lout_expect = m->layers.back().level_out;
    const size_t out_words_n = n_ct * 2ull * (lout_expect + 1) * c->n;
    if (n) *n = out_words_n;
    if (!out_words || cap < out_words_n) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        const uint32_t lin = m->layers[0].level_in;
        const uint64_t ctw = 2ull * (lin + 1) * c->n;
        if (use_graphs(c)) {
            std::lock_guard<std::mutex> g(m->plan_mu);
            // the graph takes the coefficient-domain input and gives the coefficient-domain
            // output: one H2D copy, one graph launch, one D2H copy
            hear_model::Plan *p = graph_plan(m, evk, 0, m->layers.size(), (uint32_t)n_ct, scale, st, 0, true);
            HEAR_CHECK_CUDA(cudaStreamWaitEvent(st, p->done, 0));
            HEAR_CHECK_CUDA(cudaMemcpyAsync(p->X.p, in_words, (size_t)n_ct * ctw * 8, cudaMemcpyHostToDevice, st));
            HEAR_CHECK_CUDA(cudaGraphLaunch(p->exec, st));
            g_launches += p->launches;
            HEAR_CHECK_CUDA(cudaMemcpyAsync(out_words, p->Y.p, out_words_n * 8, cudaMemcpyDeviceToHost, st));
            HEAR_CHECK_CUDA(cudaEventRecord(p->done, st));
            HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
            if (level_out) *level_out = p->level_out;
            if (scale_out) *scale_out = p->scale_out;
            return;
        }
        DevBuf X((size_t)n_ct * ctw * 8, st);
        to_device_ntt(c, in_words, lin, (uint32_t)(2 * n_ct), X.u64(), st);
        uint32_t lout;
        double sout;
        DevBuf Y = evaluate_batch(m, evk, 0, m->layers.size(), X.u64(), (uint32_t)n_ct, &lout, scale, &sout, st);
        ntt_inverse(c, Y.u64(), (uint32_t)(2 * n_ct) * (lout + 1), map_q(lout, c->n_q), st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out_words, Y.p, out_words_n * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
        if (level_out) *level_out = lout;
        if (scale_out) *scale_out = sout;
    });
}

hear_status hear_profile_begin(hear_context *ctx) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    return guard(ctx, [&] {
        std::lock_guard<std::mutex> g(ctx->prof.mu);
        ctx->prof.clear();
        ctx->prof.on = true;
    });
}

hear_status hear_profile_end(hear_context *ctx, hear_profile_entry *out, size_t cap, size_t *n) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    std::vector<hear_profile_entry> agg;
    hear_status s = guard(ctx, [&] {
        std::lock_guard<std::mutex> g(ctx->prof.mu);
        ctx->prof.on = false;
        std::map<std::string, size_t> idx;
        for (auto &r : ctx->prof.recs) {
            HEAR_CHECK_CUDA(cudaEventSynchronize(r.b));
            float ms = 0;
            HEAR_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
            auto it = idx.find(r.name);
            if (it == idx.end()) {
                hear_profile_entry e{};
                std::strncpy(e.name, r.name, sizeof(e.name) - 1);
                it = idx.emplace(r.name, agg.size()).first;
                agg.push_back(e);
            }
            hear_profile_entry &e = agg[it->second];
            e.launches += r.launches;
            e.total_ms += ms;
            e.bytes += r.bytes;
        }
        ctx->prof.clear();
    });
    if (s != HEAR_OK) return s;
    return copy_out(agg, out, cap, n);
}

uint64_t hear_launch_count(void) { return hear::g_launches.load(); }
uint64_t hear_pdl_launch_count(void) { return hear::g_pdl_launches.load(); }

hear_status hear_dbg_poly_mul(hear_context *ctx, uint32_t prime, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    if (!ctx || !a || !b || !out) return fail(HEAR_E_INVAL, "null argument");
    if (prime >= ctx->nqp()) return fail(HEAR_E_INVAL, "bad prime index");
    return guard(ctx, [&] {
        cudaStream_t st = ctx->stream;
        const uint32_t n = ctx->n;
        DevBuf d(3ull * n * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(d.p, a, n * 8, cudaMemcpyHostToDevice, st));
        HEAR_CHECK_CUDA(cudaMemcpyAsync(d.u64() + n, b, n * 8, cudaMemcpyHostToDevice, st));
        LimbMap m;
        m.per_group = 1;
        m.q_base = prime < ctx->n_q ? prime : 0;
        m.q_count = prime < ctx->n_q ? 1 : 0;
        m.n_q = ctx->n_q + (prime < ctx->n_q ? 0 : prime - ctx->n_q);
        ntt_forward(ctx, d.u64(), 2, m, st);
        // b -> Montgomery form, then a * b
        to_mont(ctx, d.u64() + n, 1, m, st);
        pointwise_mont(ctx, 1, m, d.u64(), d.u64() + n, d.u64() + 2 * n, st);
        ntt_inverse(ctx, d.u64() + 2 * n, 1, m, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, d.u64() + 2 * n, n * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_dbg_ntt_roundtrip(hear_context *ctx, uint64_t *limbs, size_t n_limb) {
    if (!ctx || !limbs || n_limb == 0) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] {
        cudaStream_t st = ctx->stream;
        const size_t words = n_limb * ctx->n;
        DevBuf d(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(d.p, limbs, words * 8, cudaMemcpyHostToDevice, st));
        LimbMap m;
        m.per_group = ctx->nqp();
        m.q_count = ctx->n_q;
        m.n_q = ctx->n_q;
        ntt_forward(ctx, d.u64(), (uint32_t)n_limb, m, st);
        ntt_inverse(ctx, d.u64(), (uint32_t)n_limb, m, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(limbs, d.p, words * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_ntt_tune(hear_context *ctx, uint32_t max_limbs, int iters, uint8_t *choice_out, float *ms_out) {
    if (!ctx || max_limbs == 0 || max_limbs > (1u << 15) || iters < 1) return fail(HEAR_E_INVAL, "bad argument");
    return guard(ctx, [&] {
        ntt_tune(ctx, max_limbs, iters, ms_out);
        if (choice_out) std::memcpy(choice_out, ctx->ntt_choice, sizeof(ctx->ntt_choice));
    });
}

hear_status hear_ntt_get_table(const hear_context *ctx, uint8_t *table) {
    if (!ctx || !table) return fail(HEAR_E_INVAL, "null argument");
    std::memcpy(table, ctx->ntt_choice, sizeof(ctx->ntt_choice));
    return HEAR_OK;
}

hear_status hear_ntt_set_table(hear_context *ctx, const uint8_t *table) {
    if (!ctx || !table) return fail(HEAR_E_INVAL, "null argument");
    for (int i = 0; i < 2 * kNttBuckets; i++)
        if (table[i] >= kNttVariants) return fail(HEAR_E_INVAL, "bad variant in table");
    std::memcpy(ctx->ntt_choice, table, sizeof(ctx->ntt_choice));
    return HEAR_OK;
}

hear_status hear_ks_tune(hear_context *ctx, uint32_t max_ct, int iters, uint8_t *choice_out, float *ms_out) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    return guard(ctx, [&] {
        if (ms_out) std::fill(ms_out, ms_out + kKsTables * kKsBuckets * kKsMaxForms, 0.0f);
        ks_tune(ctx, max_ct, iters, ms_out);
        if (choice_out) std::memcpy(choice_out, ctx->ks_choice, sizeof(ctx->ks_choice));
    });
}

hear_status hear_ks_get_table(const hear_context *ctx, uint8_t *table) {
    if (!ctx || !table) return fail(HEAR_E_INVAL, "null argument");
    std::memcpy(table, ctx->ks_choice, sizeof(ctx->ks_choice));
    return HEAR_OK;
}

hear_status hear_ks_set_table(hear_context *ctx, const uint8_t *table) {
    if (!ctx || !table) return fail(HEAR_E_INVAL, "null argument");
    for (int t = 0; t < kKsTables; t++)
        for (int b = 0; b < kKsBuckets; b++)
            if (table[t * kKsBuckets + b] >= kKsVariants[t]) return fail(HEAR_E_INVAL, "form out of range");
    std::memcpy(ctx->ks_choice, table, sizeof(ctx->ks_choice));
    return HEAR_OK;
}

hear_status hear_ks_set_variant(hear_context *ctx, int variant) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    if (variant < -1 || variant >= kKsMaxForms) return fail(HEAR_E_INVAL, "variant must be -1 or 0..7");
    ctx->ks_force = variant;
    return HEAR_OK;
}

hear_status hear_async_status(hear_context *ctx, uint32_t *timeouts) {
    if (!ctx) return fail(HEAR_E_INVAL, "null context");
    uint32_t v = 0;
    hear_status s = guard(ctx, [&] {
        HEAR_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
        v = async_timeouts(true);
    });
    if (timeouts) *timeouts = v;
    if (s != HEAR_OK) return s;
    return v ? fail(HEAR_E_TIMEOUT, std::to_string(v) + " bounded device wait(s) ran out") : HEAR_OK;
}

hear_status hear_dbg_wait_probe(hear_context *ctx, long long limit_cycles, uint32_t *timed_out) {
    if (!ctx || !timed_out || limit_cycles < 0) return fail(HEAR_E_INVAL, "bad argument");
    return guard(ctx, [&] { *timed_out = wait_probe(limit_cycles, ctx->stream); });
}

hear_status hear_ntt_set_variant(hear_context *ctx, int variant) {
    if (!ctx || variant < -1 || variant >= kNttVariants) return fail(HEAR_E_INVAL, "bad argument");
    ctx->ntt_force = variant;
    return HEAR_OK;
}

hear_status hear_dbg_ntt_time(hear_context *ctx, size_t n_limb, int iters, float *ms_fwd, float *ms_inv) {
    if (!ctx || n_limb == 0 || iters < 1 || !ms_fwd || !ms_inv) return fail(HEAR_E_INVAL, "bad argument");
    return guard(ctx, [&] {
        cudaStream_t st = ctx->stream;
        const size_t words = n_limb * ctx->n;
        DevBuf d(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemsetAsync(d.p, 0, words * 8, st));
        LimbMap m;
        m.per_group = ctx->nqp();
        m.q_count = ctx->n_q;
        m.n_q = ctx->n_q;
        cudaEvent_t e[3];
        for (auto &x : e) HEAR_CHECK_CUDA(cudaEventCreate(&x));
        ntt_forward(ctx, d.u64(), (uint32_t)n_limb, m, st);
        ntt_inverse(ctx, d.u64(), (uint32_t)n_limb, m, st);
        HEAR_CHECK_CUDA(cudaEventRecord(e[0], st));
        for (int i = 0; i < iters; i++) ntt_forward(ctx, d.u64(), (uint32_t)n_limb, m, st);
        HEAR_CHECK_CUDA(cudaEventRecord(e[1], st));
        for (int i = 0; i < iters; i++) ntt_inverse(ctx, d.u64(), (uint32_t)n_limb, m, st);
        HEAR_CHECK_CUDA(cudaEventRecord(e[2], st));
        HEAR_CHECK_CUDA(cudaEventSynchronize(e[2]));
        HEAR_CHECK_CUDA(cudaEventElapsedTime(ms_fwd, e[0], e[1]));
        HEAR_CHECK_CUDA(cudaEventElapsedTime(ms_inv, e[1], e[2]));
        *ms_fwd /= iters;
        *ms_inv /= iters;
        for (auto &x : e) cudaEventDestroy(x);
    });
}

}  // extern "C"

// ------------------------------------------------------------------ skeleton CNN
#include "cnn.h"

extern "C" {

hear_status hear_cnn_create(hear_context *ctx, const hear_cnn_input *input, const hear_cnn_layer *layers,
                            size_t n_layers, hear_cnn **out) {
    if (!ctx || !input || !layers || !out) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *out = cnn_create(ctx, input, layers, n_layers); });
}

void hear_cnn_destroy(hear_cnn *m) {
    if (!m) return;
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    delete m;
}

hear_status hear_cnn_rotations(const hear_cnn *m, int32_t *steps, size_t cap, size_t *n) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    return copy_out(m->rotations, steps, cap, n);
}

hear_status hear_cnn_ops(const hear_cnn *m, hear_cnn_op_info *ops, size_t cap, size_t *n) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    std::vector<hear_cnn_op_info> v;
    for (size_t k = 0; k < m->ops.size(); k++) {
        const hear_cnn::Op &op = m->ops[k];
        hear_cnn_op_info i{};
        i.kind = op.kind;
        i.layer = m->op_layer[k];
        i.n_in = op.n_in;
        i.n_out = op.n_out;
        i.level_in = op.level_in;
        i.level_out = op.level_out;
        i.n_babies = (uint32_t)op.babies.size();
        i.n_giants = (uint32_t)op.giants.size();
        if (op.kind == HEAR_CNN_OP_DIAG)
            i.n_keyswitch = op.n_in * (i.n_babies - 1) + op.n_out * (i.n_giants - 1);
        else if (op.kind == HEAR_CNN_OP_PACK)
            i.n_keyswitch = op.n_out * ((uint32_t)op.offs.size() - 1);
        else if (op.kind == HEAR_CNN_OP_ROTSUM)
            i.n_keyswitch = op.n_in * (uint32_t)op.steps.size();
        else if (op.kind == HEAR_CNN_OP_QUAD)
            i.n_keyswitch = op.n_in;
        v.push_back(i);
    }
    return copy_out(v, ops, cap, n);
}

hear_status hear_cnn_output_slots(const hear_cnn *m, uint32_t *slots, size_t cap, size_t *n) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    return copy_out(m->out_slots, slots, cap, n);
}

hear_status hear_cnn_encrypt(hear_context *ctx, const hear_public_key *pk, const hear_cnn *m, const double *x,
                             uint64_t seed, uint64_t ct_id, hear_ciphertext **out, void *stream) {
    if (!ctx || !pk || !m || !x || !out) return fail(HEAR_E_INVAL, "null argument");
    if (pk->ctx != ctx || m->ctx != ctx) return fail(HEAR_E_STATE, "handle from another context");
    if (m->ops.empty()) return fail(HEAR_E_STATE, "empty model");
    return guard(ctx, [&] {
        std::vector<double> z = cnn_pack_input(m, x);
        const size_t S = ctx->n / 2, n_ct = z.size() / S;
        std::vector<std::unique_ptr<hear_ciphertext>> res;
        for (size_t i = 0; i < n_ct; i++)
            res.emplace_back(encrypt_slots(ctx, pk, z.data() + i * S, ctx->default_scale, seed, ct_id + i,
                                           stream_of(ctx, stream)));
        for (size_t i = 0; i < n_ct; i++) out[i] = res[i].release();
    });
}

hear_status hear_cnn_evaluate(const hear_cnn *m, const hear_eval_keys *evk, size_t op0, size_t op1,
                              hear_ciphertext *const *in, size_t n_samples, hear_ciphertext **out, void *stream) {
    if (!m || !evk || !in || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = m->ctx;
    if (evk->ctx != c) return fail(HEAR_E_STATE, "key from another context");
    if (op0 >= op1 || op1 > m->ops.size()) return fail(HEAR_E_INVAL, "bad operation range");
    if (n_samples == 0 || n_samples > 65535) return fail(HEAR_E_INVAL, "n_samples must be in [1, 65535]");
    const hear_cnn::Op &first = m->ops[op0], &last = m->ops[op1 - 1];
    const uint32_t n_in = first.n_in, n_out = last.n_out, C = (uint32_t)n_samples;
    for (size_t k = 0; k < n_samples * n_in; k++) {
        if (!in[k] || in[k]->ctx != c) return fail(HEAR_E_STATE, "ciphertext from another context");
        if (in[k]->n_poly != 2 || in[k]->level != first.level_in)
            return fail(HEAR_E_LEVEL, "inputs must be 2-polynomial ciphertexts at the operation's level");
        if (in[k]->scale != in[0]->scale) return fail(HEAR_E_SCALE, "inputs at different scales");
    }
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        const uint64_t ctw = 2ull * (first.level_in + 1) * c->n;
        const uint64_t ctw_o = 2ull * (last.level_out + 1) * c->n;
        if (use_graphs(c)) {
            std::lock_guard<std::mutex> g(m->plan_mu);
            hear_cnn::Plan *p = cnn_graph_plan(m, evk, op0, op1, C, in[0]->scale, st);
            HEAR_CHECK_CUDA(cudaStreamWaitEvent(st, p->done, 0));
            for (uint32_t s = 0; s < C; s++)
                for (uint32_t i = 0; i < n_in; i++)
                    HEAR_CHECK_CUDA(cudaMemcpyAsync(p->X.u64() + ((uint64_t)i * C + s) * ctw,
                                                    in[(size_t)s * n_in + i]->d.p, ctw * 8,
                                                    cudaMemcpyDeviceToDevice, st));
            HEAR_CHECK_CUDA(cudaGraphLaunch(p->exec, st));
            g_launches += p->launches;
            std::vector<std::unique_ptr<hear_ciphertext>> res(n_out * (size_t)C);
            for (uint32_t s = 0; s < C; s++)
                for (uint32_t j = 0; j < n_out; j++) {
                    auto &h = res[(size_t)s * n_out + j];
                    h.reset(new_ct(c, last.level_out, 2, p->scale_out, st));
                    HEAR_CHECK_CUDA(cudaMemcpyAsync(h->d.p, p->Y.u64() + ((uint64_t)j * C + s) * ctw_o, ctw_o * 8,
                                                    cudaMemcpyDeviceToDevice, st));
                }
            HEAR_CHECK_CUDA(cudaEventRecord(p->done, st));
            for (size_t k = 0; k < res.size(); k++) out[k] = res[k].release();
            return;
        }
        DevBuf x((size_t)n_in * C * ctw * 8, st);
        for (uint32_t s = 0; s < C; s++)
            for (uint32_t i = 0; i < n_in; i++)
                HEAR_CHECK_CUDA(cudaMemcpyAsync(x.u64() + ((uint64_t)i * C + s) * ctw, in[(size_t)s * n_in + i]->d.p,
                                                ctw * 8, cudaMemcpyDeviceToDevice, st));
        double so = 0;
        DevBuf y = cnn_evaluate(m, evk, op0, op1, x.u64(), C, in[0]->scale, &so, st);
        std::vector<std::unique_ptr<hear_ciphertext>> res(n_out * (size_t)C);
        for (uint32_t s = 0; s < C; s++)
            for (uint32_t j = 0; j < n_out; j++) {
                auto &h = res[(size_t)s * n_out + j];
                h.reset(new_ct(c, last.level_out, 2, so, st));
                HEAR_CHECK_CUDA(cudaMemcpyAsync(h->d.p, y.u64() + ((uint64_t)j * C + s) * ctw_o, ctw_o * 8,
                                                cudaMemcpyDeviceToDevice, st));
            }
        for (size_t k = 0; k < res.size(); k++) out[k] = res[k].release();
    });
}

}  // extern "C"

// ------------------------------------------------------------------ slot-batched evaluation
#include "encode.h"

namespace {
hear_simd_batch *new_batch(hear_context *c, uint32_t n_ct, uint32_t level, double scale, cudaStream_t st) {
    auto b = std::make_unique<hear_simd_batch>();
    b->ctx = c;
    b->n_ct = n_ct;
    b->level = level;
    b->scale = scale;
    b->d = DevBuf((size_t)n_ct * 2 * (level + 1) * c->n * 8, st);
    return b.release();
}
void check_reduced(const hear_context *c, const uint64_t *words, size_t n_polys, uint32_t level) {
    for (size_t i = 0; i < n_polys * (level + 1); i++) {
        const uint64_t q = c->primes[i % (level + 1)];
        const uint64_t *w = words + i * c->n;
        for (uint32_t k = 0; k < c->n; k++) HEAR_REQUIRE(w[k] < q, HEAR_E_FORMAT, "residue not reduced");
    }
}
}  // namespace

extern "C" {

hear_status hear_simd_model_create(hear_context *ctx, const hear_layer_desc *layers, size_t n_layers,
                                   uint32_t level, hear_simd_model **out) {
    if (!ctx || !layers || !out) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *out = simd_model_create(ctx, layers, n_layers, level ? level : ctx->L); });
}

hear_status hear_simd_model_info(const hear_simd_model *m, uint32_t *d_in, uint32_t *d_out, uint32_t *level_in,
                                 uint32_t *level_out) {
    if (!m) return fail(HEAR_E_INVAL, "null model");
    if (d_in) *d_in = m->d_in;
    if (d_out) *d_out = m->d_out;
    if (level_in) *level_in = m->level_in;
    if (level_out) *level_out = m->level_out;
    return HEAR_OK;
}

void hear_simd_model_destroy(hear_simd_model *m) {
    if (m) cudaSetDevice(m->ctx->device);
    delete m;
}

hear_status hear_simd_encrypt(hear_context *ctx, const hear_public_key *pk, const double *x, size_t n_clips,
                              size_t n_features, double scale, uint64_t seed, uint32_t level, hear_simd_batch **out,
                              void *stream) {
    if (!ctx || !pk || !x || !out) return fail(HEAR_E_INVAL, "null argument");
    if (pk->ctx != ctx) return fail(HEAR_E_STATE, "key from another context");
    const size_t slots = ctx->n / 2;
    if (n_clips < 1 || n_clips > slots) return fail(HEAR_E_INVAL, "n_clips must be in [1, N/2]");
    if (n_features < 1 || n_features > (1u << 19)) return fail(HEAR_E_INVAL, "n_features must be in [1, 2^19]");
    const uint32_t lv = level ? level : ctx->L;
    if (lv > ctx->L) return fail(HEAR_E_LEVEL, "level above the top level");
    return guard(ctx, [&] {
        cudaStream_t st = stream_of(ctx, stream);
        const double sc = scale > 0 ? scale : ctx->default_scale;
        std::unique_ptr<hear_simd_batch> b(new_batch(ctx, (uint32_t)n_features, lv, sc, st));
        const uint64_t n = ctx->n, ctw = 2ull * (lv + 1) * n;
        // encode blocks of features on the host cores, then encrypt them one by one
        constexpr size_t kBlock = 64;
        std::vector<double> z(kBlock * slots), scales(kBlock, sc);
        std::vector<int64_t> m(kBlock * n);
        auto enc = encoder(ctx);
        for (size_t i0 = 0; i0 < n_features; i0 += kBlock) {
            const size_t cnt = std::min(kBlock, n_features - i0);
            std::fill(z.begin(), z.end(), 0.0);
            for (size_t f = 0; f < cnt; f++)
                for (size_t c = 0; c < n_clips; c++) z[f * slots + c] = x[c * n_features + i0 + f];
            encode_many(*enc, z.data(), cnt, scales.data(), m.data());
            for (size_t f = 0; f < cnt; f++) {
                const size_t i = i0 + f;
                std::unique_ptr<hear_ciphertext> ct(encrypt_encoded(ctx, pk, m.data() + f * n, sc, seed, i, st));
                // keep the limbs of the batch's level (no division: the scale is unchanged)
                HEAR_CHECK_CUDA(cudaMemcpy2DAsync(b->d.u64() + i * ctw, (size_t)(lv + 1) * n * 8, ct->d.p,
                                                  (size_t)(ct->level + 1) * n * 8, (size_t)(lv + 1) * n * 8, 2,
                                                  cudaMemcpyDeviceToDevice, st));
            }
        }
        *out = b.release();
    });
}

hear_status hear_simd_batch_info(const hear_simd_batch *b, uint32_t *n_ct, uint32_t *level, double *scale) {
    if (!b) return fail(HEAR_E_INVAL, "null batch");
    if (n_ct) *n_ct = b->n_ct;
    if (level) *level = b->level;
    if (scale) *scale = b->scale;
    return HEAR_OK;
}

hear_status hear_simd_batch_export(const hear_simd_batch *b, uint64_t *out, size_t cap, size_t *n) {
    if (!b) return fail(HEAR_E_INVAL, "null batch");
    hear_context *c = b->ctx;
    const size_t words = (size_t)b->n_ct * 2 * (b->level + 1) * c->n;
    if (n) *n = words;
    if (!out || cap < words) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = c->stream;
        DevBuf t(words * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(t.p, b->d.p, words * 8, cudaMemcpyDeviceToDevice, st));
        ntt_inverse(c, t.u64(), b->n_ct * 2 * (b->level + 1), map_q(b->level, c->n_q), st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

hear_status hear_simd_batch_import(hear_context *ctx, const uint64_t *words, size_t n_ct, uint32_t level,
                                   double scale, hear_simd_batch **out, void *stream) {
    if (!ctx || !words || !out || n_ct == 0) return fail(HEAR_E_INVAL, "null argument");
    if (level > ctx->L) return fail(HEAR_E_FORMAT, "bad level");
    return guard(ctx, [&] {
        check_reduced(ctx, words, 2 * n_ct, level);
        cudaStream_t st = stream_of(ctx, stream);
        std::unique_ptr<hear_simd_batch> b(new_batch(ctx, (uint32_t)n_ct, level, scale, st));
        to_device_ntt(ctx, words, level, (uint32_t)(2 * n_ct), b->d.u64(), st);
        *out = b.release();
    });
}

void hear_simd_batch_destroy(hear_simd_batch *b) {
    if (b) cudaSetDevice(b->ctx->device);
    delete b;
}

hear_status hear_simd_evaluate(const hear_simd_model *m, const hear_eval_keys *evk, const hear_simd_batch *in,
                               hear_simd_batch **out, void *stream) {
    if (!m || !evk || !in || !out) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = m->ctx;
    if (evk->ctx != c || in->ctx != c) return fail(HEAR_E_STATE, "keys or batch from another context");
    if (in->n_ct != m->d_in) return fail(HEAR_E_INVAL, "batch size differs from the model's input dimension");
    if (in->level != m->level_in) return fail(HEAR_E_LEVEL, "batch not at the model's input level");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        double so;
        DevBuf y = simd_evaluate(m, evk, in->d.u64(), in->scale, &so, st);
        auto b = std::make_unique<hear_simd_batch>();
        b->ctx = c;
        b->n_ct = m->d_out;
        b->level = m->level_out;
        b->scale = so;
        b->d = std::move(y);
        *out = b.release();
    });
}

hear_status hear_simd_evaluate_host(const hear_simd_model *m, const hear_eval_keys *evk, const uint64_t *in_words,
                                    double scale, uint64_t *out_words, size_t cap, size_t *n, uint32_t *level_out,
                                    double *scale_out, void *stream) {
    if (!m || !evk || !in_words) return fail(HEAR_E_INVAL, "null argument");
    hear_context *c = m->ctx;
    if (evk->ctx != c) return fail(HEAR_E_STATE, "keys from another context");
    const size_t out_n = (size_t)m->d_out * 2 * (m->level_out + 1) * c->n;
    if (n) *n = out_n;
    if (!out_words || cap < out_n) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(c, [&] {
        cudaStream_t st = stream_of(c, stream);
        DevBuf X((size_t)m->d_in * 2 * (m->level_in + 1) * c->n * 8, st);
        to_device_ntt(c, in_words, m->level_in, 2 * m->d_in, X.u64(), st);
        double so;
        DevBuf Y = simd_evaluate(m, evk, X.u64(), scale, &so, st);
        ntt_inverse(c, Y.u64(), 2 * m->d_out * (m->level_out + 1), map_q(m->level_out, c->n_q), st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(out_words, Y.p, out_n * 8, cudaMemcpyDeviceToHost, st));
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
        if (level_out) *level_out = m->level_out;
        if (scale_out) *scale_out = so;
    });
}

hear_status hear_dbg_round_scalar(double w, uint64_t q, int64_t *out) {
    if (!out || q == 0 || q >= (1ull << 62)) return fail(HEAR_E_INVAL, "bad argument");
    return guard(nullptr, [&] { *out = round_scalar(w, q); });
}

hear_status hear_dbg_imad_peak(hear_context *ctx, int kind, uint32_t iters, double *lane_ops_per_s) {
    if (!ctx || !lane_ops_per_s) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *lane_ops_per_s = imad_peak(ctx, kind, iters); });
}

hear_status hear_dbg_bfly_peak(hear_context *ctx, int inverse, uint32_t iters, double *butterflies_per_s) {
    if (!ctx || !butterflies_per_s) return fail(HEAR_E_INVAL, "null argument");
    return guard(ctx, [&] { *butterflies_per_s = bfly_peak(ctx, inverse == 0, iters); });
}

hear_status hear_simd_decrypt(hear_context *ctx, const hear_secret_key *sk, const hear_simd_batch *b,
                              size_t n_clips, double *out, size_t cap, size_t *n) {
    if (!ctx || !sk || !b) return fail(HEAR_E_INVAL, "null argument");
    if (b->ctx != ctx) return fail(HEAR_E_STATE, "batch from another context");
    if (n_clips < 1 || n_clips > ctx->n / 2) return fail(HEAR_E_INVAL, "n_clips must be in [1, N/2]");
    if (n) *n = n_clips * b->n_ct;
    if (!out || cap < n_clips * b->n_ct) return fail(HEAR_E_INVAL, "output capacity too small");
    return guard(ctx, [&] {
        cudaStream_t st = ctx->stream;
        const uint64_t ctw = 2ull * (b->level + 1) * ctx->n;
        std::vector<double> slots(ctx->n / 2);
        for (uint32_t o = 0; o < b->n_ct; o++) {
            std::unique_ptr<hear_ciphertext> ct(new_ct(ctx, b->level, 2, b->scale, st));
            HEAR_CHECK_CUDA(cudaMemcpyAsync(ct->d.p, b->d.u64() + o * ctw, ctw * 8, cudaMemcpyDeviceToDevice, st));
            decrypt_slots(ctx, sk, ct.get(), slots.data());
            for (size_t c = 0; c < n_clips; c++) out[c * b->n_ct + o] = slots[c];
        }
    });
}

}  // extern "C"
