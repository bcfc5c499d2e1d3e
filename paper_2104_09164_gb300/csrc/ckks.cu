// ckks.cu -- RNS-CKKS key generation, encryption, decryption and the batched homomorphic
// operations the encrypted network is made of, composed from the kernels of ntt.cu and
// kernels.cu.  Everything between the host encode and the host CRT lift runs on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include "ckks.h"

namespace hear {

// randomness streams (purpose ids of the ChaCha20 nonce)
enum Purpose : uint32_t {
    kSk = 1, kPkA = 2, kPkE = 3, kKskA = 4, kKskE = 5, kEncV = 8, kEncE0 = 9, kEncE1 = 10
};

namespace {
std::mutex g_enc_mu;
std::map<hear_context *, std::shared_ptr<EncoderTables>> g_enc;

DevBuf upload(const void *host, size_t bytes, cudaStream_t st) {
    DevBuf b(bytes, st);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, st));
    return b;
}
}  // namespace

std::shared_ptr<EncoderTables> encoder(hear_context *ctx) {
    std::lock_guard<std::mutex> g(g_enc_mu);
    auto it = g_enc.find(ctx);
    if (it != g_enc.end()) return it->second;
    auto t = make_encoder_tables(ctx->log_n);
    g_enc[ctx] = t;
    return t;
}
void forget_encoder(hear_context *ctx) {
    std::lock_guard<std::mutex> g(g_enc_mu);
    g_enc.erase(ctx);
}

uint32_t galois_inverse(const hear_context *c, uint32_t g) {
    // the units of Z/2N form a group of order N, so g^(N-1) = g^-1
    return (uint32_t)hm::powmod(g, c->n - 1, 2ull * c->n);
}

uint32_t galois_of(const hear_context *c, int64_t step) {
    const int64_t slots = c->n / 2;
    int64_t r = ((step % slots) + slots) % slots;
    return (uint32_t)hm::powmod(5, (uint64_t)r, 2ull * c->n);
}

// ------------------------------------------------------------------ keys
void keygen(hear_context *c, uint64_t seed, const int32_t *steps, size_t n_steps, hear_secret_key **sk_out,
            hear_public_key **pk_out, hear_eval_keys **evk_out) {
    cudaStream_t st = c->stream;
    const uint32_t n = c->n, nqp = c->nqp(), nq = c->n_q;
    LimbMap all;   // every prime, in index order
    all.per_group = nqp;
    all.q_count = nq;
    all.n_q = nq;
    const LimbMap mq = map_q(c->L, nq);

    auto sk = std::make_unique<hear_secret_key>();
    sk->ctx = c;
    DevBuf s8(n, st);
    sample_small(c, seed, kSk, 0, kTernary, (int8_t *)s8.p, st);
    sk->s.resize(n);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(sk->s.data(), s8.p, n, cudaMemcpyDeviceToHost, st));
    DevBuf s_ntt((size_t)nqp * n * 8, st);
    small_to_limbs(c, (const int8_t *)s8.p, s_ntt.u64(), nqp, all, st);
    ntt_forward(c, s_ntt.u64(), nqp, all, st);
    sk->s_mont = DevBuf((size_t)nqp * n * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(sk->s_mont.p, s_ntt.p, (size_t)nqp * n * 8, cudaMemcpyDeviceToDevice, st));
    to_mont(c, sk->s_mont.u64(), nqp, all, st);

    // public key (b, a) = (-a s + e, a) over Q_L
    auto pk = std::make_unique<hear_public_key>();
    pk->ctx = c;
    pk->pk_mont = DevBuf(2ull * nq * n * 8, nullptr);
    uint64_t *pb = pk->pk_mont.u64(), *pa = pb + (size_t)nq * n;
    DevBuf e8(n, st), en((size_t)nqp * n * 8, st);
    sample_uniform(c, seed, kPkA, 0, pa, nq, mq, st);
    ntt_forward(c, pa, nq, mq, st);
    sample_small(c, seed, kPkE, 0, kGauss, (int8_t *)e8.p, st);
    small_to_limbs(c, (const int8_t *)e8.p, en.u64(), nq, mq, st);
    ntt_forward(c, en.u64(), nq, mq, st);
    pk_combine(c, pa, sk->s_mont.u64(), en.u64(), pb, st);
    LimbMap two_q = mq;
    to_mont(c, pb, 2 * nq, two_q, st);

    // switching keys: relinearisation (s^2) and one per rotation (sigma_g(s))
    auto evk = std::make_unique<hear_eval_keys>();
    evk->ctx = c;
    static std::atomic<uint64_t> serials{0};
    evk->serial = ++serials;
    std::vector<uint64_t> pmod(nqp, 0);
    for (uint32_t t = 0; t < nq; t++) {
        uint64_t v = 1;
        for (uint32_t k = 0; k < c->K; k++) v = hm::mulmod(v, c->primes[nq + k] % c->primes[t], c->primes[t]);
        pmod[t] = v;
    }
    DevBuf d_pmod = upload(pmod.data(), pmod.size() * 8, st);
    std::vector<uint32_t> gals{1u};
    std::set<uint32_t> seen{1u};
    for (size_t i = 0; i < n_steps; i++) {
        uint32_t g = galois_of(c, steps[i]);
        if (g != 1 && seen.insert(g).second) gals.push_back(g);
    }
    const uint32_t dnum = c->dnum_max();
    const size_t plane = (size_t)nqp * n;
    DevBuf sp((size_t)nqp * n * 8, st), a_tmp(plane * 8, st);
    for (uint32_t g : gals) {
        if (g == 1) pointwise_mont(c, nqp, all, s_ntt.u64(), sk->s_mont.u64(), sp.u64(), st);   // s^2
        else automorphism(c, nqp - 1, 1, g, s_ntt.u64(), sp.u64(), st);                          // sigma_g(s)
        to_mont(c, sp.u64(), nqp, all, st);
        DevBuf key((size_t)dnum * 2 * plane * 8, nullptr);
        for (uint32_t j = 0; j < dnum; j++) {
            uint64_t base = ((uint64_t)g << 16) | ((uint64_t)j << 8);
            uint64_t *kb = key.u64() + (size_t)j * 2 * plane, *ka = kb + plane;
            sample_uniform(c, seed, kKskA, base, ka, nqp, all, st);
            ntt_forward(c, ka, nqp, all, st);
            sample_small(c, seed, kKskE, base, kGauss, (int8_t *)e8.p, st);
            small_to_limbs(c, (const int8_t *)e8.p, en.u64(), nqp, all, st);
            ntt_forward(c, en.u64(), nqp, all, st);
            swk_combine(c, ka, sk->s_mont.u64(), en.u64(), sp.u64(), d_pmod.u64(), j, kb, st);
        }
        LimbMap km = all;
        to_mont(c, key.u64(), dnum * 2 * nqp, km, st);
        if (g != 1) {
            // stored sigma_g^{-1}-permuted: the inner product then reads keys and digits
            // coalesced and applies sigma_g to its output instead of to every digit
            DevBuf perm((size_t)dnum * 2 * plane * 8, nullptr);
            automorphism(c, nqp - 1, dnum * 2, galois_inverse(c, g), key.u64(), perm.u64(), st);
            key = std::move(perm);
        }
        evk->keys.emplace(g, std::move(key));
    }
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    *sk_out = sk.release();
    *pk_out = pk.release();
    *evk_out = evk.release();
}

// ------------------------------------------------------------------ encryption
hear_ciphertext *encrypt_slots(hear_context *c, const hear_public_key *pk, const double *z, double scale,
                               uint64_t seed, uint64_t ct_id, cudaStream_t st) {
    std::vector<int64_t> m(c->n);
    encode_dd(*encoder(c), z, scale, m.data());
    return encrypt_encoded(c, pk, m.data(), scale, seed, ct_id, st);
}

hear_ciphertext *encrypt_encoded(hear_context *c, const hear_public_key *pk, const int64_t *m, double scale,
                                 uint64_t seed, uint64_t ct_id, cudaStream_t st) {
    const uint32_t n = c->n, nq = c->n_q;
    const LimbMap mq = map_q(c->L, nq);
    DevBuf dm = upload(m, n * 8, st);
    const size_t limbs = (size_t)nq * n;
    DevBuf buf(4 * limbs * 8, st), e8(n, st);
    uint64_t *mn = buf.u64(), *vn = mn + limbs, *e0 = vn + limbs, *e1 = e0 + limbs;
    i64_to_limbs(c, (const int64_t *)dm.p, mn, nq, mq, st);
    sample_small(c, seed, kEncV, ct_id, kTernary, (int8_t *)e8.p, st);
    small_to_limbs(c, (const int8_t *)e8.p, vn, nq, mq, st);
    sample_small(c, seed, kEncE0, ct_id, kGauss, (int8_t *)e8.p, st);
    small_to_limbs(c, (const int8_t *)e8.p, e0, nq, mq, st);
    sample_small(c, seed, kEncE1, ct_id, kGauss, (int8_t *)e8.p, st);
    small_to_limbs(c, (const int8_t *)e8.p, e1, nq, mq, st);
    LimbMap four = mq;
    ntt_forward(c, mn, 4 * nq, four, st);
    auto ct = std::make_unique<hear_ciphertext>();
    ct->ctx = c;
    ct->level = c->L;
    ct->n_poly = 2;
    ct->scale = scale;
    ct->d = DevBuf(2 * limbs * 8, st);
    encrypt_combine(c, vn, e0, e1, mn, pk->pk_mont.u64(), ct->d.u64(), st);
    return ct.release();
}

void decrypt_slots(hear_context *c, const hear_secret_key *sk, const hear_ciphertext *ct, double *out) {
    cudaStream_t st = c->stream;
    const uint32_t n = c->n, L1 = ct->level + 1;
    DevBuf m((size_t)L1 * n * 8, st);
    decrypt_combine(c, ct->level, ct->d.u64(), sk->s_mont.u64(), m.u64(), st);
    ntt_inverse(c, m.u64(), L1, map_q(ct->level, c->n_q), st);
    std::vector<uint64_t> res((size_t)L1 * n);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(res.data(), m.p, res.size() * 8, cudaMemcpyDeviceToHost, st));
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<double> v(n);
    crt_to_double(res.data(), c->primes.data(), L1, n, 1.0 / ct->scale, v.data());
    decode_double(c->log_n, v.data(), out);
}

DevBuf encode_plain(hear_context *c, const double *z, double scale, uint32_t level, cudaStream_t st, bool mont) {
    const uint32_t n = c->n, L1 = level + 1;
    std::vector<int64_t> m(n);
    encode_dd(*encoder(c), z, scale, m.data());
    DevBuf dm = upload(m.data(), n * 8, st);
    DevBuf pt((size_t)L1 * n * 8, nullptr);
    i64_to_limbs(c, (const int64_t *)dm.p, pt.u64(), L1, map_q(level, c->n_q), st);
    ntt_forward(c, pt.u64(), L1, map_q(level, c->n_q), st);
    if (mont) to_mont(c, pt.u64(), L1, map_q(level, c->n_q), st);
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    return pt;
}

// ------------------------------------------------------------------ key switching compositions
namespace {
// device table of R jobs: key pointers, inverse galois elements, galois elements
struct JobTable {
    const uint64_t *d = nullptr;
    uint32_t R = 0;
    const uint64_t *const *keys() const { return reinterpret_cast<const uint64_t *const *>(d); }
    const uint32_t *ginv() const { return reinterpret_cast<const uint32_t *>(d + R); }
    const uint32_t *gal() const { return ginv() + R; }
};
JobTable make_jobs(hear_context *c, const std::vector<Rot> &rots, cudaStream_t st) {
    JobTable t;
    t.R = (uint32_t)rots.size();
    std::vector<uint64_t> host(t.R + (2 * t.R + 1) / 2, 0);
    uint32_t *g32 = reinterpret_cast<uint32_t *>(host.data() + t.R);
    for (uint32_t r = 0; r < t.R; r++) {
        host[r] = (uint64_t)(uintptr_t)rots[r].key;
        g32[r] = galois_inverse(c, rots[r].galois);
        g32[t.R + r] = rots[r].galois;
    }
    std::lock_guard<std::mutex> g(c->tab_mu);
    auto it = c->job_tables.find(host);
    if (it == c->job_tables.end()) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        HEAR_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
        HEAR_REQUIRE(cs == cudaStreamCaptureStatusNone, HEAR_E_STATE, "key-switch table missing during capture");
        DevBuf d(host.size() * 8, nullptr);
        HEAR_CHECK_CUDA(cudaMemcpy(d.p, host.data(), host.size() * 8, cudaMemcpyHostToDevice));
        it = c->job_tables.emplace(host, std::move(d)).first;
    }
    t.d = it->second.u64();
    return t;
}
}  // namespace

void rotate_hoisted(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *x, const std::vector<Rot> &rots,
                    uint64_t *out, cudaStream_t st) {
    if (rots.empty()) return;
    const uint32_t n = c->n, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level), R = (uint32_t)rots.size();
    const uint64_t plane = (uint64_t)L1 * n, ctw = 2 * plane;
    DevBuf ext((size_t)n_ct * dnum * W * n * 8, st), tmp((size_t)R * n_ct * ctw * 8, st),
        acc((size_t)R * n_ct * 2 * W * n * 8, st);
    modup(c, level, n_ct, x + plane, ctw, ext.u64(), tmp.u64(), st);
    JobTable jobs = make_jobs(c, rots, st);
    ks_inner(c, level, R, n_ct, ext.u64(), false, jobs.keys(), jobs.ginv(), acc.u64(), x + plane, ctw, st);
    moddown(c, level, R * n_ct, acc.u64(), out, x, ctw, 1u, true, jobs.gal(), n_ct, tmp.u64(), st);
}

void rotate_hoisted_ext(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *x, const std::vector<Rot> &rots,
                        uint64_t *out_ext, const uint64_t *pmod, cudaStream_t st) {
    if (rots.empty()) return;
    const uint32_t n = c->n, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level), R = (uint32_t)rots.size();
    const uint64_t plane = (uint64_t)L1 * n, ctw = 2 * plane;
    DevBuf ext((size_t)n_ct * dnum * W * n * 8, st), tmp((size_t)n_ct * plane * 8, st);
    modup(c, level, n_ct, x + plane, ctw, ext.u64(), tmp.u64(), st);
    JobTable jobs = make_jobs(c, rots, st);
    ks_inner(c, level, R, n_ct, ext.u64(), false, jobs.keys(), jobs.ginv(), out_ext, x + plane, ctw, st, pmod);
}

void rotate_each(hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *x,
                 const std::vector<Rot> &rots, uint64_t *out, cudaStream_t st) {
    const uint32_t n = c->n, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level), n_ct = R * C;
    const uint64_t plane = (uint64_t)L1 * n, ctw = 2 * plane;
    DevBuf ext((size_t)n_ct * dnum * W * n * 8, st), tmp((size_t)n_ct * ctw * 8, st),
        acc((size_t)n_ct * 2 * W * n * 8, st);
    modup(c, level, n_ct, x + plane, ctw, ext.u64(), tmp.u64(), st);
    JobTable jobs = make_jobs(c, rots, st);
    ks_inner(c, level, R, C, ext.u64(), true, jobs.keys(), jobs.ginv(), acc.u64(), x + plane, ctw, st);
    moddown(c, level, n_ct, acc.u64(), out, x, ctw, 1u, false, jobs.gal(), C, tmp.u64(), st);
}

void rotate_each_ext(hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *x,
                     const std::vector<Rot> &rots, uint64_t *out_ext, const uint64_t *pmod, cudaStream_t st) {
    const uint32_t n = c->n, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level), n_ct = R * C;
    const uint64_t plane = (uint64_t)L1 * n, ctw = 2 * plane;
    DevBuf ext((size_t)n_ct * dnum * W * n * 8, st), tmp((size_t)n_ct * plane * 8, st);
    modup(c, level, n_ct, x + plane, ctw, ext.u64(), tmp.u64(), st);
    JobTable jobs = make_jobs(c, rots, st);
    ks_inner(c, level, R, C, ext.u64(), true, jobs.keys(), jobs.ginv(), out_ext, x + plane, ctw, st, pmod);
}

void mul_relin(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *a, const uint64_t *b,
               const uint64_t *relin_key, uint64_t *out, cudaStream_t st) {
    const uint64_t plane = (uint64_t)(level + 1) * c->n;
    DevBuf d3((size_t)n_ct * 3 * plane * 8, st);
    tensor_ct(c, level, n_ct, a, b, d3.u64(), st);
    relin3(c, level, n_ct, d3.u64(), relin_key, out, st);
}

void relin3(hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *d3, const uint64_t *relin_key,
            uint64_t *out, cudaStream_t st) {
    const uint32_t n = c->n, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level);
    const uint64_t plane = (uint64_t)L1 * n;
    DevBuf ext((size_t)n_ct * dnum * W * n * 8, st), tmp((size_t)n_ct * 2 * plane * 8, st),
        acc((size_t)n_ct * 2 * W * n * 8, st);
    modup(c, level, n_ct, d3 + 2 * plane, 3 * plane, ext.u64(), tmp.u64(), st);
    JobTable jobs = make_jobs(c, {Rot{relin_key, 1u}}, st);
    ks_inner(c, level, 1, n_ct, ext.u64(), false, jobs.keys(), jobs.ginv(), acc.u64(), d3 + 2 * plane, 3 * plane,
             st);
    moddown(c, level, n_ct, acc.u64(), out, d3, 3 * plane, 3u, false, nullptr, 1, tmp.u64(), st);
}

// ------------------------------------------------------------------ network
namespace {

// rounds of the sum of `count` (a power of two) copies rho^(j*step*k): each round folds r =
// min(radix, remaining) copies with r - 1 rotations of one hoisted ModUp
std::vector<std::vector<int32_t>> rotsum_rounds(uint32_t step, uint32_t count, uint32_t k, uint32_t radix) {
    std::vector<std::vector<int32_t>> rounds;
    while (count > 1) {
        const uint32_t r = std::min(radix, count);
        std::vector<int32_t> round;
        for (uint32_t j = 1; j < r; j++) round.push_back((int32_t)(j * step * k));
        rounds.push_back(round);
        step *= r;
        count /= r;
    }
    return rounds;
}

void build_fc(hear_context *c, hear_model::Fc &fc, const double *W, uint32_t d_out, uint32_t d_in, uint32_t level,
              uint32_t k, uint32_t M, uint32_t radix, uint32_t n1_opt = 0, bool dh = false) {
    HEAR_REQUIRE(d_out && d_in && (d_out & (d_out - 1)) == 0 && (d_in & (d_in - 1)) == 0 && d_in % d_out == 0 &&
                     M % d_in == 0,
                 HEAR_E_INVAL, "FC dimensions must be powers of two with d_out | d_in | clip_dim");
    HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
    cudaStream_t st = c->stream;
    fc.d_out = d_out;
    fc.d_in = d_in;
    fc.D = d_out;
    fc.level = level;
    uint32_t n1 = 1;
    while (n1 * n1 < fc.D) n1 *= 2;
    if (n1_opt) n1 = n1_opt;
    n1 = std::min(n1, fc.D);
    fc.n1 = n1;
    fc.n2 = (fc.D + n1 - 1) / n1;
    fc.dh = dh;
    const uint32_t n = c->n, slots = n / 2, L1 = level + (dh ? 1 + c->K : 1);
    const LimbMap pmap = dh ? map_qp(level, c->n_q, c->K) : map_q(level, c->n_q);
    if (dh) {
        std::vector<uint64_t> pm;
        for (uint32_t t = 0; t <= level; t++) {
            const uint64_t q = c->primes[t];
            uint64_t v = 1;
            for (uint32_t kk = 0; kk < c->K; kk++) v = hm::mulmod(v, c->primes[c->n_q + kk] % q, q);
            pm.push_back(v);
            pm.push_back(hm::shoup_companion(v, q));
        }
        fc.pmod = DevBuf(pm.size() * 8, nullptr);
        HEAR_CHECK_CUDA(cudaMemcpy(fc.pmod.p, pm.data(), pm.size() * 8, cudaMemcpyHostToDevice));
    }
    const double ql = (double)c->primes[level];
    // diagonal plaintexts, pre-rotated by rho^(-j n1) (baby-step strategy re-association)
    std::vector<std::pair<uint32_t, uint32_t>> jobs;
    for (uint32_t j = 0; j < fc.n2; j++)
        for (uint32_t b = 0; b < n1; b++)
            if (j * n1 + b < fc.D) jobs.push_back({j, b});
    const uint64_t plane = (uint64_t)L1 * n;
    fc.pts = DevBuf((size_t)fc.n2 * n1 * plane * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemsetAsync(fc.pts.p, 0, fc.pts.bytes, st));
    auto enc = encoder(c);
    const size_t chunk = 64;
    std::vector<double> z;
    std::vector<int64_t> m;
    std::vector<double> scales;
    for (size_t s0 = 0; s0 < jobs.size(); s0 += chunk) {
        size_t cnt = std::min(chunk, jobs.size() - s0);
        z.assign(cnt * slots, 0.0);
        m.assign(cnt * n, 0);
        scales.assign(cnt, ql);
        for (size_t q = 0; q < cnt; q++) {
            uint32_t j = jobs[s0 + q].first, b = jobs[s0 + q].second, i = j * n1 + b;
            double *zz = &z[q * slots];
            for (uint32_t p = 0; p < M; p++) {
                uint32_t src = (p + M - (j * n1) % M) % M;       // rho^(-j n1)(diag_i)[p] = diag_i[p - j n1]
                double v = W[(size_t)(src % d_out) * d_in + (src + i) % d_in];
                for (uint32_t cc = 0; cc < k; cc++) zz[(size_t)p * k + cc] = v;
            }
        }
        encode_many(*enc, z.data(), cnt, scales.data(), m.data());
        DevBuf dm = upload(m.data(), m.size() * 8, st);
        for (size_t q = 0; q < cnt; q++) {
            uint32_t j = jobs[s0 + q].first, b = jobs[s0 + q].second;
            uint64_t *pt = fc.pts.u64() + ((size_t)j * n1 + b) * plane;
            i64_to_limbs(c, (const int64_t *)dm.p + q * n, pt, L1, pmap, st);
            ntt_forward(c, pt, L1, pmap, st);
            to_mont(c, pt, L1, pmap, st);
        }
        HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    fc.rotsum = rotsum_rounds(d_out, d_in / d_out, k, radix);
}

void fc_rotations(const hear_model::Fc &fc, uint32_t k, std::set<int32_t> &out) {
    for (uint32_t b = 1; b < fc.n1; b++) out.insert((int32_t)(b * k));
    for (uint32_t j = 1; j < fc.n2; j++) out.insert((int32_t)(j * fc.n1 * k));
    for (auto &round : fc.rotsum)
        for (int32_t s : round) out.insert(s);
}

const uint64_t *need_key(const hear_eval_keys *evk, uint32_t g) {
    const uint64_t *k = evk->key(g);
    HEAR_REQUIRE(k, HEAR_E_NOKEY, "missing switching key for galois element " + std::to_string(g));
    return k;
}

// rotate-and-sum in rounds: x <- x + sum_s rho^s(x) over the steps of each round, the
// rotations of a round sharing one ModUp of x (hoisting).  pmod (hoisted sums): each round
// is summed over Q_l u P -- P x + sum_s (P sigma_s(c0) + u0_s, u1_s) -- and ModDowned once.
void rotsum(hear_context *c, const hear_eval_keys *evk, uint32_t level, uint32_t n_ct, uint64_t *x,
            const std::vector<std::vector<int32_t>> &rounds, cudaStream_t st, const uint64_t *pmod = nullptr) {
    const uint32_t L1 = level + 1, W = L1 + c->K;
    const uint64_t ctw = 2ull * L1 * c->n, batch = (uint64_t)n_ct * ctw, batch_e = (uint64_t)n_ct * 2 * W * c->n;
    for (auto &round : rounds) {
        std::vector<Rot> rots;
        for (int32_t s : round) {
            uint32_t g = galois_of(c, s);
            rots.push_back(Rot{need_key(evk, g), g});
        }
        const uint32_t R = (uint32_t)rots.size();
        if (pmod) {
            // ModDown(P x + sum_s r_s) = x + ModDown(sum_s r_s): the sum is read by the ModDown
            DevBuf r((size_t)R * batch_e * 8, st), tmp((size_t)batch * 8, st);
            rotate_hoisted_ext(c, level, n_ct, x, rots, r.u64(), pmod, st);
            moddown(c, level, n_ct, r.u64(), x, x, ctw, 3u, false, nullptr, 1, tmp.u64(), st, R, batch_e);
            continue;
        }
        DevBuf r((size_t)R * batch * 8, st);
        rotate_hoisted(c, level, n_ct, x, rots, r.u64(), st);
        sum_add_ct(c, level, 2 * n_ct, r.u64(), batch, R, x, x, st);
    }
}

DevBuf eval_fc(const hear_model *m, const hear_model::Fc &fc, const hear_eval_keys *evk, const uint64_t *x,
               uint32_t n_ct, cudaStream_t st) {
    hear_context *c = m->ctx;
    const uint32_t level = fc.level, n = c->n, L1 = level + 1, n1 = fc.n1, n2 = fc.n2, k = m->k;
    const uint64_t ctw = 2ull * L1 * n, batch = (uint64_t)n_ct * ctw;
    std::vector<Rot> rots;
    for (uint32_t b = 1; b < n1; b++) {
        uint32_t g = galois_of(c, (int64_t)b * k);
        rots.push_back(Rot{need_key(evk, g), g});
    }
    // hoisted sums: the giant rotations stay over Q_l u P and are added to inner sum 0 there
    // (ModDowned once with them); pmod = ([P]_{q_t}, Shoup) for t <= level
    const uint64_t *pmod = m->hoist_sums ? m->pmod_all.u64() : nullptr;
    const uint32_t W = L1 + c->K;
    const uint64_t batch_e = (uint64_t)n_ct * 2 * W * n;
    DevBuf G((size_t)n2 * batch * 8, st);
    // hoisted sums: the giant rotations over Q_l u P in slots 1 .. n2-1 of Re (slot 0: inner
    // sum 0 over Q_l u P with hoisted ModDown of the babies), ModDowned together
    DevBuf Re;
    if (pmod && n2 > 1) Re = DevBuf((size_t)n2 * batch_e * 8, st);
    if (fc.dh) {
        // hoisted ModDown: the babies stay over Q_l u P (slot 0 = P x), the inner sums are
        // formed there with plaintexts over Q_l u P, and each giant-step sum is ModDowned
        // once (ModDown(P a + b) = a + ModDown(b))
        DevBuf babies((size_t)n1 * batch_e * 8, st);
        scale_p_ext(c, level, 2 * n_ct, x, babies.u64(), fc.pmod.u64(), st);
        rotate_hoisted_ext(c, level, n_ct, x, rots, babies.u64() + batch_e, fc.pmod.u64(), st);
        DevBuf Ge((size_t)n2 * batch_e * 8, st), tmp((size_t)n2 * batch * 8, st);
        lincomb_ext(c, level, n_ct, n1, n2, babies.u64(), fc.pts.u64(), Ge.u64(), st);
        if (pmod && n2 > 1) {
            // inner sums j >= 1 back to Q_l (they are rotated next); inner sum 0 stays extended
            moddown(c, level, (n2 - 1) * n_ct, Ge.u64() + batch_e, G.u64() + batch, nullptr, 0, 0u, false, nullptr, 1,
                    tmp.u64(), st);
            HEAR_CHECK_CUDA(cudaMemcpyAsync(Re.p, Ge.p, batch_e * 8, cudaMemcpyDeviceToDevice, st));
        } else {
            moddown(c, level, n2 * n_ct, Ge.u64(), G.u64(), nullptr, 0, 0u, false, nullptr, 1, tmp.u64(), st);
        }
    } else {
        // baby steps rho^(b k)(x), b < n1, hoisted; slot 0 holds x itself so that the inner
        // sums read one contiguous [n1][n_ct] batch
        DevBuf babies((size_t)n1 * batch * 8, st);
        HEAR_CHECK_CUDA(cudaMemcpyAsync(babies.p, x, batch * 8, cudaMemcpyDeviceToDevice, st));
        rotate_hoisted(c, level, n_ct, x, rots, babies.u64() + batch, st);
        // giant-step inner sums sum_b pt_{j,b} (.) baby_b (lazy: no rescale yet)
        lincomb(c, level, n_ct, n1, n2, babies.u64(), fc.pts.u64(), G.u64(), st);
    }
    // giant rotations rho^(j n1 k), j >= 1, of the un-rescaled sums, then accumulate
    if (n2 > 1) {
        std::vector<Rot> gr;
        for (uint32_t j = 1; j < n2; j++) {
            uint32_t g = galois_of(c, (int64_t)j * n1 * k);
            gr.push_back(Rot{need_key(evk, g), g});
        }
        if (pmod) {
            DevBuf tmp((size_t)batch * 8, st);
            rotate_each_ext(c, level, n2 - 1, n_ct, G.u64() + batch, gr, Re.u64() + batch_e, pmod, st);
            if (fc.dh)   // ModDown(inner sum 0 + sum_j r_j), inner sum 0 over Q_l u P in slot 0
                moddown(c, level, n_ct, Re.u64(), G.u64(), nullptr, 0, 0u, false, nullptr, 1, tmp.u64(), st, n2,
                        batch_e);
            else         // inner sum 0 over Q_l: G_0 + ModDown(sum_j r_j)
                moddown(c, level, n_ct, Re.u64() + batch_e, G.u64(), G.u64(), ctw, 3u, false, nullptr, 1, tmp.u64(),
                        st, n2 - 1, batch_e);
        } else {
            DevBuf R((size_t)(n2 - 1) * batch * 8, st);
            rotate_each(c, level, n2 - 1, n_ct, G.u64() + batch, gr, R.u64(), st);
            sum_add_ct(c, level, 2 * n_ct, R.u64(), batch, n2 - 1, G.u64(), G.u64(), st);
        }
    }
    // one rescale (lazy rescaling), then rotate-and-sum over the d_in / d_out blocks
    DevBuf Y((size_t)n_ct * 2 * level * n * 8, st), tmp((size_t)n_ct * 2 * level * n * 8, st);
    rescale(c, level, 2 * n_ct, G.u64(), Y.u64(), tmp.u64(), st);
    rotsum(c, evk, level - 1, n_ct, Y.u64(), fc.rotsum, st, pmod);
    return Y;
}

}  // namespace

hear_model *model_create(hear_context *c, const hear_layer_desc *layers, size_t n_layers, uint32_t clip_dim,
                         uint32_t start_level, uint32_t rotsum_radix, uint32_t fc_n1, bool hoist_moddown,
                         bool hoist_sums) {
    HEAR_REQUIRE(rotsum_radix >= 2 && (rotsum_radix & (rotsum_radix - 1)) == 0 && rotsum_radix <= 64, HEAR_E_INVAL,
                 "rotsum radix must be a power of two in [2, 64]");
    HEAR_REQUIRE(layers && n_layers > 0, HEAR_E_INVAL, "no layers");
    HEAR_REQUIRE(start_level >= 1 && start_level <= c->L, HEAR_E_LEVEL, "start level outside [1, L]");
    const uint32_t slots = c->n / 2;
    HEAR_REQUIRE(clip_dim && (clip_dim & (clip_dim - 1)) == 0 && clip_dim <= slots, HEAR_E_INVAL,
                 "clip_dim must be a power of two <= N/2");
    auto m = std::make_unique<hear_model>();
    m->ctx = c;
    m->clip_dim = clip_dim;
    m->rotsum_radix = rotsum_radix;
    m->fc_n1 = fc_n1;
    m->hoist_moddown = hoist_moddown;
    m->hoist_sums = hoist_sums;
    {
        // ([P]_{q_t}, Shoup) for every ciphertext prime (hoisted sums)
        std::vector<uint64_t> pm;
        for (uint32_t t = 0; t < c->n_q; t++) {
            const uint64_t q = c->primes[t];
            uint64_t v = 1;
            for (uint32_t kk = 0; kk < c->K; kk++) v = hm::mulmod(v, c->primes[c->n_q + kk] % q, q);
            pm.push_back(v);
            pm.push_back(hm::shoup_companion(v, q));
        }
        m->pmod_all = DevBuf(pm.size() * 8, nullptr);
        HEAR_CHECK_CUDA(cudaMemcpy(m->pmod_all.p, pm.data(), pm.size() * 8, cudaMemcpyHostToDevice));
    }
    m->k = slots / clip_dim;
    m->M = clip_dim;
    uint32_t level = start_level, dim = clip_dim;
    std::set<int32_t> rots;
    for (size_t li = 0; li < n_layers; li++) {
        const hear_layer_desc &d = layers[li];
        hear_model::Layer L;
        L.kind = d.kind;
        L.level_in = level;
        if (d.kind == HEAR_LAYER_FC) {
            HEAR_REQUIRE(d.w && d.d_in == dim, HEAR_E_INVAL, "FC input dimension mismatch");
            build_fc(c, L.fc, d.w, d.d_out, d.d_in, level, m->k, m->M, rotsum_radix, fc_n1, hoist_moddown);
            if (d.bias) {
                L.fc.bias.assign(d.bias, d.bias + d.d_out);
                for (double b : L.fc.bias) HEAR_REQUIRE(std::isfinite(b), HEAR_E_INVAL, "bias is not finite");
            }
            fc_rotations(L.fc, m->k, rots);
            level -= 1;
            dim = d.d_out;
        } else if (d.kind == HEAR_LAYER_SQUARE) {
            HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
            level -= 1;
        } else if (d.kind == HEAR_LAYER_FC_SQ_FC) {
            HEAR_REQUIRE(d.w && d.w2 && d.d_in == dim && li + 1 == n_layers, HEAR_E_INVAL,
                         "FC_SQ_FC must be the last layer and match the input dimension");
            HEAR_REQUIRE(level >= 2, HEAR_E_LEVEL, "not enough levels for the network");
            const uint32_t d1 = d.d_out, d2 = d.d_out2;
            build_fc(c, L.fc, d.w, d1, d.d_in, level, m->k, m->M, rotsum_radix);
            std::vector<double> U((size_t)d2 * d1 * d.d_in);
            for (uint32_t cc = 0; cc < d2; cc++)
                for (uint32_t r = 0; r < d1; r++)
                    for (uint32_t col = 0; col < d.d_in; col++)
                        U[((size_t)cc * d1 + r) * d.d_in + col] = d.w2[(size_t)cc * d1 + r] * d.w[(size_t)r * d.d_in + col];
            build_fc(c, L.fc2, U.data(), d2 * d1, d.d_in, level, m->k, m->M, rotsum_radix);
            fc_rotations(L.fc, m->k, rots);
            fc_rotations(L.fc2, m->k, rots);
            L.final_rotsum = rotsum_rounds(1, d1, m->k, rotsum_radix);
            for (auto &round : L.final_rotsum)
                for (int32_t s : round) rots.insert(s);
            level -= 2;
            for (uint32_t cc = 0; cc < d2; cc++) m->out_pos.push_back(cc * d1);
            dim = 0;
        } else {
            throw Error(HEAR_E_INVAL, "unknown layer kind");
        }
        L.level_out = level;
        m->layers.push_back(std::move(L));
    }
    if (m->out_pos.empty())
        for (uint32_t cc = 0; cc < dim; cc++) m->out_pos.push_back(cc);
    m->rotations.assign(rots.begin(), rots.end());
    return m.release();
}

namespace {
// the bias plaintext of FC layer li for an output at `scale`: b[p mod d_out] in every slot
// p*k + c, encoded at that scale with the output level's limbs (normal NTT form)
const uint64_t *bias_pt(const hear_model *m, size_t li, double scale, cudaStream_t st) {
    const hear_model::Fc &fc = m->layers[li].fc;
    uint64_t bits;
    std::memcpy(&bits, &scale, 8);
    std::lock_guard<std::mutex> g(m->bias_mu);
    auto key = std::make_pair(li, bits);
    auto it = m->bias_pts.find(key);
    if (it != m->bias_pts.end()) return it->second.u64();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HEAR_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    HEAR_REQUIRE(cs == cudaStreamCaptureStatusNone, HEAR_E_STATE, "bias plaintext missing during capture");
    hear_context *c = m->ctx;
    std::vector<double> z(c->n / 2);
    for (uint32_t p = 0; p < m->M; p++)
        for (uint32_t cc = 0; cc < m->k; cc++) z[(size_t)p * m->k + cc] = fc.bias[p % fc.d_out];
    DevBuf pt = encode_plain(c, z.data(), scale, m->layers[li].level_out, c->stream, false);
    return m->bias_pts.emplace(key, std::move(pt)).first->second.u64();
}
}  // namespace

DevBuf evaluate_batch(const hear_model *m, const hear_eval_keys *evk, size_t l0, size_t l1, const uint64_t *x,
                      uint32_t n_ct, uint32_t *level_out, double scale_in, double *scale_out, cudaStream_t st) {
    hear_context *c = m->ctx;
    const uint32_t n = c->n;
    {
        // every scale-dependent plaintext before the first launch (none inside a capture)
        double s = scale_in;
        for (size_t li = l0; li < l1; li++) {
            const hear_model::Layer &L = m->layers[li];
            if (L.kind == HEAR_LAYER_FC) {
                const double ql = (double)c->primes[L.fc.level];
                s = s * ql / ql;
                if (!L.fc.bias.empty()) bias_pt(m, li, s, st);
            } else if (L.kind == HEAR_LAYER_SQUARE) {
                s = s * s / (double)c->primes[L.level_in];
            } else {
                const double ql = (double)c->primes[L.fc.level], s1 = s * ql / ql;
                s = s1 * s1 / (double)c->primes[L.level_in - 1];
            }
        }
    }
    DevBuf cur;
    const uint64_t *xin = x;
    double scale = scale_in;
    uint32_t level = m->layers[l0].level_in;
    for (size_t li = l0; li < l1; li++) {
        const hear_model::Layer &L = m->layers[li];
        DevBuf next;
        if (L.kind == HEAR_LAYER_FC) {
            const double ql = (double)c->primes[L.fc.level];
            next = eval_fc(m, L.fc, evk, xin, n_ct, st);
            scale = scale * ql / ql;
            if (!L.fc.bias.empty())
                add_plain(c, L.level_out, n_ct, n_ct, next.u64(), bias_pt(m, li, scale, st), st);
        } else if (L.kind == HEAR_LAYER_SQUARE) {
            const uint64_t *rk = need_key(evk, 1);
            DevBuf prod((size_t)n_ct * 2 * (level + 1) * n * 8, st);
            mul_relin(c, level, n_ct, xin, xin, rk, prod.u64(), st);
            next = DevBuf((size_t)n_ct * 2 * level * n * 8, st);
            DevBuf tmp((size_t)n_ct * 2 * level * n * 8, st);
            rescale(c, level, 2 * n_ct, prod.u64(), next.u64(), tmp.u64(), st);
            scale = scale * scale / (double)c->primes[level];
        } else {
            const double ql = (double)c->primes[L.fc.level];
            DevBuf y = eval_fc(m, L.fc, evk, xin, n_ct, st);
            DevBuf u = eval_fc(m, L.fc2, evk, xin, n_ct, st);
            const double s1 = scale * ql / ql;
            const uint32_t lv = level - 1;
            const uint64_t *rk = need_key(evk, 1);
            DevBuf prod((size_t)n_ct * 2 * (lv + 1) * n * 8, st);
            mul_relin(c, lv, n_ct, y.u64(), u.u64(), rk, prod.u64(), st);
            next = DevBuf((size_t)n_ct * 2 * lv * n * 8, st);
            DevBuf tmp((size_t)n_ct * 2 * lv * n * 8, st);
            rescale(c, lv, 2 * n_ct, prod.u64(), next.u64(), tmp.u64(), st);
            scale = s1 * s1 / (double)c->primes[lv];
            rotsum(c, evk, lv - 1, n_ct, next.u64(), L.final_rotsum, st,
                   m->hoist_sums ? m->pmod_all.u64() : nullptr);
        }
        level = L.level_out;
        cur = std::move(next);
        xin = cur.u64();
    }
    *level_out = level;
    *scale_out = scale;
    return cur;
}

hear_model::Plan *graph_plan(const hear_model *m, const hear_eval_keys *evk, size_t l0, size_t l1, uint32_t n_ct,
                             double scale_in, cudaStream_t st, uint32_t slot, bool host_io) {
    for (auto &p : m->plans)
        if (p->evk_serial == evk->serial && p->l0 == l0 && p->l1 == l1 && p->n_ct == n_ct && p->scale_in == scale_in &&
            p->slot == slot && p->host_io == host_io)
            return p.get();
    hear_context *c = m->ctx;
    auto plan = std::make_unique<hear_model::Plan>();
    plan->evk_serial = evk->serial;
    plan->slot = slot;
    plan->host_io = host_io;
    plan->l0 = l0;
    plan->l1 = l1;
    plan->n_ct = n_ct;
    plan->scale_in = scale_in;
    const uint32_t lin = m->layers[l0].level_in;
    plan->level_out = m->layers[l1 - 1].level_out;
    const uint64_t in_words = (uint64_t)n_ct * 2 * (lin + 1) * c->n;
    const uint64_t out_words = (uint64_t)n_ct * 2 * (plan->level_out + 1) * c->n;
    plan->X = DevBuf(in_words * 8, nullptr);
    plan->Y = DevBuf(out_words * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemsetAsync(plan->X.p, 0, in_words * 8, st));
    {   // direct run: builds every key-switch table the capture will need
        uint32_t lo;
        double so;
        DevBuf y = evaluate_batch(m, evk, l0, l1, plan->X.u64(), n_ct, &lo, scale_in, &so, st);
    }
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    cudaStream_t cs;
    HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const uint64_t launches0 = g_launches.load();
    cudaGraph_t graph = nullptr;
    HEAR_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        uint32_t lo;
        double so;
        if (host_io) ntt_forward(c, plan->X.u64(), n_ct * 2 * (lin + 1), map_q(lin, c->n_q), cs);
        DevBuf y = evaluate_batch(m, evk, l0, l1, plan->X.u64(), n_ct, &lo, scale_in, &so, cs);
        plan->scale_out = so;
        if (host_io)
            ntt_inverse_from(c, y.u64(), (uint64_t)(lo + 1) * c->n, plan->Y.u64(), n_ct * 2 * (lo + 1),
                             map_q(lo, c->n_q), cs);
        else
            HEAR_CHECK_CUDA(cudaMemcpyAsync(plan->Y.p, y.p, out_words * 8, cudaMemcpyDeviceToDevice, cs));
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        throw;
    }
    HEAR_CHECK_CUDA(cudaStreamEndCapture(cs, &graph));
    plan->launches = g_launches.load() - launches0;
    cudaError_t e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    HEAR_CHECK_CUDA(e);
    HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&plan->done, cudaEventDisableTiming));
    m->plans.push_back(std::move(plan));
    return m->plans.back().get();
}

hear_multi *multi_create(const hear_model *const *models, const hear_eval_keys *const *evks, size_t n_jobs,
                         const uint32_t *n_ct, const double *scales, cudaStream_t st) {
    auto mu = std::make_unique<hear_multi>();
    for (size_t i = 0; i < n_jobs; i++) {
        const hear_model *m = models[i];
        hear_context *c = m->ctx;
        mu->models.push_back(m);
        mu->evks.push_back(evks[i]);
        mu->n_ct.push_back(n_ct[i]);
        mu->scale_in.push_back(scales[i]);
        mu->level_in.push_back(m->layers.front().level_in);
        mu->level_out.push_back(m->layers.back().level_out);
        const uint64_t in_words = (uint64_t)n_ct[i] * 2 * (mu->level_in[i] + 1) * c->n;
        const uint64_t out_words = (uint64_t)n_ct[i] * 2 * (mu->level_out[i] + 1) * c->n;
        mu->X.emplace_back(in_words * 8, nullptr);
        mu->Y.emplace_back(out_words * 8, nullptr);
        HEAR_CHECK_CUDA(cudaMemsetAsync(mu->X[i].p, 0, in_words * 8, st));
        uint32_t lo;
        double so;
        DevBuf y = evaluate_batch(m, evks[i], 0, m->layers.size(), mu->X[i].u64(), n_ct[i], &lo, scales[i], &so, st);
        mu->scale_out.push_back(so);
    }
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<cudaStream_t> cs(n_jobs, nullptr);
    std::vector<cudaEvent_t> ev(n_jobs, nullptr);
    auto cleanup = [&] {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        for (auto s : cs)
            if (s) cudaStreamDestroy(s);
    };
    cudaGraph_t graph = nullptr;
    try {
        for (size_t i = 0; i < n_jobs; i++) {
            HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking));
            HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        }
        const uint64_t launches0 = g_launches.load();
        HEAR_CHECK_CUDA(cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal));
        try {
            // fork: every job's stream joins the capture after its start, then runs its network
            HEAR_CHECK_CUDA(cudaEventRecord(ev[0], cs[0]));
            for (size_t i = 1; i < n_jobs; i++) HEAR_CHECK_CUDA(cudaStreamWaitEvent(cs[i], ev[0], 0));
            for (size_t i = 0; i < n_jobs; i++) {
                const hear_model *m = mu->models[i];
                uint32_t lo;
                double so;
                DevBuf y = evaluate_batch(m, mu->evks[i], 0, m->layers.size(), mu->X[i].u64(), mu->n_ct[i], &lo,
                                          mu->scale_in[i], &so, cs[i]);
                HEAR_CHECK_CUDA(cudaMemcpyAsync(mu->Y[i].p, y.p, mu->Y[i].bytes, cudaMemcpyDeviceToDevice, cs[i]));
            }
            // join
            for (size_t i = 1; i < n_jobs; i++) {
                HEAR_CHECK_CUDA(cudaEventRecord(ev[i], cs[i]));
                HEAR_CHECK_CUDA(cudaStreamWaitEvent(cs[0], ev[i], 0));
            }
        } catch (...) {
            cudaStreamEndCapture(cs[0], &graph);
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            throw;
        }
        HEAR_CHECK_CUDA(cudaStreamEndCapture(cs[0], &graph));
        mu->launches = g_launches.load() - launches0;
        cudaError_t e = cudaGraphInstantiate(&mu->exec, graph, 0);
        cudaGraphDestroy(graph);
        HEAR_CHECK_CUDA(e);
        HEAR_CHECK_CUDA(cudaEventCreateWithFlags(&mu->done, cudaEventDisableTiming));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    return mu.release();
}

}  // namespace hear

hear_multi::~hear_multi() {
    if (!models.empty()) cudaSetDevice(models.front()->ctx->device);
    if (done) cudaEventSynchronize(done);
    if (exec) cudaGraphExecDestroy(exec);
    if (done) cudaEventDestroy(done);
}

hear_model::Plan::~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (done) cudaEventDestroy(done);
}
