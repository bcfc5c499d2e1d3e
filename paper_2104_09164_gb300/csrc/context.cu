// context.cu -- parameter set: prime chain, NTT twiddle tables, basis-conversion constants.
//
// RNS-CKKS (Methods, "Algorithmic and cryptographic optimizations": RNS variant of CKKS):
// Q = q_0 ... q_L word-size primes, special primes p_0..p_{K-1} for hybrid key switching
// with digits of alpha = K limbs.  Every prime is 1 mod 2N so that X^N + 1 splits and the
// negacyclic NTT exists.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <cstdlib>
#include "internal.h"
#include "hostmath.h"
#include "launch.cuh"

namespace hear {

// ------------------------------------------------------------------ device memory
thread_local const Allocator *tl_allocator = nullptr;

DevBuf::DevBuf(size_t b, cudaStream_t st) : bytes(b), s(st) {
    if (b == 0) return;
    if (const Allocator *a = tl_allocator) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (st && cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            (void)cudaGetLastError();
            cs = cudaStreamCaptureStatusNone;
        }
        if (cs == cudaStreamCaptureStatusNone) {
            p = a->alloc(b, static_cast<void *>(st), a->user);
            if (!p)
                throw Error(HEAR_E_NOMEM, std::string("the allocator returned no memory for ") + std::to_string(b) +
                                              " bytes");
            free_fn = a->free;
            free_user = a->user;
            return;
        }
    }
    cudaError_t e = st ? cudaMallocAsync(&p, b, st) : cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw Error(HEAR_E_NOMEM, std::string("device allocation of ") + std::to_string(b) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
}
void DevBuf::reset() {
    if (p) {
        if (free_fn) free_fn(p, static_cast<void *>(s), free_user);
        else if (s) cudaFreeAsync(p, s);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    free_fn = nullptr;
    free_user = nullptr;
}
DevBuf::~DevBuf() { reset(); }
DevBuf &DevBuf::operator=(DevBuf &&o) noexcept {
    if (this != &o) {
        reset();
        p = o.p; bytes = o.bytes; s = o.s; free_fn = o.free_fn; free_user = o.free_user;
        o.p = nullptr; o.bytes = 0; o.free_fn = nullptr; o.free_user = nullptr;
    }
    return *this;
}

std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_pdl_launches{0};

bool pdl_allowed(cudaStream_t st) {
    static const bool enabled = [] {
        const char *e = std::getenv("HEAR_PDL");
        return !(e && e[0] == '0');
    }();
    if (!enabled) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, &edges, &nd) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cs != cudaStreamCaptureStatusActive || nd == 0) return false;
    for (size_t i = 0; i < nd; i++) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(deps[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) {
            cudaGetLastError();
            return false;
        }
    }
    g_pdl_launches++;
    return true;
}

cudaEvent_t Profiler::get() {
    if (!spare.empty()) {
        cudaEvent_t e = spare.back();
        spare.pop_back();
        return e;
    }
    cudaEvent_t e;
    HEAR_CHECK_CUDA(cudaEventCreate(&e));
    return e;
}
void Profiler::clear() {
    for (auto &r : recs) {
        spare.push_back(r.a);
        spare.push_back(r.b);
    }
    recs.clear();
}

ProfScope::ProfScope(const hear_context *ctx, const char *nm, cudaStream_t st, double algo_bytes, uint32_t n_launch)
    : c(ctx), name(nm), s(st), bytes(algo_bytes), launches(n_launch) {
    g_launches += n_launch;
    if (c->prof.on) {
        std::lock_guard<std::mutex> g(c->prof.mu);
        a = c->prof.get();
        cudaEventRecord(a, s);
    }
}
ProfScope::~ProfScope() {
    if (a) {
        std::lock_guard<std::mutex> g(c->prof.mu);
        cudaEvent_t b = c->prof.get();
        cudaEventRecord(b, s);
        c->prof.recs.push_back(Profiler::Rec{name, a, b, bytes, launches});
    }
}

namespace {

uint32_t bitrev(uint32_t x, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// prime factors of n by trial division (n < 2^61)
std::vector<uint64_t> prime_factors(uint64_t n) {
    std::vector<uint64_t> f;
    for (uint64_t d = 2; d * d <= n; d += (d == 2 ? 1 : 2)) {
        if (n % d == 0) {
            f.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) f.push_back(n);
    return f;
}

// psi = g^((q-1)/2N) for the least generator g of Z_q^*
uint64_t root_2n(uint64_t q, uint64_t two_n) {
    auto fac = prime_factors(q - 1);
    for (uint64_t g = 2;; g++) {
        bool gen = true;
        for (uint64_t f : fac)
            if (hm::powmod(g, (q - 1) / f, q) == 1) { gen = false; break; }
        if (gen) return hm::powmod(g, (q - 1) / two_n, q);
    }
}

void push_pair(std::vector<uint64_t> &v, uint64_t w, uint64_t q) {
    v.push_back(w);
    v.push_back(hm::shoup_companion(w, q));
}

}  // namespace

// Discrete Gaussian CDT: S_k = 1 + 2 sum_{x=1..k} exp(-x^2/(2 sigma^2)) summed in double in
// increasing x; thresholds T_k = floor(S_k/S_B * 2^63) for k < B = floor(6 sigma), T_B = 2^63.
std::vector<uint64_t> make_cdt(double sigma) {
    int B = (int)std::floor(6.0 * sigma);
    B = std::max(1, std::min(B, 62));
    std::vector<double> S(B + 1);
    double acc = 1.0;
    S[0] = acc;
    for (int x = 1; x <= B; x++) {
        acc += 2.0 * std::exp(-((double)x * (double)x) / (2.0 * sigma * sigma));
        S[x] = acc;
    }
    std::vector<uint64_t> T(B + 1);
    for (int k = 0; k < B; k++) T[k] = (uint64_t)(S[k] / S[B] * 9223372036854775808.0);
    T[B] = 1ull << 63;
    return T;
}

void build_context(hear_context *c, const hear_params_desc *d, int device) {
    HEAR_REQUIRE(d && d->q_bits && d->p_bits, HEAR_E_INVAL, "null parameter description");
    HEAR_REQUIRE(d->log_n >= 11 && d->log_n <= 16, HEAR_E_UNSUPPORTED, "log_n must be in [11, 16]");
    HEAR_REQUIRE(d->n_q >= 1 && d->n_p >= 1 && d->n_q + d->n_p <= (uint32_t)kMaxPrimes, HEAR_E_UNSUPPORTED,
                 "need 1 <= n_q, 1 <= n_p, n_q + n_p <= 48");
    HEAR_REQUIRE(d->sigma > 0 && d->sigma < 10, HEAR_E_INVAL, "sigma out of range");
    c->device = device;
    std::memset(c->ntt_choice, kNttAuto, sizeof(c->ntt_choice));
    c->log_n = d->log_n;
    c->n = 1u << d->log_n;
    c->n_q = d->n_q;
    c->n_p = d->n_p;
    c->L = d->n_q - 1;
    c->K = d->n_p;
    // hybrid key switching: digits of alpha = K limbs (0 = that default); a digit modulus
    // larger than P would let the key-switching error grow by Q_j / P
    HEAR_REQUIRE(d->alpha == 0 || d->alpha == d->n_p, HEAR_E_UNSUPPORTED,
                 "alpha (limbs per key-switching digit) must equal n_p (or be 0 for that default)");
    c->alpha = d->n_p;
    c->default_scale = std::ldexp(1.0, 0) * std::pow(2.0, d->log2_scale);
    c->sigma = d->sigma;
    HEAR_CHECK_CUDA(cudaSetDevice(device));
    HEAR_CHECK_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    // keep freed stream-ordered memory cached in this process's pool (the default threshold
    // of zero hands it back at every synchronisation)
    HEAR_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&c->pool, device));
    uint64_t keep = ~0ull;
    HEAR_CHECK_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));

    // ---- primes: largest unused prime below 2^bits that is 1 mod 2N, chain order
    std::vector<uint32_t> bits(d->q_bits, d->q_bits + d->n_q);
    bits.insert(bits.end(), d->p_bits, d->p_bits + d->n_p);
    const uint64_t two_n = 2ull * c->n;
    for (uint32_t b : bits) {
        HEAR_REQUIRE(b >= c->log_n + 2 && b <= 60, HEAR_E_UNSUPPORTED, "prime bit size must be in [log_n+2, 60]");
        uint64_t top = 1ull << b, found = 0;
        for (uint64_t cand = top - two_n + 1; cand > two_n; cand -= two_n) {
            if (std::find(c->primes.begin(), c->primes.end(), cand) != c->primes.end()) continue;
            if (hm::is_prime(cand)) { found = cand; break; }
        }
        HEAR_REQUIRE(found, HEAR_E_UNSUPPORTED, "no prime of the requested size");
        c->primes.push_back(found);
    }
    const uint32_t np = c->nqp();
    const uint32_t n = c->n;

    // ---- per-prime constants and twiddle tables
    std::vector<DevPrime> dp(np);
    std::vector<uint64_t> tw(4ull * np * n);
    for (uint32_t i = 0; i < np; i++) {
        uint64_t q = c->primes[i];
        uint64_t psi = root_2n(q, two_n);
        c->psi.push_back(psi);
        uint64_t psi_inv = hm::invmod(psi, q);
        DevPrime &p = dp[i];
        p.q = q;
        p.qinv = hm::inv_2_64(q);
        uint64_t r1 = (uint64_t)(((hm::u128)1 << 64) % q);
        p.r2 = hm::mulmod(r1, r1, q);
        hm::u128 ratio = (~(hm::u128)0) / q;
        p.ratio_hi = (uint64_t)(ratio >> 64);
        p.ratio_lo = (uint64_t)ratio;
        p.n_inv = hm::invmod(n % q, q);
        p.n_inv_sh = hm::shoup_companion(p.n_inv, q);
        p.one_sh = hm::shoup_companion(1, q);
        // powers psi^k and psi^-k, k < N, stored at bit-reversed positions
        uint64_t *fw = &tw[(0ull * np + i) * n], *fs = &tw[(1ull * np + i) * n];
        uint64_t *iw = &tw[(2ull * np + i) * n], *is = &tw[(3ull * np + i) * n];
        uint64_t a = 1, b = 1;
        for (uint32_t k = 0; k < n; k++) {
            uint32_t r = bitrev(k, c->log_n);
            fw[r] = a;
            iw[r] = b;
            a = hm::mulmod(a, psi, q);
            b = hm::mulmod(b, psi_inv, q);
        }
        for (uint32_t k = 0; k < n; k++) {
            fs[k] = hm::shoup_companion(fw[k], q);
            is[k] = hm::shoup_companion(iw[k], q);
        }
    }
    c->d_primes = DevBuf(np * sizeof(DevPrime), nullptr);
    HEAR_CHECK_CUDA(cudaMemcpy(c->d_primes.p, dp.data(), np * sizeof(DevPrime), cudaMemcpyHostToDevice));
    c->d_tw = DevBuf(tw.size() * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemcpy(c->d_tw.p, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));

    c->cdt = make_cdt(c->sigma);
    c->d_cdt = DevBuf(c->cdt.size() * 8, nullptr);
    HEAR_CHECK_CUDA(cudaMemcpy(c->d_cdt.p, c->cdt.data(), c->cdt.size() * 8, cudaMemcpyHostToDevice));

    // ---- basis-conversion constants per level
    const uint32_t K = c->K, alpha = c->alpha;
    for (uint32_t l = 0; l <= c->L; l++) {
        auto lc = std::make_unique<LevelConsts>();
        const uint32_t L1 = l + 1, W = L1 + K, dnum = c->dnum(l);
        lc->level = l;
        lc->dnum = dnum;
        lc->width = W;
        auto prime_of = [&](uint32_t t) { return t < L1 ? c->primes[t] : c->primes[c->n_q + (t - L1)]; };
        std::vector<uint64_t> v;
        // ModUp: qhat_inv_i = [(Q_j/q_i)^-1]_{q_i}, qhat_mod = [Q_j/q_i]_t
        lc->off_qhat_inv = v.size();
        for (uint32_t i = 0; i < L1; i++) {
            uint32_t j = i / alpha, lo = j * alpha, hi = std::min(lo + alpha, L1);
            uint64_t q = c->primes[i], prod = 1;
            for (uint32_t i2 = lo; i2 < hi; i2++)
                if (i2 != i) prod = hm::mulmod(prod, c->primes[i2] % q, q);
            push_pair(v, hm::invmod(prod, q), q);
        }
        lc->off_qhat_mod = v.size();
        for (uint32_t j = 0; j < dnum; j++) {
            uint32_t lo = j * alpha, hi = std::min(lo + alpha, L1);
            for (uint32_t ii = 0; ii < alpha; ii++) {
                uint32_t i = lo + ii;
                for (uint32_t t = 0; t < W; t++) {
                    uint64_t pt = prime_of(t), prod = 1;
                    if (i < hi)
                        for (uint32_t i2 = lo; i2 < hi; i2++)
                            if (i2 != i) prod = hm::mulmod(prod, c->primes[i2] % pt, pt);
                    push_pair(v, i < hi ? prod : 0, pt);
                }
            }
        }
        // ModDown: phat_inv_k = [(P/p_k)^-1]_{p_k}, phat_mod[k][i] = [P/p_k]_{q_i}, P^-1 mod q_i
        lc->off_phat_inv = v.size();
        for (uint32_t k = 0; k < K; k++) {
            uint64_t pk = c->primes[c->n_q + k], prod = 1;
            for (uint32_t k2 = 0; k2 < K; k2++)
                if (k2 != k) prod = hm::mulmod(prod, c->primes[c->n_q + k2] % pk, pk);
            push_pair(v, hm::invmod(prod, pk), pk);
        }
        lc->off_phat_mod = v.size();
        for (uint32_t k = 0; k < K; k++)
            for (uint32_t i = 0; i < L1; i++) {
                uint64_t q = c->primes[i], prod = 1;
                for (uint32_t k2 = 0; k2 < K; k2++)
                    if (k2 != k) prod = hm::mulmod(prod, c->primes[c->n_q + k2] % q, q);
                push_pair(v, prod, q);
            }
        lc->off_p_inv = v.size();
        for (uint32_t i = 0; i < L1; i++) {
            uint64_t q = c->primes[i], prod = 1;
            for (uint32_t k = 0; k < K; k++) prod = hm::mulmod(prod, c->primes[c->n_q + k] % q, q);
            push_pair(v, hm::invmod(prod, q), q);
        }
        // rescale from level l: q_l^-1 mod q_i, i < l
        lc->off_ql_inv = v.size();
        for (uint32_t i = 0; i < l; i++) {
            uint64_t q = c->primes[i];
            push_pair(v, hm::invmod(c->primes[l] % q, q), q);
        }
        if (v.empty()) v.push_back(0);
        lc->d = DevBuf(v.size() * 8, nullptr);
        HEAR_CHECK_CUDA(cudaMemcpy(lc->d.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice));
        c->levels.push_back(std::move(lc));
    }
    HEAR_CHECK_CUDA(cudaDeviceSynchronize());
}

}  // namespace hear
