/*
 * hear_oracle.c -- plain, slow, obviously-correct CPU oracle for the RNS-CKKS hot path
 * of HEAR / Fast-HEAR (arXiv 2104.09164).  TEST INFRASTRUCTURE ONLY (see header).
 *
 * Everything here is written from the definitions:
 *   - RNS-CKKS (paper, Methods, "Algorithmic and cryptographic optimizations": the RNS
 *     variant of CKKS): limbs, NTT-based negacyclic products, hybrid key switching
 *     (ModUp -> inner product with the switching key -> ModDown), rescale by the last
 *     prime.
 *   - rotations rho^l (Methods, "Single-channel homomorphic convolutions"): Galois
 *     automorphism X -> X^g, g = 5^l mod 2N.
 *   - hoisting (Methods, "Algorithmic and cryptographic optimizations", item (i)):
 *     ModUp of c1 is shared by all rotations of one ciphertext; sigma_g is applied to
 *     the extended digits.
 * No blocking, fusion or reordering: each function does one mathematical step.
 */
#include "hear_oracle.h"
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ======================================================================== */
/* Modular arithmetic: Barrett reduction of a 128-bit product, mu = 2^128/q   */
/* ======================================================================== */
typedef struct { uint64_t q, mu_hi, mu_lo; } om_mod;

static om_mod om_make(uint64_t q)
{
    om_mod m;
    u128 mu = (~(u128)0) / q;     /* = floor(2^128/q) for odd q > 1 */
    m.q = q;
    m.mu_hi = (uint64_t)(mu >> 64);
    m.mu_lo = (uint64_t)mu;
    return m;
}

/* x < q^2 * 16 (q < 2^61): returns x mod q */
static inline uint64_t om_reduce(u128 x, const om_mod *m)
{
    uint64_t x0 = (uint64_t)x, x1 = (uint64_t)(x >> 64);
    u128 t = ((u128)x0 * m->mu_lo) >> 64;
    t += (u128)x0 * m->mu_hi;
    t += (u128)x1 * m->mu_lo;
    u128 qhat = (t >> 64) + (u128)x1 * m->mu_hi;   /* <= floor(x/q), short by at most 3 */
    uint64_t r = x0 - (uint64_t)qhat * m->q;
    while (r >= m->q) r -= m->q;
    return r;
}
static inline uint64_t om_mul(uint64_t a, uint64_t b, const om_mod *m)
{
    return om_reduce((u128)a * b, m);
}
static inline uint64_t om_add(uint64_t a, uint64_t b, uint64_t q)
{
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
static inline uint64_t om_sub(uint64_t a, uint64_t b, uint64_t q)
{
    return a >= b ? a - b : a + q - b;
}
static uint64_t om_pow(uint64_t a, uint64_t e, const om_mod *m)
{
    uint64_t r = 1 % m->q;
    a %= m->q;
    while (e) {
        if (e & 1) r = om_mul(r, a, m);
        a = om_mul(a, a, m);
        e >>= 1;
    }
    return r;
}
/* inverse by Fermat (q prime) */
static uint64_t om_inv(uint64_t a, const om_mod *m) { return om_pow(a, m->q - 2, m); }

uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q)
{
    om_mod m = om_make(q);
    return om_mul(a % q, b % q, &m);
}

/* ======================================================================== */
/* Primes                                                                   */
/* ======================================================================== */
static uint64_t pow_u128(uint64_t a, uint64_t e, uint64_t n)
{
    u128 r = 1, b = a % n;
    while (e) {
        if (e & 1) r = (r * b) % n;
        b = (b * b) % n;
        e >>= 1;
    }
    return (uint64_t)r;
}

/* deterministic Miller-Rabin, bases 2..37 (valid for all n < 3.3e24) */
int or_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = pow_u128(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = (uint64_t)(((u128)x * x) % n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

int or_gen_primes(uint32_t log_n, const uint32_t *bits, uint32_t count, uint64_t *out)
{
    uint64_t two_n = 2ull << log_n;
    for (uint32_t c = 0; c < count; c++) {
        if (bits[c] < log_n + 2 || bits[c] > 61) return -1;
        uint64_t top = 1ull << bits[c];
        uint64_t found = 0;
        for (uint64_t t = 1; two_n * t < top; t++) {
            uint64_t q = top - two_n * t + 1;
            int used = 0;
            for (uint32_t u = 0; u < c; u++) if (out[u] == q) used = 1;
            if (!used && or_is_prime(q)) { found = q; break; }
        }
        if (!found) return -2;
        out[c] = found;
    }
    return 0;
}

/* ======================================================================== */
/* Context                                                                  */
/* ======================================================================== */
#define OR_MAXP 64
#define OR_CDT_MAX 64

typedef struct {
    om_mod m;
    uint64_t psi, psi_inv, n_inv;
    uint64_t *psi_pow, *psi_inv_pow;   /* psi^k, psi^-k, k < N */
    uint64_t *om_pow, *om_inv_pow;     /* omega^k, omega^-k (omega = psi^2), k < N/2 */
} or_prime;

struct or_ctx {
    uint32_t log_n, n_q, n_p;
    size_t n;
    or_prime pr[OR_MAXP];
    double sigma;
    uint32_t cdt_n;                    /* thresholds for |e| = 0..cdt_n-1 */
    uint64_t cdt[OR_CDT_MAX];
};

static void prime_init(or_prime *p, uint64_t q, uint32_t log_n)
{
    size_t n = (size_t)1 << log_n;
    p->m = om_make(q);
    /* psi: the first x = 2,3,.. whose power x^((q-1)/2N) has order exactly 2N */
    uint64_t two_n = 2 * (uint64_t)n;
    for (uint64_t x = 2;; x++) {
        uint64_t g = om_pow(x, (q - 1) / two_n, &p->m);
        if (om_pow(g, n, &p->m) == q - 1) { p->psi = g; break; }
    }
    p->psi_inv = om_inv(p->psi, &p->m);
    p->n_inv = om_inv((uint64_t)n % q, &p->m);
    p->psi_pow = malloc(n * 8);
    p->psi_inv_pow = malloc(n * 8);
    p->om_pow = malloc(n / 2 * 8 + 8);
    p->om_inv_pow = malloc(n / 2 * 8 + 8);
    uint64_t a = 1, b = 1;
    for (size_t k = 0; k < n; k++) {
        p->psi_pow[k] = a; p->psi_inv_pow[k] = b;
        a = om_mul(a, p->psi, &p->m);
        b = om_mul(b, p->psi_inv, &p->m);
    }
    uint64_t w = om_mul(p->psi, p->psi, &p->m), wi = om_mul(p->psi_inv, p->psi_inv, &p->m);
    a = 1; b = 1;
    for (size_t k = 0; k < n / 2; k++) {
        p->om_pow[k] = a; p->om_inv_pow[k] = b;
        a = om_mul(a, w, &p->m);
        b = om_mul(b, wi, &p->m);
    }
}

/* CDT of the discrete Gaussian rho(x) = exp(-x^2/(2 sigma^2)) on |x| <= B, B = floor(6 sigma):
 * S_k = rho(0) + 2*sum_{x=1..k} rho(x) accumulated in double in increasing x,
 * T_k = floor(S_k / S_B * 2^63) for k < B and T_B = 2^63. */
static void cdt_init(or_ctx *c)
{
    int B = (int)floor(6.0 * c->sigma);
    if (B < 1) B = 1;
    if (B > OR_CDT_MAX - 1) B = OR_CDT_MAX - 1;
    double S[OR_CDT_MAX];
    double acc = 1.0;
    S[0] = acc;
    for (int x = 1; x <= B; x++) {
        double e = -((double)x * (double)x) / (2.0 * c->sigma * c->sigma);
        acc += 2.0 * exp(e);
        S[x] = acc;
    }
    for (int k = 0; k < B; k++) c->cdt[k] = (uint64_t)(S[k] / S[B] * 9223372036854775808.0);
    c->cdt[B] = 1ull << 63;
    c->cdt_n = (uint32_t)B + 1;
}

or_ctx *or_ctx_create(uint32_t log_n, uint32_t n_q, const uint32_t *q_bits,
                      uint32_t n_p, const uint32_t *p_bits, double sigma)
{
    if (log_n < 2 || log_n > 17 || n_q < 1 || n_p < 1 || n_q + n_p > OR_MAXP) return NULL;
    uint32_t bits[OR_MAXP];
    uint64_t primes[OR_MAXP];
    for (uint32_t i = 0; i < n_q; i++) bits[i] = q_bits[i];
    for (uint32_t i = 0; i < n_p; i++) bits[n_q + i] = p_bits[i];
    if (or_gen_primes(log_n, bits, n_q + n_p, primes) != 0) return NULL;
    or_ctx *c = calloc(1, sizeof(or_ctx));
    c->log_n = log_n; c->n = (size_t)1 << log_n; c->n_q = n_q; c->n_p = n_p;
    c->sigma = sigma;
    for (uint32_t i = 0; i < n_q + n_p; i++) prime_init(&c->pr[i], primes[i], log_n);
    cdt_init(c);
    return c;
}

void or_ctx_destroy(or_ctx *c)
{
    if (!c) return;
    for (uint32_t i = 0; i < c->n_q + c->n_p; i++) {
        free(c->pr[i].psi_pow); free(c->pr[i].psi_inv_pow);
        free(c->pr[i].om_pow); free(c->pr[i].om_inv_pow);
    }
    free(c);
}

int or_ctx_primes(const or_ctx *c, uint64_t *out)
{
    for (uint32_t i = 0; i < c->n_q + c->n_p; i++) out[i] = c->pr[i].m.q;
    return 0;
}
int or_ctx_psi(const or_ctx *c, uint64_t *out)
{
    for (uint32_t i = 0; i < c->n_q + c->n_p; i++) out[i] = c->pr[i].psi;
    return 0;
}
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* prime index of limb t of a polynomial over Q_l u P */
static inline uint32_t qp_prime(const or_ctx *c, uint32_t level, uint32_t t)
{
    return t <= level ? t : c->n_q + (t - level - 1);
}

/* ======================================================================== */
/* NTT, natural order: A[i] = sum_k a_k psi^((2i+1)k)                        */
/* (twist by psi^k, then a cyclic radix-2 DFT with omega = psi^2)            */
/* ======================================================================== */
static void bitrev_permute(uint64_t *a, size_t n)
{
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

static void cyclic_dft(uint64_t *a, size_t n, const uint64_t *wpow, const om_mod *m)
{
    bitrev_permute(a, n);
    for (size_t len = 2; len <= n; len <<= 1) {
        size_t half = len >> 1, step = n / len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = om_mul(a[i + j + half], wpow[j * step], m);
                a[i + j] = om_add(u, v, m->q);
                a[i + j + half] = om_sub(u, v, m->q);
            }
        }
    }
}

static void ntt_fwd_1(const or_ctx *c, uint32_t pi, uint64_t *a)
{
    const or_prime *p = &c->pr[pi];
    for (size_t k = 0; k < c->n; k++) a[k] = om_mul(a[k], p->psi_pow[k], &p->m);
    cyclic_dft(a, c->n, p->om_pow, &p->m);
}

static void ntt_inv_1(const or_ctx *c, uint32_t pi, uint64_t *a)
{
    const or_prime *p = &c->pr[pi];
    cyclic_dft(a, c->n, p->om_inv_pow, &p->m);
    for (size_t k = 0; k < c->n; k++)
        a[k] = om_mul(om_mul(a[k], p->n_inv, &p->m), p->psi_inv_pow[k], &p->m);
}

int or_ntt_fwd(const or_ctx *c, const uint32_t *prime, uint32_t n_limb, uint64_t *a)
{
    #pragma omp parallel for schedule(dynamic)
    for (uint32_t t = 0; t < n_limb; t++) ntt_fwd_1(c, prime[t], a + (size_t)t * c->n);
    return 0;
}
int or_ntt_inv(const or_ctx *c, const uint32_t *prime, uint32_t n_limb, uint64_t *a)
{
    #pragma omp parallel for schedule(dynamic)
    for (uint32_t t = 0; t < n_limb; t++) ntt_inv_1(c, prime[t], a + (size_t)t * c->n);
    return 0;
}

/* ======================================================================== */
/* ChaCha20 (RFC 8439 section 2.3) as a counter-based generator              */
/* key = seed (u64 LE) || 24 zero bytes, nonce = (purpose, index lo, index hi),  */
/* block counter = word / 8; word w = block words 2(w%8) | 2(w%8)+1 << 32.    */
/* ======================================================================== */
static inline uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }
#define QR(a, b, c, d) do { \
    a += b; d ^= a; d = rotl32(d, 16); c += d; b ^= c; b = rotl32(b, 12); \
    a += b; d ^= a; d = rotl32(d, 8);  c += d; b ^= c; b = rotl32(b, 7); } while (0)

void or_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3],
                       uint32_t out[16])
{
    uint32_t s[16], x[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) s[4 + i] = key[i];
    s[12] = counter;
    s[13] = nonce[0]; s[14] = nonce[1]; s[15] = nonce[2];
    memcpy(x, s, sizeof s);
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]); QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]); QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]); QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]); QR(x[3], x[4], x[9], x[14]);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

void or_stream_words(uint64_t seed, uint32_t purpose, uint64_t index, uint64_t w0,
                     size_t n, uint64_t *out)
{
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {purpose, (uint32_t)index, (uint32_t)(index >> 32)};
    uint32_t blk[16];
    uint64_t cur = ~0ull;
    for (size_t i = 0; i < n; i++) {
        uint64_t w = w0 + i;
        if (w / 8 != cur) { cur = w / 8; or_chacha20_block(key, (uint32_t)cur, nonce, blk); }
        uint32_t k = (uint32_t)(w % 8);
        out[i] = (uint64_t)blk[2 * k] | ((uint64_t)blk[2 * k + 1] << 32);
    }
}

int or_cdt_table(const or_ctx *c, uint64_t *out, uint32_t cap, uint32_t *n)
{
    *n = c->cdt_n;
    if (cap < c->cdt_n) return -1;
    for (uint32_t k = 0; k < c->cdt_n; k++) out[k] = c->cdt[k];
    return 0;
}

/* ternary: word mod 3 - 1 */
void or_sample_ternary(uint64_t seed, uint32_t purpose, uint64_t index, size_t n, int8_t *out)
{
    uint64_t *w = malloc(n * 8);
    or_stream_words(seed, purpose, index, 0, n, w);
    for (size_t k = 0; k < n; k++) out[k] = (int8_t)((int)(w[k] % 3) - 1);
    free(w);
}

/* discrete Gaussian by CDT inversion: u = w >> 1, |e| = min{k : u < T_k}, sign = w & 1 */
int or_sample_gauss(const or_ctx *c, uint64_t seed, uint32_t purpose, uint64_t index,
                    size_t n, int8_t *out)
{
    uint64_t *w = malloc(n * 8);
    or_stream_words(seed, purpose, index, 0, n, w);
    for (size_t k = 0; k < n; k++) {
        uint64_t u = w[k] >> 1;
        int mag = 0;
        while (!(u < c->cdt[mag])) mag++;
        out[k] = (int8_t)((w[k] & 1) ? -mag : mag);
    }
    free(w);
    return 0;
}

/* uniform mod q: (w_{2k+1} * 2^64 + w_{2k}) mod q */
void or_sample_uniform(uint64_t seed, uint32_t purpose, uint64_t index, uint64_t q,
                       size_t n, uint64_t *out)
{
    uint64_t *w = malloc(2 * n * 8);
    or_stream_words(seed, purpose, index, 0, 2 * n, w);
    for (size_t k = 0; k < n; k++) {
        u128 x = ((u128)w[2 * k + 1] << 64) | w[2 * k];
        out[k] = (uint64_t)(x % q);
    }
    free(w);
}

/* purpose ids of the randomness streams */
enum { P_SK = 1, P_PK_A = 2, P_PK_E = 3, P_KSK_A = 4, P_KSK_E = 5,
       P_ENC_V = 8, P_ENC_E0 = 9, P_ENC_E1 = 10 };

/* ======================================================================== */
/* Double-double arithmetic (hi + lo, ~106-bit significand)                  */
/* ======================================================================== */
typedef struct { double hi, lo; } dd;

static inline dd dd_two_sum(double a, double b)
{
    dd r; r.hi = a + b; double bb = r.hi - a;
    r.lo = (a - (r.hi - bb)) + (b - bb);
    return r;
}
static inline dd dd_quick(double a, double b)
{
    dd r; r.hi = a + b; r.lo = b - (r.hi - a);
    return r;
}
static inline dd dd_two_prod(double a, double b)
{
    dd r; r.hi = a * b; r.lo = fma(a, b, -r.hi);
    return r;
}
static inline dd dd_add(dd a, dd b)
{
    dd s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi; s = dd_quick(s.hi, s.lo);
    s.lo += t.lo; return dd_quick(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { a.hi = -a.hi; a.lo = -a.lo; return a; }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_mul(dd a, dd b)
{
    dd p = dd_two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return dd_quick(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b)
{
    dd p = dd_two_prod(a.hi, b);
    p.lo += a.lo * b;
    return dd_quick(p.hi, p.lo);
}
static inline dd dd_div_d(dd a, double b)
{
    double q1 = a.hi / b;
    dd p = dd_two_prod(q1, b);
    double r = ((a.hi - p.hi) - p.lo + a.lo) / b;
    return dd_quick(q1, r);
}
static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }

/* 2*pi as a double-double */
static const dd DD_2PI = {6.283185307179586232e+00, 2.449293598294706414e-16};

/* Taylor series of sin and cos on |x| <= pi/4 */
static void dd_taylor_sincos(dd x, dd *s, dd *c)
{
    dd x2 = dd_mul(x, x);
    dd term = x, sum = x;
    for (int k = 1; k < 40; k++) {
        term = dd_div_d(dd_mul(term, x2), (double)((2 * k) * (2 * k + 1)));
        term = dd_neg(term);
        sum = dd_add(sum, term);
        if (fabs(term.hi) < 1e-36) break;
    }
    *s = sum;
    term = dd_from(1.0); sum = term;
    for (int k = 1; k < 40; k++) {
        term = dd_div_d(dd_mul(term, x2), (double)((2 * k - 1) * (2 * k)));
        term = dd_neg(term);
        sum = dd_add(sum, term);
        if (fabs(term.hi) < 1e-36) break;
    }
    *c = sum;
}

/* cos and sin of 2*pi*m/M for a power of two M >= 8, by exact octant reduction of m */
static void dd_cossin(uint64_t m, uint64_t M, dd *c, dd *s)
{
    m %= M;
    uint64_t quarter = M / 4, eighth = M / 8;
    uint64_t qd = m / quarter, r = m % quarter;
    int swap = 0;
    if (r > eighth) { r = quarter - r; swap = 1; }
    dd x = dd_mul_d(DD_2PI, (double)r / (double)M);
    dd sx, cx;
    dd_taylor_sincos(x, &sx, &cx);
    if (swap) { dd t = sx; sx = cx; cx = t; }
    switch (qd) {
    case 0: *c = cx; *s = sx; break;
    case 1: *c = dd_neg(sx); *s = cx; break;
    case 2: *c = dd_neg(cx); *s = dd_neg(sx); break;
    default: *c = sx; *s = dd_neg(cx); break;
    }
}

void or_dd_cossin(uint64_t m, uint64_t M, double *c_hi, double *c_lo, double *s_hi, double *s_lo)
{
    dd c, s;
    dd_cossin(m, M, &c, &s);
    *c_hi = c.hi; *c_lo = c.lo; *s_hi = s.hi; *s_lo = s.lo;
}

/* complex dd */
typedef struct { dd re, im; } cdd;
static inline cdd cdd_mul(cdd a, cdd b)
{
    cdd r;
    r.re = dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
    r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
    return r;
}
static inline cdd cdd_add(cdd a, cdd b) { cdd r = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return r; }
static inline cdd cdd_sub(cdd a, cdd b) { cdd r = {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; return r; }

/* in-place forward DFT F[k] = sum_t A[t] e^{-2 pi i t k / M}, radix-2, M power of two */
static void cdd_dft(cdd *a, size_t M)
{
    for (size_t i = 1, j = 0; i < M; i++) {
        size_t bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cdd t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    cdd *w = malloc(M / 2 * sizeof(cdd));
    for (size_t k = 0; k < M / 2; k++) {
        dd c, s;
        dd_cossin(k, M, &c, &s);
        w[k].re = c; w[k].im = dd_neg(s);        /* e^{-2 pi i k / M} */
    }
    for (size_t len = 2; len <= M; len <<= 1) {
        size_t half = len / 2, step = M / len;
        for (size_t i = 0; i < M; i += len)
            for (size_t j = 0; j < half; j++) {
                cdd u = a[i + j], v = cdd_mul(a[i + j + half], w[j * step]);
                a[i + j] = cdd_add(u, v);
                a[i + j + half] = cdd_sub(u, v);
            }
    }
    free(w);
}

/* Encoding: slot j <-> root zeta^(5^j mod 2N), zeta = e^{i pi / N} (real slot values).
 * tau^-1: m_k = (1/N) sum_{t odd} A[t] zeta^{-t k} with A[5^j] = A[2N - 5^j] = z_j,
 * computed as a length-2N DFT in double-double; then round half away from zero of
 * scale * m_k. */
int or_encode(const or_ctx *c, const double *z, double scale, int64_t *m_out, int *near_ties)
{
    size_t n = c->n, M = 2 * n;
    cdd *a = calloc(M, sizeof(cdd));
    uint64_t t = 1;
    for (size_t j = 0; j < n / 2; j++) {
        a[t].re = dd_from(z[j]);
        a[M - t].re = dd_from(z[j]);
        t = (t * 5) % M;
    }
    cdd_dft(a, M);
    int ties = 0;
    double f = scale / (double)n;   /* exact: n is a power of two */
    for (size_t k = 0; k < n; k++) {
        dd v = dd_mul_d(a[k].re, f);
        double fl = floor(v.hi);
        double frac = (v.hi - fl) + v.lo;
        while (frac >= 1.0) { fl += 1.0; frac -= 1.0; }
        while (frac < 0.0) { fl -= 1.0; frac += 1.0; }
        if (fabs(frac - 0.5) < 0x1p-30) ties++;
        double r;
        if (frac > 0.5) r = fl + 1.0;
        else if (frac < 0.5) r = fl;
        else r = (fl >= 0.0) ? fl + 1.0 : fl;   /* tie: away from zero */
        m_out[k] = (int64_t)r;
    }
    free(a);
    if (near_ties) *near_ties = ties;
    return 0;
}

/* ======================================================================== */
/* Ring helpers                                                             */
/* ======================================================================== */
static inline uint64_t signed_mod(int64_t v, uint64_t q)
{
    if (v >= 0) return (uint64_t)v % q;
    uint64_t r = (uint64_t)(-(v + 1)) % q;      /* avoids overflow at INT64_MIN */
    return q - 1 - r;
}

/* small integer polynomial -> NTT-domain limbs for the listed primes */
static void small_to_ntt(const or_ctx *c, const int8_t *e, const uint32_t *prime,
                         uint32_t n_limb, uint64_t *out)
{
    for (uint32_t t = 0; t < n_limb; t++) {
        uint64_t q = c->pr[prime[t]].m.q;
        for (size_t k = 0; k < c->n; k++) out[(size_t)t * c->n + k] = signed_mod(e[k], q);
    }
    or_ntt_fwd(c, prime, n_limb, out);
}

int or_to_coeff(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out)
{
    uint32_t L1 = level + 1;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) pr[t] = t;
    memcpy(out, in, (size_t)n_poly * L1 * c->n * 8);
    for (uint32_t p = 0; p < n_poly; p++) or_ntt_inv(c, pr, L1, out + (size_t)p * L1 * c->n);
    return 0;
}
int or_from_coeff(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out)
{
    uint32_t L1 = level + 1;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) pr[t] = t;
    memcpy(out, in, (size_t)n_poly * L1 * c->n * 8);
    for (uint32_t p = 0; p < n_poly; p++) or_ntt_fwd(c, pr, L1, out + (size_t)p * L1 * c->n);
    return 0;
}

int or_encode_pt(const or_ctx *c, uint32_t level, const int64_t *m, uint64_t *pt)
{
    uint32_t L1 = level + 1;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) {
        pr[t] = t;
        uint64_t q = c->pr[t].m.q;
        for (size_t k = 0; k < c->n; k++) pt[(size_t)t * c->n + k] = signed_mod(m[k], q);
    }
    or_ntt_fwd(c, pr, L1, pt);
    return 0;
}

/* ======================================================================== */
/* Keys                                                                     */
/* ======================================================================== */
int or_keygen_sk(const or_ctx *c, uint64_t seed, int8_t *s_out)
{
    or_sample_ternary(seed, P_SK, 0, c->n, s_out);
    return 0;
}

int or_sk_ntt(const or_ctx *c, const int8_t *s, uint64_t *out)
{
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < c->n_q + c->n_p; t++) pr[t] = t;
    small_to_ntt(c, s, pr, c->n_q + c->n_p, out);
    return 0;
}

/* pk = (-a*s + e, a) over Q_L */
int or_keygen_pk(const or_ctx *c, uint64_t seed, const int8_t *s, uint64_t *pk)
{
    size_t n = c->n;
    uint32_t L1 = c->n_q;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) pr[t] = t;
    uint64_t *sn = malloc((size_t)L1 * n * 8), *en = malloc((size_t)L1 * n * 8);
    int8_t *e = malloc(n);
    small_to_ntt(c, s, pr, L1, sn);
    or_sample_gauss(c, seed, P_PK_E, 0, n, e);
    small_to_ntt(c, e, pr, L1, en);
    uint64_t *b = pk, *a = pk + (size_t)L1 * n;
    for (uint32_t t = 0; t < L1; t++) or_sample_uniform(seed, P_PK_A, t, c->pr[t].m.q, n, a + (size_t)t * n);
    or_ntt_fwd(c, pr, L1, a);
    for (uint32_t t = 0; t < L1; t++) {
        const om_mod *m = &c->pr[t].m;
        for (size_t k = 0; k < n; k++) {
            size_t i = (size_t)t * n + k;
            b[i] = om_add(om_sub(0, om_mul(a[i], sn[i], m), m->q), en[i], m->q);
        }
    }
    free(sn); free(en); free(e);
    return 0;
}

uint32_t or_dnum(const or_ctx *c, uint32_t level)
{
    uint32_t alpha = c->n_p;
    return (level + 1 + alpha - 1) / alpha;
}

/* sigma_g on a coefficient-domain integer polynomial: a(X) -> a(X^g) in Z[X]/(X^N+1) */
static void small_automorphism(const or_ctx *c, uint32_t g, const int8_t *in, int8_t *out)
{
    size_t n = c->n;
    uint64_t two_n = 2 * n;
    for (size_t k = 0; k < n; k++) {
        uint64_t e = ((uint64_t)k * g) % two_n;
        if (e < n) out[e] = in[k];
        else out[e - n] = (int8_t)(-in[k]);
    }
}

int or_keygen_swk(const or_ctx *c, uint64_t seed, const int8_t *s, uint32_t galois, uint64_t *out)
{
    size_t n = c->n;
    uint32_t nqp = c->n_q + c->n_p, alpha = c->n_p, dnum = or_dnum(c, c->n_q - 1);
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < nqp; t++) pr[t] = t;
    size_t limbs = (size_t)nqp * n;
    uint64_t *sn = malloc(limbs * 8), *sp = malloc(limbs * 8), *en = malloc(limbs * 8);
    int8_t *e = malloc(n), *sg = malloc(n);
    small_to_ntt(c, s, pr, nqp, sn);
    if (galois == 1) {
        for (uint32_t t = 0; t < nqp; t++) {
            const om_mod *m = &c->pr[t].m;
            for (size_t k = 0; k < n; k++) {
                size_t i = (size_t)t * n + k;
                sp[i] = om_mul(sn[i], sn[i], m);
            }
        }
    } else {
        small_automorphism(c, galois, s, sg);
        small_to_ntt(c, sg, pr, nqp, sp);
    }
    /* P mod q_t */
    uint64_t Pmod[OR_MAXP];
    for (uint32_t t = 0; t < c->n_q; t++) {
        const om_mod *m = &c->pr[t].m;
        uint64_t v = 1;
        for (uint32_t k = 0; k < c->n_p; k++) v = om_mul(v, c->pr[c->n_q + k].m.q % m->q, m);
        Pmod[t] = v;
    }
    for (uint32_t j = 0; j < dnum; j++) {
        uint64_t *b = out + (size_t)j * 2 * limbs, *a = b + limbs;
        uint64_t base = ((uint64_t)galois << 16) | ((uint64_t)j << 8);
        for (uint32_t t = 0; t < nqp; t++)
            or_sample_uniform(seed, P_KSK_A, base | t, c->pr[t].m.q, n, a + (size_t)t * n);
        or_ntt_fwd(c, pr, nqp, a);
        or_sample_gauss(c, seed, P_KSK_E, base, n, e);
        small_to_ntt(c, e, pr, nqp, en);
        for (uint32_t t = 0; t < nqp; t++) {
            const om_mod *m = &c->pr[t].m;
            int in_digit = (t < c->n_q) && (t / alpha == j);
            for (size_t k = 0; k < n; k++) {
                size_t i = (size_t)t * n + k;
                uint64_t v = om_add(om_sub(0, om_mul(a[i], sn[i], m), m->q), en[i], m->q);
                if (in_digit) v = om_add(v, om_mul(Pmod[t], sp[i], m), m->q);
                b[i] = v;
            }
        }
    }
    free(sn); free(sp); free(en); free(e); free(sg);
    return 0;
}

/* ======================================================================== */
/* Encryption / decryption                                                  */
/* ======================================================================== */
int or_encrypt(const or_ctx *c, const uint64_t *pk, const int64_t *m, uint64_t seed,
               uint64_t ct_id, uint64_t *ct)
{
    size_t n = c->n;
    uint32_t L1 = c->n_q;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) pr[t] = t;
    size_t limbs = (size_t)L1 * n;
    uint64_t *vn = malloc(limbs * 8), *e0 = malloc(limbs * 8), *e1 = malloc(limbs * 8),
             *mn = malloc(limbs * 8);
    int8_t *tmp = malloc(n);
    or_sample_ternary(seed, P_ENC_V, ct_id, n, tmp);
    small_to_ntt(c, tmp, pr, L1, vn);
    or_sample_gauss(c, seed, P_ENC_E0, ct_id, n, tmp);
    small_to_ntt(c, tmp, pr, L1, e0);
    or_sample_gauss(c, seed, P_ENC_E1, ct_id, n, tmp);
    small_to_ntt(c, tmp, pr, L1, e1);
    or_encode_pt(c, L1 - 1, m, mn);
    const uint64_t *pk0 = pk, *pk1 = pk + limbs;
    for (uint32_t t = 0; t < L1; t++) {
        const om_mod *md = &c->pr[t].m;
        for (size_t k = 0; k < n; k++) {
            size_t i = (size_t)t * n + k;
            ct[i] = om_add(om_add(om_mul(vn[i], pk0[i], md), e0[i], md->q), mn[i], md->q);
            ct[limbs + i] = om_add(om_mul(vn[i], pk1[i], md), e1[i], md->q);
        }
    }
    free(vn); free(e0); free(e1); free(mn); free(tmp);
    return 0;
}

int or_decrypt(const or_ctx *c, const uint64_t *s_ntt, uint32_t level, const uint64_t *ct,
               uint64_t *m_out)
{
    size_t n = c->n;
    uint32_t L1 = level + 1;
    size_t limbs = (size_t)L1 * n;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) {
        pr[t] = t;
        const om_mod *md = &c->pr[t].m;
        for (size_t k = 0; k < n; k++) {
            size_t i = (size_t)t * n + k;
            m_out[i] = om_add(ct[i], om_mul(ct[limbs + i], s_ntt[i], md), md->q);
        }
    }
    or_ntt_inv(c, pr, L1, m_out);
    return 0;
}

/* ======================================================================== */
/* Ciphertext primitives (NTT domain)                                       */
/* ======================================================================== */
int or_add(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b, uint64_t *out)
{
    size_t n = c->n;
    for (uint32_t p = 0; p < n_poly; p++)
        for (uint32_t t = 0; t <= level; t++) {
            uint64_t q = c->pr[t].m.q;
            size_t o = ((size_t)p * (level + 1) + t) * n;
            for (size_t k = 0; k < n; k++) out[o + k] = om_add(a[o + k], b[o + k], q);
        }
    return 0;
}

int or_mulplain(const or_ctx *c, uint32_t level, const uint64_t *ct, const uint64_t *pt, uint64_t *out)
{
    size_t n = c->n, limbs = (size_t)(level + 1) * n;
    for (uint32_t p = 0; p < 2; p++)
        for (uint32_t t = 0; t <= level; t++) {
            const om_mod *m = &c->pr[t].m;
            for (size_t k = 0; k < n; k++) {
                size_t i = (size_t)t * n + k;
                out[p * limbs + i] = om_mul(ct[p * limbs + i], pt[i], m);
            }
        }
    return 0;
}

/* (a0,a1) x (b0,b1) -> (a0 b0, a0 b1 + a1 b0, a1 b1) */
int or_tensor(const or_ctx *c, uint32_t level, const uint64_t *a, const uint64_t *b, uint64_t *out3)
{
    size_t n = c->n, limbs = (size_t)(level + 1) * n;
    for (uint32_t t = 0; t <= level; t++) {
        const om_mod *m = &c->pr[t].m;
        for (size_t k = 0; k < n; k++) {
            size_t i = (size_t)t * n + k;
            uint64_t a0 = a[i], a1 = a[limbs + i], b0 = b[i], b1 = b[limbs + i];
            out3[i] = om_mul(a0, b0, m);
            out3[limbs + i] = om_add(om_mul(a0, b1, m), om_mul(a1, b0, m), m->q);
            out3[2 * limbs + i] = om_mul(a1, b1, m);
        }
    }
    return 0;
}

/* sigma_g in the coefficient domain: coefficient k moves to k*g mod 2N, negated past N */
int or_automorphism_coeff(const or_ctx *c, uint32_t n_limb, const uint32_t *prime,
                          uint32_t galois, const uint64_t *in, uint64_t *out)
{
    size_t n = c->n;
    uint64_t two_n = 2 * n;
    for (uint32_t t = 0; t < n_limb; t++) {
        uint64_t q = c->pr[prime[t]].m.q;
        const uint64_t *a = in + (size_t)t * n;
        uint64_t *o = out + (size_t)t * n;
        for (size_t k = 0; k < n; k++) {
            uint64_t e = ((uint64_t)k * galois) % two_n;
            if (e < n) o[e] = a[k];
            else o[e - n] = a[k] ? q - a[k] : 0;
        }
    }
    return 0;
}

/* sigma_g in the oracle NTT domain: (sigma_g a)(psi^(2i+1)) = a(psi^((2i+1)g)) */
int or_automorphism_ntt(const or_ctx *c, uint32_t n_limb, uint32_t galois,
                        const uint64_t *in, uint64_t *out)
{
    size_t n = c->n;
    uint64_t two_n = 2 * n;
    for (uint32_t t = 0; t < n_limb; t++) {
        const uint64_t *a = in + (size_t)t * n;
        uint64_t *o = out + (size_t)t * n;
        for (size_t i = 0; i < n; i++) {
            uint64_t e = ((2 * (uint64_t)i + 1) * galois) % two_n;
            o[i] = a[(e - 1) / 2];
        }
    }
    return 0;
}

/* ModUp of the digits of d (level l): for digit j with limbs I_j (product Q_j),
 * Conv_{I_j -> t}(a) = sum_{i in I_j} [a_i * (Q_j/q_i)^-1]_{q_i} * (Q_j/q_i) mod t,
 * a_i in [0, q_i) (no correction term); limbs in I_j keep d's own residues. */
int or_modup(const or_ctx *c, uint32_t level, const uint64_t *d, uint64_t *ext)
{
    size_t n = c->n;
    uint32_t L1 = level + 1, K = c->n_p, alpha = c->n_p, W = L1 + K;
    uint32_t dnum = or_dnum(c, level);
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < L1; t++) pr[t] = t;
    uint64_t *a = malloc((size_t)L1 * n * 8);
    memcpy(a, d, (size_t)L1 * n * 8);
    or_ntt_inv(c, pr, L1, a);
    uint32_t wp[OR_MAXP];
    for (uint32_t t = 0; t < W; t++) wp[t] = qp_prime(c, level, t);
    for (uint32_t j = 0; j < dnum; j++) {
        uint32_t lo = j * alpha, hi = (j + 1) * alpha < L1 ? (j + 1) * alpha : L1;
        uint64_t *e = ext + (size_t)j * W * n;
        /* [ (Q_j/q_i)^-1 ]_{q_i} */
        uint64_t qhat_inv[OR_MAXP];
        for (uint32_t i = lo; i < hi; i++) {
            const om_mod *mi = &c->pr[i].m;
            uint64_t v = 1;
            for (uint32_t i2 = lo; i2 < hi; i2++)
                if (i2 != i) v = om_mul(v, c->pr[i2].m.q % mi->q, mi);
            qhat_inv[i] = om_inv(v, mi);
        }
        #pragma omp parallel for schedule(static)
        for (uint32_t t = 0; t < W; t++) {
            uint64_t *o = e + (size_t)t * n;
            if (t >= lo && t < hi) {
                memcpy(o, d + (size_t)t * n, n * 8);   /* own residue, NTT domain */
                continue;
            }
            const om_mod *mt = &c->pr[wp[t]].m;
            uint64_t qhat_t[OR_MAXP];
            for (uint32_t i = lo; i < hi; i++) {
                uint64_t v = 1;
                for (uint32_t i2 = lo; i2 < hi; i2++)
                    if (i2 != i) v = om_mul(v, c->pr[i2].m.q % mt->q, mt);
                qhat_t[i] = v;
            }
            for (size_t k = 0; k < n; k++) {
                uint64_t acc = 0;
                for (uint32_t i = lo; i < hi; i++) {
                    uint64_t y = om_mul(a[(size_t)i * n + k], qhat_inv[i], &c->pr[i].m);
                    acc = om_add(acc, om_mul(y % mt->q, qhat_t[i], mt), mt->q);
                }
                o[k] = acc;
            }
            ntt_fwd_1(c, wp[t], o);
        }
    }
    free(a);
    return 0;
}

int or_ks_inner(const or_ctx *c, uint32_t level, const uint64_t *ext, const uint64_t *swk,
                uint32_t galois, uint64_t *out)
{
    size_t n = c->n;
    uint32_t L1 = level + 1, K = c->n_p, W = L1 + K, nqp = c->n_q + c->n_p;
    uint32_t dnum = or_dnum(c, level);
    size_t key_limbs = (size_t)nqp * n;
    uint64_t *perm = malloc((size_t)W * n * 8);
    memset(out, 0, (size_t)2 * W * n * 8);
    for (uint32_t j = 0; j < dnum; j++) {
        const uint64_t *e = ext + (size_t)j * W * n;
        if (galois != 1) { or_automorphism_ntt(c, W, galois, e, perm); e = perm; }
        for (uint32_t b = 0; b < 2; b++) {
            const uint64_t *key = swk + ((size_t)j * 2 + b) * key_limbs;
            #pragma omp parallel for schedule(static)
            for (uint32_t t = 0; t < W; t++) {
                uint32_t p = qp_prime(c, level, t);
                const om_mod *m = &c->pr[p].m;
                const uint64_t *kl = key + (size_t)p * n, *el = e + (size_t)t * n;
                uint64_t *o = out + ((size_t)b * W + t) * n;
                for (size_t k = 0; k < n; k++) o[k] = om_add(o[k], om_mul(el[k], kl[k], m), m->q);
            }
        }
    }
    free(perm);
    return 0;
}

/* Arithmetic over Q_l u P (limb t < l+1: q_t, else the special prime p_(t-l-1)), used by
 * the hoisted-ModDown evaluation of baby-step rotations. */
/* out[p] = a[p] (.) b for n_poly polynomials a [n_poly][W][N] and one b [W][N] */
int or_mul_ext(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b,
               uint64_t *out)
{
    size_t n = c->n;
    uint32_t W = level + 1 + c->n_p;
    for (uint32_t p = 0; p < n_poly; p++)
        for (uint32_t t = 0; t < W; t++) {
            const om_mod *m = &c->pr[qp_prime(c, level, t)].m;
            size_t o = ((size_t)p * W + t) * n;
            for (size_t k = 0; k < n; k++) out[o + k] = om_mul(a[o + k], b[(size_t)t * n + k], m);
        }
    return 0;
}

int or_add_ext(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b,
               uint64_t *out)
{
    size_t n = c->n;
    uint32_t W = level + 1 + c->n_p;
    for (uint32_t p = 0; p < n_poly; p++)
        for (uint32_t t = 0; t < W; t++) {
            uint64_t q = c->pr[qp_prime(c, level, t)].m.q;
            size_t o = ((size_t)p * W + t) * n;
            for (size_t k = 0; k < n; k++) out[o + k] = om_add(a[o + k], b[o + k], q);
        }
    return 0;
}

/* P * x lifted to Q_l u P: limb t < l+1 is [P]_{q_t} x_t, the special-prime limbs are 0
 * (n_poly polynomials x [n_poly][l+1][N] -> out [n_poly][W][N]) */
int or_scale_p_ext(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *x, uint64_t *out)
{
    size_t n = c->n;
    uint32_t L1 = level + 1, W = L1 + c->n_p;
    for (uint32_t p = 0; p < n_poly; p++)
        for (uint32_t t = 0; t < W; t++) {
            size_t o = ((size_t)p * W + t) * n;
            if (t >= L1) {
                memset(out + o, 0, n * 8);
                continue;
            }
            const om_mod *m = &c->pr[t].m;
            uint64_t Pm = 1;
            for (uint32_t k = 0; k < c->n_p; k++) Pm = om_mul(Pm, c->pr[c->n_q + k].m.q % m->q, m);
            const uint64_t *xi = x + ((size_t)p * L1 + t) * n;
            for (size_t k = 0; k < n; k++) out[o + k] = om_mul(xi[k], Pm, m);
        }
    return 0;
}

/* plaintext of integer coefficients m over Q_l u P, NTT domain */
int or_encode_pt_ext(const or_ctx *c, uint32_t level, const int64_t *m, uint64_t *pt)
{
    uint32_t W = level + 1 + c->n_p;
    uint32_t pr[OR_MAXP] = {0};
    for (uint32_t t = 0; t < W; t++) {
        pr[t] = qp_prime(c, level, t);
        uint64_t q = c->pr[pr[t]].m.q;
        for (size_t k = 0; k < c->n; k++) pt[(size_t)t * c->n + k] = signed_mod(m[k], q);
    }
    or_ntt_fwd(c, pr, W, pt);
    return 0;
}

/* ModDown: out_i = (x_i - Conv_{P->q_i}(x_P)) * P^-1 mod q_i, with the fast basis
 * conversion Conv_{P->q}(x) = sum_k [x_k * (P/p_k)^-1]_{p_k} * (P/p_k) mod q (x_k in [0,p_k),
 * no correction term). */
int or_moddown(const or_ctx *c, uint32_t level, const uint64_t *x, uint64_t *out)
{
    size_t n = c->n;
    uint32_t L1 = level + 1, K = c->n_p;
    uint32_t ppr[OR_MAXP] = {0};
    for (uint32_t k = 0; k < K; k++) ppr[k] = c->n_q + k;
    uint64_t *xp = malloc((size_t)K * n * 8);
    memcpy(xp, x + (size_t)L1 * n, (size_t)K * n * 8);
    or_ntt_inv(c, ppr, K, xp);
    /* y_k = x_k * [(P/p_k)^-1]_{p_k} */
    for (uint32_t k = 0; k < K; k++) {
        const om_mod *mk = &c->pr[c->n_q + k].m;
        uint64_t v = 1;
        for (uint32_t k2 = 0; k2 < K; k2++)
            if (k2 != k) v = om_mul(v, c->pr[c->n_q + k2].m.q % mk->q, mk);
        uint64_t vi = om_inv(v, mk);
        for (size_t i = 0; i < n; i++) xp[(size_t)k * n + i] = om_mul(xp[(size_t)k * n + i], vi, mk);
    }
    #pragma omp parallel for schedule(static)
    for (uint32_t t = 0; t < L1; t++) {
        const om_mod *mt = &c->pr[t].m;
        uint64_t phat[OR_MAXP], Pm = 1;
        for (uint32_t k = 0; k < K; k++) {
            uint64_t v = 1;
            for (uint32_t k2 = 0; k2 < K; k2++)
                if (k2 != k) v = om_mul(v, c->pr[c->n_q + k2].m.q % mt->q, mt);
            phat[k] = v;
            Pm = om_mul(Pm, c->pr[c->n_q + k].m.q % mt->q, mt);
        }
        uint64_t Pinv = om_inv(Pm, mt);
        uint64_t *conv = malloc(n * 8);
        for (size_t i = 0; i < n; i++) {
            uint64_t acc = 0;
            for (uint32_t k = 0; k < K; k++)
                acc = om_add(acc, om_mul(xp[(size_t)k * n + i] % mt->q, phat[k], mt), mt->q);
            conv[i] = acc;
        }
        ntt_fwd_1(c, t, conv);
        const uint64_t *xi = x + (size_t)t * n;
        uint64_t *o = out + (size_t)t * n;
        for (size_t i = 0; i < n; i++) o[i] = om_mul(om_sub(xi[i], conv[i], mt->q), Pinv, mt);
        free(conv);
    }
    free(xp);
    return 0;
}

/* Rescale by q_l: c_i <- (c_i - [c_l]_centred mod q_i) * q_l^-1 mod q_i, i < l,
 * with the centred lift of c_l in (-q_l/2, q_l/2]. */
int or_rescale(const or_ctx *c, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out)
{
    if (level == 0) return -1;
    size_t n = c->n;
    uint32_t L1 = level + 1;
    uint64_t ql = c->pr[level].m.q;
    for (uint32_t p = 0; p < n_poly; p++) {
        const uint64_t *ci = in + (size_t)p * L1 * n;
        uint64_t *co = out + (size_t)p * level * n;
        uint64_t *last = malloc(n * 8);
        memcpy(last, ci + (size_t)level * n, n * 8);
        ntt_inv_1(c, level, last);
        #pragma omp parallel for schedule(static)
        for (uint32_t t = 0; t < level; t++) {
            const om_mod *mt = &c->pr[t].m;
            uint64_t *w = malloc(n * 8);
            for (size_t k = 0; k < n; k++) {
                int64_t v = last[k] > (ql - 1) / 2 ? (int64_t)last[k] - (int64_t)ql : (int64_t)last[k];
                w[k] = signed_mod(v, mt->q);
            }
            ntt_fwd_1(c, t, w);
            uint64_t qinv = om_inv(ql % mt->q, mt);
            for (size_t k = 0; k < n; k++)
                co[(size_t)t * n + k] = om_mul(om_sub(ci[(size_t)t * n + k], w[k], mt->q), qinv, mt);
            free(w);
        }
        free(last);
    }
    return 0;
}
