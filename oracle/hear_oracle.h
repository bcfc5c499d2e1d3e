/*
 * hear_oracle.h -- plain CPU oracle for the RNS-CKKS hot path of HEAR / Fast-HEAR
 * (arXiv 2104.09164).  TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference legs may load this library.  It shares no
 * code, header, table or constant generator with the CUDA library under
 * paper_2104_09164_gb300/.
 *
 * What it follows (paper section "Methods"):
 *   - RNS variant of CKKS ("Algorithmic and cryptographic optimizations", cites
 *     Cheon-Han-Kim-Kim-Song SAC'18): ciphertexts over R_Q = Z_Q[X]/(X^N+1), Q a
 *     product of word-size primes, one residue polynomial ("limb") per prime.
 *   - slot rotation rho^l, "a rotation to the left by l positions" ("Single-channel
 *     homomorphic convolutions"), realised by the Galois automorphism X -> X^(5^l).
 *   - hoisting, lazy rescaling ("Algorithmic and cryptographic optimizations").
 *
 * Representation used by every function below unless stated otherwise:
 *   - a polynomial with n_limb limbs is uint64_t[n_limb][N], limb t reduced mod its
 *     prime; "NTT domain" = the ORACLE's own natural-order evaluation form
 *     A[i] = a(psi^(2i+1)), psi the oracle's primitive 2N-th root (see or_ctx_psi).
 *     Callers that compare against another implementation convert to the coefficient
 *     domain first (or_to_coeff).
 *   - prime indices: 0..n_q-1 are the ciphertext primes q_0..q_{n_q-1} (top level
 *     L = n_q-1), n_q..n_q+n_p-1 are the special primes p_0..p_{K-1}.
 *   - a polynomial "over Q_l u P" at level l has l+1+K limbs: q_0..q_l, p_0..p_{K-1}.
 *   - digits of the hybrid key switching: alpha = K limbs per digit, digit j covers
 *     limbs [j*alpha, min((j+1)*alpha, l+1)), dnum(l) = ceil((l+1)/alpha).
 *
 * Functions return 0 on success and a negative value on bad arguments.
 */
#ifndef HEAR_ORACLE_H
#define HEAR_ORACLE_H
#include <stdint.h>
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_ctx or_ctx;

/* ---- word-size modular arithmetic and primes ---- */
uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q);
int or_is_prime(uint64_t n);
/* Chain rule: for each requested bit size b (chain order q_0, q_1.., p_0..) take the
 * largest prime q < 2^b with q = 1 mod 2N not already taken. */
int or_gen_primes(uint32_t log_n, const uint32_t *bits, uint32_t count, uint64_t *out);

/* ---- context ---- */
or_ctx *or_ctx_create(uint32_t log_n, uint32_t n_q, const uint32_t *q_bits,
                      uint32_t n_p, const uint32_t *p_bits, double sigma);
void or_ctx_destroy(or_ctx *);
int or_ctx_primes(const or_ctx *, uint64_t *out);       /* n_q + n_p words */
int or_ctx_psi(const or_ctx *, uint64_t *out);          /* n_q + n_p words */
int or_set_threads(int n);                              /* OpenMP threads, 0 = default */

/* ---- NTT (oracle order), per limb; prime[t] gives limb t's prime index ---- */
int or_ntt_fwd(const or_ctx *, const uint32_t *prime, uint32_t n_limb, uint64_t *a);
int or_ntt_inv(const or_ctx *, const uint32_t *prime, uint32_t n_limb, uint64_t *a);

/* ---- randomness: ChaCha20 block function (RFC 8439) as a counter-based generator ---- */
void or_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3],
                       uint32_t out[16]);
/* words w0..w0+n-1 of stream(seed, purpose, index) */
void or_stream_words(uint64_t seed, uint32_t purpose, uint64_t index, uint64_t w0,
                     size_t n, uint64_t *out);
int or_cdt_table(const or_ctx *, uint64_t *out, uint32_t cap, uint32_t *n);
void or_sample_ternary(uint64_t seed, uint32_t purpose, uint64_t index, size_t n, int8_t *out);
int or_sample_gauss(const or_ctx *, uint64_t seed, uint32_t purpose, uint64_t index,
                    size_t n, int8_t *out);
void or_sample_uniform(uint64_t seed, uint32_t purpose, uint64_t index, uint64_t q,
                       size_t n, uint64_t *out);

/* ---- encoding (canonical embedding, double-double arithmetic) ---- */
/* z: N/2 real slot values; m_out: N integer coefficients round(scale * tau^-1(z)).
 * *near_ties = number of coefficients whose fractional part lies within 2^-30 of 1/2. */
int or_encode(const or_ctx *, const double *z, double scale, int64_t *m_out, int *near_ties);
/* dd twiddle helper exposed for pinning: cos/sin(2*pi*m/M) as hi+lo pairs */
void or_dd_cossin(uint64_t m, uint64_t M, double *c_hi, double *c_lo, double *s_hi, double *s_lo);

/* ---- keys (all outputs in the oracle NTT domain) ---- */
int or_keygen_sk(const or_ctx *, uint64_t seed, int8_t *s_out);                 /* N coeffs */
int or_sk_ntt(const or_ctx *, const int8_t *s, uint64_t *out);  /* [n_q+n_p][N] */
int or_keygen_pk(const or_ctx *, uint64_t seed, const int8_t *s, uint64_t *pk); /* [2][n_q][N] */
/* switching key from s' to s; galois = 1 means s' = s^2 (relinearisation), otherwise
 * s' = sigma_galois(s).  out: [dnum_max][2][n_q+n_p][N] */
int or_keygen_swk(const or_ctx *, uint64_t seed, const int8_t *s, uint32_t galois, uint64_t *out);
uint32_t or_dnum(const or_ctx *, uint32_t level);

/* ---- encryption / decryption ---- */
int or_encrypt(const or_ctx *, const uint64_t *pk, const int64_t *m, uint64_t seed,
               uint64_t ct_id, uint64_t *ct);                                   /* [2][n_q][N] */
/* m = c0 + c1*s at level l, returned in the COEFFICIENT domain [l+1][N] */
int or_decrypt(const or_ctx *, const uint64_t *s_ntt, uint32_t level, const uint64_t *ct,
               uint64_t *m_out);

/* ---- ring / ciphertext primitives (NTT domain, level l = limbs 0..l) ---- */
int or_to_coeff(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out);
int or_from_coeff(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out);
int or_encode_pt(const or_ctx *, uint32_t level, const int64_t *m, uint64_t *pt);  /* [l+1][N] */
int or_add(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b, uint64_t *out);
int or_mulplain(const or_ctx *, uint32_t level, const uint64_t *ct, const uint64_t *pt, uint64_t *out);
int or_tensor(const or_ctx *, uint32_t level, const uint64_t *a, const uint64_t *b, uint64_t *out3);
int or_automorphism_coeff(const or_ctx *, uint32_t n_limb, const uint32_t *prime,
                          uint32_t galois, const uint64_t *in, uint64_t *out);
int or_automorphism_ntt(const or_ctx *, uint32_t n_limb, uint32_t galois,
                        const uint64_t *in, uint64_t *out);
/* ModUp: d [l+1][N] -> ext [dnum(l)][l+1+K][N] */
int or_modup(const or_ctx *, uint32_t level, const uint64_t *d, uint64_t *ext);
/* key inner product with sigma_galois applied to the extended digits first
 * (galois = 1: none).  swk is the top-level key [dnum_max][2][n_q+n_p][N].
 * out: [2][l+1+K][N] */
int or_ks_inner(const or_ctx *, uint32_t level, const uint64_t *ext, const uint64_t *swk,
                uint32_t galois, uint64_t *out);
/* Q_l u P arithmetic for hoisted ModDown: products with one plaintext, sums, P * x lift,
 * plaintext encoding (NTT domain); polynomials [n_poly][l+1+K][N] */
int or_mul_ext(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b,
               uint64_t *out);
int or_add_ext(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *a, const uint64_t *b,
               uint64_t *out);
int or_scale_p_ext(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *x, uint64_t *out);
int or_encode_pt_ext(const or_ctx *, uint32_t level, const int64_t *m, uint64_t *pt);
/* ModDown: x [l+1+K][N] over Q_l u P -> out [l+1][N] */
int or_moddown(const or_ctx *, uint32_t level, const uint64_t *x, uint64_t *out);
/* Rescale by q_l: [n_poly][l+1][N] -> [n_poly][l][N] */
int or_rescale(const or_ctx *, uint32_t level, uint32_t n_poly, const uint64_t *in, uint64_t *out);

#ifdef __cplusplus
}
#endif
#endif
