// kernels.cuh -- launchers of the elementwise, sampling and basis-conversion kernels.
#pragma once
#include "internal.h"

namespace hear {

enum SmallKind { kTernary = 0, kGauss = 1 };

// ---- representation changes ----
void to_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s);
void from_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s);
void small_to_limbs(const hear_context *c, const int8_t *e, uint64_t *out, uint32_t n_limbs, LimbMap m,
                    cudaStream_t s);
void i64_to_limbs(const hear_context *c, const int64_t *v, uint64_t *out, uint32_t n_limbs, LimbMap m,
                  cudaStream_t s);
// n_polys polynomials at `level`, polynomial g from v + g*N (int64 coefficients)
void i64_to_limbs_batch(const hear_context *c, const int64_t *v, uint64_t *out, uint32_t n_polys, uint32_t level,
                        cudaStream_t s);

// ---- ChaCha20 samplers ----
void sample_small(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index, SmallKind kind,
                  int8_t *out, cudaStream_t s);
void sample_uniform(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index_base,
                    uint64_t *out, uint32_t n_limbs, LimbMap m, cudaStream_t s);

// ---- key / encryption combines ----
// pk: b = e - a*s (a, e NTT normal form, s Montgomery)
void pk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e,
                uint64_t *b, cudaStream_t st);
// switching key digit j: b = e - a*s + [t in digit] (P mod q_t) * s'   over all n_q+n_p primes
void swk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e,
                 const uint64_t *sp_mont, const uint64_t *p_mod, uint32_t digit, uint64_t *b, cudaStream_t st);
void encrypt_combine(const hear_context *c, const uint64_t *v, const uint64_t *e0, const uint64_t *e1,
                     const uint64_t *m, const uint64_t *pk_mont, uint64_t *ct, cudaStream_t st);
void decrypt_combine(const hear_context *c, uint32_t level, const uint64_t *ct, const uint64_t *s_mont,
                     uint64_t *out, cudaStream_t st);

// ---- ciphertext arithmetic (NTT domain), batch of n_ct ciphertexts of n_poly polys ----
void add_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, const uint64_t *b,
            uint64_t *out, cudaStream_t st);
void tensor_ct(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *a, const uint64_t *b,
               uint64_t *out3, cudaStream_t st);
// out = sigma_g(in) for n_polys_total polynomials at `level`
void automorphism(const hear_context *c, uint32_t level, uint32_t n_polys_total, uint32_t galois,
                  const uint64_t *in, uint64_t *out, cudaStream_t st);
// BSGS inner sums on contiguous storage: out[j][c] = sum_{b < n1} pt[j*n1 + b] (.) baby[b][c]
// baby [n1][n_ct][2][level+1][N], pt [n2*n1][level+1][N] (Montgomery; zero for missing
// diagonals), out [n2][n_ct][2][level+1][N]
void lincomb(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t n1, uint32_t n2, const uint64_t *baby,
             const uint64_t *pt, uint64_t *out, cudaStream_t st);
// the same over Q_l u P: baby [n1][n_ct][2][W][N], pt [n2*n1][W][N], out [n2][n_ct][2][W][N]
void lincomb_ext(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t n1, uint32_t n2, const uint64_t *baby,
                 const uint64_t *pt, uint64_t *out, cudaStream_t st);
// P x over Q_l u P for n_polys polynomials x [.][l+1][N] -> out [.][W][N]; pmod = ([P]_{q_t},
// Shoup) pairs for t <= l
void scale_p_ext(const hear_context *c, uint32_t level, uint32_t n_polys, const uint64_t *x, uint64_t *out,
                 const uint64_t *pmod, cudaStream_t st);
// out (batch [n_ct][2][level+1][N]) = ct (batch) (.) pt   (pt Montgomery, no accumulation)
void mulplain(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *ct, const uint64_t *pt,
              uint64_t *out, cudaStream_t st);
// out[z] = ct[z] (.) pt[z / cts_per_pt]  (plaintexts [.][level+1][N], Montgomery)
void mulplain_grouped(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t cts_per_pt, const uint64_t *ct,
                      const uint64_t *pt, uint64_t *out, cudaStream_t st);
// c0 of ct[z] += pt[z / cts_per_pt]  (plaintexts in normal NTT form), in place
void add_plain(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t cts_per_pt, uint64_t *ct,
               const uint64_t *pt, cudaStream_t st);

// ---- key switching ----
// ext [n_ct][dnum][W][N] from c1 (NTT, [n_ct] polys at stride c1_stride words); tmp: n_ct*(l+1)*N words
void modup(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *c1, uint64_t c1_stride,
           uint64_t *ext, uint64_t *tmp, cudaStream_t st);
// Set-up of the bulk-copy key inner products (their dynamic shared memory) on the current
// device; called once per context at creation.
void ks_bulk_setup();
// Bounded device waits that ran out since the last clear (process-wide counter on the
// current device); clear = reset it to zero.
uint32_t async_timeouts(bool clear);
// One wait on an mbarrier that nothing completes, limited to limit_cycles SM cycles: 1 if it
// ran out (counted like any other), 0 if it completed.  Synchronises `st`.
uint32_t wait_probe(long long limit_cycles, cudaStream_t st);
// Key inner product, R jobs of C ciphertexts: out[r*C + c] ([2][W][N]) =
//   sum_j sigma_{g_r}(ext_j) (.) key_r[j],  ext = ext[c] (shared) or ext[r*C + c] (per job).
// d_keys[r]: switching key stored sigma_{g_r}^{-1}-permuted; d_ginv[r] = g_r^{-1} mod 2N.
// c1 / c1_stride: the polynomials modup() extended (with one-limb digits modup leaves each
// digit's own limb there instead of copying it into ext)
// pmod (optional, ([P]_{q_t}, Shoup) pairs): the outputs are the rotations before ModDown,
// (P sigma_g(c0) + u0, u1) over Q_l u P, with c0 the plane before c1 (shared digits only)
void ks_inner(const hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *ext, bool ext_per_job,
              const uint64_t *const *d_keys, const uint32_t *d_ginv, uint64_t *out, const uint64_t *c1,
              uint64_t c1_stride, cudaStream_t st, const uint64_t *pmod = nullptr);
// ModDown of acc [n_ct][2][W][N] (destroys its P limbs) into out [n_ct][2][l+1][N], adding an
// addend ciphertext (ciphertext index c, or c mod cts_per_job if add_shared, at addend +
// index*add_stride, polys [2][l+1][N]; poly p only if add_mask bit p) gathered through
// sigma_g with g = d_gal[c / cts_per_job] (d_gal null = identity).  tmp: n_ct*2*(l+1)*N words
// acc_count > 1: the ModDown of the sum of acc_count such inputs, input r at acc + r * acc_cstride
// (each left unchanged)
void moddown(const hear_context *c, uint32_t level, uint32_t n_ct, uint64_t *acc, uint64_t *out,
             const uint64_t *addend, uint64_t add_stride, uint32_t add_mask, bool add_shared, const uint32_t *d_gal,
             uint32_t cts_per_job, uint64_t *tmp, cudaStream_t st, uint32_t acc_count = 1, uint64_t acc_cstride = 0);
// out = sum of cnt batches a + j*stride (n_polys_total polynomials at level)
void sum_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, uint64_t stride,
            uint32_t cnt, uint64_t *out, cudaStream_t st);
// out = base + sum of cnt batches a + j*stride (out may alias base)
void sum_add_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, uint64_t stride,
                uint32_t cnt, const uint64_t *base, uint64_t *out, cudaStream_t st);
// out = a (.) b_mont over n_limbs limbs (Montgomery product: a * b)
void pointwise_mont(const hear_context *c, uint32_t n_limbs, LimbMap m, const uint64_t *a, const uint64_t *b_mont,
                    uint64_t *out, cudaStream_t st);
// rescale batch [n_polys][l+1][N] -> out [n_polys][l][N]; destroys limb l of `in`; tmp n_polys*l*N words
void rescale(const hear_context *c, uint32_t level, uint32_t n_polys, uint64_t *in, uint64_t *out, uint64_t *tmp,
             cudaStream_t st);

// time every launch form of the inner products / inner sums and fill c->ks_choice (ms_out:
// [kKsTables][kKsBuckets][4] or null)
void ks_tune(hear_context *c, uint32_t max_ct, int iters, float *ms_out);

}  // namespace hear
