// kernels.cu -- elementwise, sampling and basis-conversion kernels of RNS-CKKS on sm_103a.
//
// Grids are 3-D: x covers the coefficient index of a limb (256 consecutive residues per
// CTA, so every warp reads and writes 256 contiguous bytes), y and z cover limbs and
// ciphertexts, so no thread ever divides a 64-bit index.  The NTT-domain ordering is that
// of ntt.cu: index i holds the evaluation at psi^(2 brv(i) + 1).
#include <functional>
#include "kernels.cuh"
#include "modarith.cuh"
#include "launch.cuh"

namespace hear {
namespace {

constexpr int kBlock = 256;

// grid for n coefficients x ny x nz; ny, nz <= 65535 is checked by the launchers
inline dim3 grid3(uint32_t n, uint32_t ny, uint32_t nz) { return dim3(n / kBlock, ny, nz); }
#define COEF() (blockIdx.x * kBlock + threadIdx.x)

// limb index of a LimbMap launch: y + z * gridDim.y
__device__ __forceinline__ uint32_t limb_yz() { return blockIdx.y + blockIdx.z * gridDim.y; }

// ------------------------------------------------------------------ representation
__global__ void k_to_mont(uint64_t *d, uint32_t n_limbs, LimbMap m, const DevPrime *P, uint32_t n, int dir) {
    pdl_enter();
    uint32_t b = limb_yz(), pi;
    if (b >= n_limbs || !m.resolve(b, &pi)) return;
    const DevPrime p = P[pi];
    uint64_t &x = d[m.offset(b, n) + COEF()];
    x = dir ? mont_mul(x, p.r2, p.q, p.qinv) : mont_mul(x, 1, p.q, p.qinv);
}

__global__ void k_pointwise_mont(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t n_limbs, LimbMap m,
                                 const DevPrime *P, uint32_t n) {
    pdl_enter();
    uint32_t bb = limb_yz(), pi;
    if (bb >= n_limbs || !m.resolve(bb, &pi)) return;
    const DevPrime p = P[pi];
    uint64_t off = m.offset(bb, n) + COEF();
    out[off] = mont_mul(a[off], b[off], p.q, p.qinv);
}

__global__ void k_small_to_limbs(const int8_t *e, uint64_t *out, uint32_t n_limbs, LimbMap m, const DevPrime *P,
                                 uint32_t n) {
    pdl_enter();
    uint32_t b = limb_yz(), pi, k = COEF();
    if (b >= n_limbs || !m.resolve(b, &pi)) return;
    int v = e[k];
    uint64_t q = P[pi].q;
    out[m.offset(b, n) + k] = v < 0 ? q - (uint64_t)(-v) : (uint64_t)v;
}

// group g of the limb map reads v + g * v_stride (v_stride 0: one vector for every limb)
__global__ void k_i64_to_limbs(const int64_t *v, uint64_t *out, uint32_t n_limbs, LimbMap m, const DevPrime *P,
                               uint32_t n, uint64_t v_stride) {
    pdl_enter();
    uint32_t b = limb_yz(), pi, k = COEF();
    if (b >= n_limbs || !m.resolve(b, &pi)) return;
    const DevPrime p = P[pi];
    int64_t x = v[(uint64_t)(b / m.per_group) * v_stride + k];
    uint64_t mag = x < 0 ? (uint64_t)0 - (uint64_t)x : (uint64_t)x;
    uint64_t r = reduce64(mag, p);
    out[m.offset(b, n) + k] = (x < 0) ? neg_mod(r, p.q) : r;
}

// ------------------------------------------------------------------ ChaCha20 (RFC 8439)
__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return __funnelshift_l(x, x, r); }
__device__ __forceinline__ void qround(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d) {
    a += b; d ^= a; d = rotl(d, 16);
    c += d; b ^= c; b = rotl(b, 12);
    a += b; d ^= a; d = rotl(d, 8);
    c += d; b ^= c; b = rotl(b, 7);
}
// block `counter` of the stream keyed by (seed || 0^24), nonce (purpose, index lo, index hi);
// returns the eight 64-bit words w[8*counter .. 8*counter+7]
__device__ void chacha_words(uint64_t seed, uint32_t purpose, uint64_t index, uint32_t counter, uint64_t w[8]) {
    uint32_t s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                      (uint32_t)seed, (uint32_t)(seed >> 32), 0u, 0u, 0u, 0u, 0u, 0u,
                      counter, purpose, (uint32_t)index, (uint32_t)(index >> 32)};
    uint32_t x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll
    for (int r = 0; r < 10; r++) {
        qround(x[0], x[4], x[8], x[12]);
        qround(x[1], x[5], x[9], x[13]);
        qround(x[2], x[6], x[10], x[14]);
        qround(x[3], x[7], x[11], x[15]);
        qround(x[0], x[5], x[10], x[15]);
        qround(x[1], x[6], x[11], x[12]);
        qround(x[2], x[7], x[8], x[13]);
        qround(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 8; i++)
        w[i] = (uint64_t)(x[2 * i] + s[2 * i]) | ((uint64_t)(x[2 * i + 1] + s[2 * i + 1]) << 32);
}

__global__ void k_sample_small(uint64_t seed, uint32_t purpose, uint64_t index, uint32_t n, int kind,
                               const uint64_t *cdt, uint32_t cdt_n, int8_t *out) {
    pdl_enter();
    uint32_t blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= n / 8) return;
    uint64_t w[8];
    chacha_words(seed, purpose, index, blk, w);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        int v;
        if (kind == kTernary) {
            v = (int)(w[j] % 3) - 1;
        } else {
            uint64_t u = w[j] >> 1;
            int mag = 0;
            while (mag + 1 < (int)cdt_n && !(u < cdt[mag])) mag++;
            v = (w[j] & 1) ? -mag : mag;
        }
        out[blk * 8 + j] = (int8_t)v;
    }
}

// uniform residues: coefficient k of limb b is (w_{2k+1} 2^64 + w_{2k}) mod q, stream index
// index_base | prime(b); one thread per ChaCha20 block (four coefficients)
__global__ void k_sample_uniform(uint64_t seed, uint32_t purpose, uint64_t index_base, uint64_t *out,
                                 uint32_t n_limbs, LimbMap m, const DevPrime *P, uint32_t n) {
    pdl_enter();
    uint32_t b = limb_yz(), pi, blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_limbs || blk >= n / 4 || !m.resolve(b, &pi)) return;
    const DevPrime p = P[pi];
    uint64_t w[8];
    chacha_words(seed, purpose, index_base | pi, blk, w);
    uint64_t *o = out + m.offset(b, n) + (uint64_t)blk * 4;
#pragma unroll
    for (int j = 0; j < 4; j++) o[j] = barrett_reduce(u128{w[2 * j], w[2 * j + 1]}, p.q, p.ratio_hi, p.ratio_lo);
}

// ------------------------------------------------------------------ keys and encryption
// y = limb (prime index == limb index in these layouts)
__global__ void k_pk_combine(const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, uint64_t *b,
                             const DevPrime *P, uint32_t n) {
    pdl_enter();
    const DevPrime p = P[blockIdx.y];
    uint64_t i = (uint64_t)blockIdx.y * n + COEF();
    b[i] = sub_mod(e[i], mont_mul(a[i], s_mont[i], p.q, p.qinv), p.q);
}

__global__ void k_swk_combine(const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, const uint64_t *sp_mont,
                              const uint64_t *p_mod, uint32_t lo, uint32_t hi, const DevPrime *P, uint32_t n,
                              uint64_t *b) {
    pdl_enter();
    const uint32_t t = blockIdx.y;
    const DevPrime p = P[t];
    uint64_t i = (uint64_t)t * n + COEF();
    uint64_t v = sub_mod(e[i], mont_mul(a[i], s_mont[i], p.q, p.qinv), p.q);
    if (t >= lo && t < hi) v = add_mod(v, mont_mul(p_mod[t], sp_mont[i], p.q, p.qinv), p.q);
    b[i] = v;
}

__global__ void k_encrypt_combine(const uint64_t *v, const uint64_t *e0, const uint64_t *e1, const uint64_t *m,
                                  const uint64_t *pk_mont, uint64_t *ct, uint64_t limbs, const DevPrime *P,
                                  uint32_t n) {
    pdl_enter();
    const DevPrime p = P[blockIdx.y];
    uint64_t i = (uint64_t)blockIdx.y * n + COEF();
    ct[i] = add_mod(add_mod(mont_mul(v[i], pk_mont[i], p.q, p.qinv), e0[i], p.q), m[i], p.q);
    ct[limbs + i] = add_mod(mont_mul(v[i], pk_mont[limbs + i], p.q, p.qinv), e1[i], p.q);
}

__global__ void k_decrypt_combine(const uint64_t *ct, const uint64_t *s_mont, uint64_t *out, uint64_t limbs,
                                  const DevPrime *P, uint32_t n) {
    pdl_enter();
    const DevPrime p = P[blockIdx.y];
    uint64_t i = (uint64_t)blockIdx.y * n + COEF();
    out[i] = add_mod(ct[i], mont_mul(ct[limbs + i], s_mont[i], p.q, p.qinv), p.q);
}

// ------------------------------------------------------------------ ciphertext arithmetic
// y = limb t, z = polynomial
__global__ void k_add(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t L1, const DevPrime *P,
                      uint32_t n) {
    pdl_enter();
    uint64_t i = ((uint64_t)blockIdx.z * L1 + blockIdx.y) * n + COEF();
    out[i] = add_mod(a[i], b[i], P[blockIdx.y].q);
}

// out = a_0 + a_1 + ... + a_{cnt-1} (batches at stride `stride` words); y = limb, z = polynomial
// (base = null) or out = base + a_0 + ... + a_{cnt-1}
__global__ void k_sum(const uint64_t *a, uint64_t stride, uint32_t cnt, const uint64_t *base, uint64_t *out,
                      uint32_t L1, const DevPrime *P, uint32_t n) {
    pdl_enter();
    uint64_t i = ((uint64_t)blockIdx.z * L1 + blockIdx.y) * n + COEF();
    const uint64_t q = P[blockIdx.y].q;
    uint64_t s = base ? base[i] : 0;
    for (uint32_t j = 0; j < cnt; j++) s = add_mod(s, a[j * stride + i], q);
    out[i] = s;
}

// y = limb t, z = ciphertext
__global__ void k_tensor(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t L1, const DevPrime *P,
                         uint32_t n) {
    pdl_enter();
    const uint64_t plane = (uint64_t)L1 * n, c = blockIdx.z;
    const uint64_t r = (uint64_t)blockIdx.y * n + COEF();
    const DevPrime p = P[blockIdx.y];
    const uint64_t *ac = a + c * 2 * plane, *bc = b + c * 2 * plane;
    uint64_t *oc = out + c * 3 * plane;
    uint64_t a0 = ac[r], a1 = ac[plane + r], b0 = bc[r], b1 = bc[plane + r];
    oc[r] = mul_mod(a0, b0, p);
    u128 s = mul_wide(a0, b1);
    add_to(s, mul_wide(a1, b0));
    oc[plane + r] = barrett_reduce(s, p.q, p.ratio_hi, p.ratio_lo);
    oc[2 * plane + r] = mul_mod(a1, b1, p);
}

// y + z * gridDim.y = limb of the whole batch
__global__ void k_automorphism(const uint64_t *in, uint64_t *out, uint32_t n_limbs, uint32_t galois,
                               uint32_t log_n) {
    pdl_enter();
    uint32_t b = limb_yz(), k = COEF();
    if (b >= n_limbs) return;
    const uint64_t base = (uint64_t)b << log_n;
    out[base + k] = in[base + auto_index(k, galois, log_n)];
}

// lazily accumulate x*y into acc keeping acc.hi < q (so the final Montgomery reduce is valid)
__device__ __forceinline__ void mac_raw(u128 &acc, uint64_t x, uint64_t y);
__device__ __forceinline__ void mac_lazy(u128 &acc, uint64_t x, uint64_t y, uint64_t q) {
    mac_raw(acc, x, y);
    if (acc.hi >= q) acc.hi -= q;
}
// accumulate without the check: up to 8 products of residues below q < 2^61 keep acc.hi
// below q + 8 q^2 / 2^64 < 2q; fold() then restores acc.hi < q
// acc += x * y as one carry chain over 32-bit halves (x = x1 2^32 + x0, y likewise): the
// partial products x0 y0 and x1 y1 land on words 0-1 and 2-3, x0 y1 and x1 y0 on words 1-2,
// each chain propagating its carry to word 3 -- ten multiply-adds for the 128-bit sum
__device__ __forceinline__ void mac_raw(u128 &acc, uint64_t x, uint64_t y) {
    uint32_t a0, a1, a2, a3, x0, x1, y0, y1;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(a0), "=r"(a1) : "l"(acc.lo));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(a2), "=r"(a3) : "l"(acc.hi));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(x0), "=r"(x1) : "l"(x));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(y0), "=r"(y1) : "l"(y));
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3)
        : "r"(x0), "r"(x1), "r"(y0), "r"(y1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(acc.lo) : "r"(a0), "r"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(acc.hi) : "r"(a2), "r"(a3));
}
__device__ __forceinline__ void fold(u128 &acc, uint64_t q) {
    if (acc.hi >= q) acc.hi -= q;
}

// BSGS inner sums out[j][c] = sum_b pt[j][b] (.) baby[b][c] on contiguous storage:
// baby [n1][C][2][L1][N], pt [n2*n1][L1][N] (Montgomery), out [n2][C][2][L1][N].
// CTA = 8 warps, each one polynomial (c, poly) of the batch; lanes over 32 consecutive
// coefficients.  Grid x = group of 8 polynomials (fastest), y = coefficient tile, z = limb:
// all CTAs of one (limb, tile) run back to back, so the plaintext tile they share comes
// from HBM once and from L2 (and, within a CTA, L1) afterwards.  Each thread walks the
// giant steps in chunks of JC accumulators; its baby words stay in L1/L2 across chunks.
// With few ciphertexts (2C <= 4 polynomials, one CTA column) the warps beyond 2C would idle:
// jw = 8 / 2C warps then share each polynomial, warp w taking polynomial w mod 2C and the
// giant-step chunks (JC outputs each) jpart, jpart + jw, .. with jpart = w / 2C.
// Limbs t >= lq are over the special primes (inner sums over Q_l u P): prime n_q + t - lq.
// JC = giant-step outputs accumulated per pass over the babies (4, 2 or 1; or 8 with the
// registers of two CTAs per SM): fewer accumulators re-read the babies more often but leave
// more chunks to spread over the warps when there are few ciphertexts
template <int JC>
__global__ void __launch_bounds__(256, JC == 8 ? 2 : 4) k_lincomb(uint32_t L1, uint32_t C, uint32_t n1, uint32_t n2,
                                                 const uint64_t *__restrict__ baby, const uint64_t *__restrict__ pt,
                                                 uint64_t *__restrict__ out, const DevPrime *P, uint32_t n,
                                                 uint32_t jw, uint32_t lq, uint32_t n_q) {
    pdl_enter();
    const uint32_t w = threadIdx.x >> 5;
    uint32_t cp, jpart;                                           // cp = c * 2 + poly
    if (jw > 1) {
        cp = w % (2 * C);
        jpart = w / (2 * C);
        if (jpart >= jw) return;
    } else {
        cp = blockIdx.x * 8 + w;
        jpart = 0;
        if (cp >= 2 * C) return;
    }
    const uint32_t t = blockIdx.z, k = blockIdx.y * 32 + (threadIdx.x & 31);
    const uint64_t plane = (uint64_t)L1 * n, r = (uint64_t)t * n + k;
    const uint32_t pi = t < lq ? t : n_q + (t - lq);
    const uint64_t q = P[pi].q, qinv = P[pi].qinv;
    const uint64_t bstride = 2ull * C * plane;                    // between baby steps / giant outputs
    const uint64_t *bp = baby + (uint64_t)cp * plane + r;
    for (uint32_t j0 = JC * jpart; j0 < n2; j0 += JC * jw) {
        u128 acc[JC];
#pragma unroll
        for (int jj = 0; jj < JC; jj++) acc[jj] = u128{0, 0};
        const uint64_t *pp = pt + ((uint64_t)j0 * n1) * plane + r;
        const uint32_t jn = min((uint32_t)JC, n2 - j0);
        uint32_t b = 0;
        // two baby steps per iteration: ten independent loads in flight per thread
        for (; b + 2 <= n1; b += 2) {
            const uint64_t x0 = bp[(uint64_t)b * bstride], x1 = bp[(uint64_t)(b + 1) * bstride];
            uint64_t w0[JC], w1[JC];
#pragma unroll
            for (int jj = 0; jj < JC; jj++) {
                if (jj < (int)jn) {
                    w0[jj] = __ldg(pp + ((uint64_t)jj * n1 + b) * plane);
                    w1[jj] = __ldg(pp + ((uint64_t)jj * n1 + b + 1) * plane);
                }
            }
#pragma unroll
            for (int jj = 0; jj < JC; jj++) {
                if (jj < (int)jn) {
                    mac_raw(acc[jj], x0, w0[jj]);
                    mac_raw(acc[jj], x1, w1[jj]);
                    fold(acc[jj], q);
                }
            }
        }
        for (; b < n1; b++) {
            const uint64_t x = bp[(uint64_t)b * bstride];
#pragma unroll
            for (int jj = 0; jj < JC; jj++)
                if (jj < (int)jn) mac_lazy(acc[jj], x, __ldg(pp + ((uint64_t)jj * n1 + b) * plane), q);
        }
        uint64_t *op = out + (uint64_t)j0 * bstride + (uint64_t)cp * plane + r;
#pragma unroll
        for (int jj = 0; jj < JC; jj++)
            if (j0 + jj < n2) op[(uint64_t)jj * bstride] = mont_reduce(acc[jj], q, qinv);
    }
}

// BSGS inner sums for a batch of C <= 4 ciphertexts (P2 = 2C polynomials): a CTA owns 32
// coefficients of one limb and its 8 warps split the baby steps (warp w takes b = w, w + 8,
// ..); for a chunk of JS = max(1, 8 / P2) giant-step outputs every thread accumulates all P2
// polynomials, so a plaintext word is loaded once per CTA, and it keeps the P2 + JS loads of
// two baby steps in flight at a time.  The warps' partial 128-bit sums (each with hi < q) meet in
// shared memory; warp i adds the 8 partials of output pair i (hi < 8q, brought below q by
// subtracting multiples of q 2^64) and reduces.  Same residues as k_lincomb.
template <int C>
__global__ void __launch_bounds__(256, 3) k_lincomb_split(uint32_t L1, uint32_t n1, uint32_t n2,
                                                          const uint64_t *__restrict__ baby,
                                                          const uint64_t *__restrict__ pt, uint64_t *__restrict__ out,
                                                          const DevPrime *P, uint32_t n, uint32_t lq, uint32_t n_q) {
    constexpr int P2 = 2 * C, JS = P2 >= 8 ? 1 : 8 / P2, NP = JS * P2;   // NP <= 8 output pairs
    __shared__ u128 part[8][NP][32];
    pdl_enter();
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t = blockIdx.y, k = blockIdx.x * 32 + lane;
    const uint64_t plane = (uint64_t)L1 * n, r = (uint64_t)t * n + k;
    const uint32_t pi = t < lq ? t : n_q + (t - lq);
    const uint64_t q = P[pi].q, qinv = P[pi].qinv;
    const uint64_t bstride = (uint64_t)P2 * plane;        // between baby steps / giant outputs
    for (uint32_t j0 = 0; j0 < n2; j0 += JS) {
        const uint32_t jn = min((uint32_t)JS, n2 - j0);
        u128 acc[NP];
#pragma unroll
        for (int i = 0; i < NP; i++) acc[i] = u128{0, 0};
        // two of the warp's baby steps (b, b + 8) per iteration: all their loads in flight at once
        for (uint32_t b = w; b < n1; b += 16) {
            const bool two = b + 8 < n1;
            uint64_t x[2][P2], y[2][JS];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t bb = b + 8 * h;
                if (h == 0 || two) {
#pragma unroll
                    for (int cp = 0; cp < P2; cp++) x[h][cp] = baby[(uint64_t)bb * bstride + (uint64_t)cp * plane + r];
#pragma unroll
                    for (int jj = 0; jj < JS; jj++)
                        if (jj < (int)jn) y[h][jj] = __ldg(pt + ((uint64_t)(j0 + jj) * n1 + bb) * plane + r);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; h++)
                if (h == 0 || two)
#pragma unroll
                    for (int jj = 0; jj < JS; jj++)
                        if (jj < (int)jn)
#pragma unroll
                            for (int cp = 0; cp < P2; cp++) mac_raw(acc[jj * P2 + cp], x[h][cp], y[h][jj]);
#pragma unroll
            for (int i = 0; i < NP; i++) fold(acc[i], q);      // after at most two products
        }
#pragma unroll
        for (int i = 0; i < NP; i++) {
            fold(acc[i], q);
            part[w][i][lane] = acc[i];
        }
        __syncthreads();
        if (w < jn * P2) {
            u128 sum = part[0][w][lane];
#pragma unroll
            for (int v = 1; v < 8; v++) {
                const u128 a = part[v][w][lane];
                const uint64_t lo = sum.lo + a.lo;
                sum.hi += a.hi + (lo < sum.lo ? 1 : 0);
                sum.lo = lo;
            }
            if (sum.hi >= 4 * q) sum.hi -= 4 * q;
            if (sum.hi >= 2 * q) sum.hi -= 2 * q;
            if (sum.hi >= q) sum.hi -= q;
            const uint32_t jj = w / P2, cp = w % P2;
            out[(uint64_t)(j0 + jj) * bstride + (uint64_t)cp * plane + r] = mont_reduce(sum, q, qinv);
        }
        __syncthreads();
    }
}

// y = poly*L1 + limb, z = ciphertext; ciphertext z meets plaintext z / cts_per_pt
__global__ void k_mulplain(const uint64_t *ct, const uint64_t *pt, uint64_t *out, uint32_t L1, const DevPrime *P,
                           uint32_t n, uint32_t cts_per_pt) {
    pdl_enter();
    const uint32_t t = blockIdx.y % L1;
    const DevPrime p = P[t];
    const uint64_t i = ((uint64_t)blockIdx.z * 2 * L1 + blockIdx.y) * n + COEF();
    const uint64_t *pz = pt + (uint64_t)(blockIdx.z / cts_per_pt) * L1 * n;
    out[i] = mont_mul(ct[i], pz[(uint64_t)t * n + COEF()], p.q, p.qinv);
}

// c0 of ciphertext z += plaintext z / cts_per_pt (normal NTT form); y = limb
__global__ void k_add_plain(uint64_t *ct, const uint64_t *pt, uint32_t L1, const DevPrime *P, uint32_t n,
                            uint32_t cts_per_pt) {
    pdl_enter();
    const uint32_t t = blockIdx.y;
    const uint64_t i = ((uint64_t)blockIdx.z * 2 * L1 + t) * n + COEF();
    const uint64_t *pz = pt + (uint64_t)(blockIdx.z / cts_per_pt) * L1 * n;
    ct[i] = add_mod(ct[i], pz[(uint64_t)t * n + COEF()], P[t].q);
}

// ------------------------------------------------------------------ key switching
// ModUp conversion, one thread per (ciphertext c = z, digit j = y, coefficient): the
// digit's alpha residues y_i = a_i * qhat_inv_i are formed once, then every target limb t
// outside the digit receives sum_i y_i * [Q_j/q_i]_t mod t; the digit's own limbs copy c1
// (NTT domain).
__global__ void k_modup_conv(const uint64_t *c1, uint64_t c1_stride, const uint64_t *y, uint64_t *ext,
                             uint32_t L1, uint32_t W, uint32_t dnum, uint32_t alpha, uint32_t n_q,
                             const uint64_t *qhat_inv, const uint64_t *qhat_mod, const DevPrime *P, uint32_t n) {
    pdl_enter();
    const uint32_t k = COEF(), j = blockIdx.y, c = blockIdx.z;
    const uint32_t lo = j * alpha, hi = min(lo + alpha, L1);
    uint64_t *e = ext + ((uint64_t)c * dnum + j) * W * n + k;
    uint64_t ys[4] = {0, 0, 0, 0};
#pragma unroll
    for (int ii = 0; ii < 4; ii++) {
        const uint32_t src = lo + ii;
        if (src < hi) {
            const DevPrime ps = P[src];
            ys[ii] = shoup(y[((uint64_t)c * L1 + src) * n + k], qhat_inv[2 * src], qhat_inv[2 * src + 1], ps.q);
            e[(uint64_t)src * n] = c1[c * c1_stride + (uint64_t)src * n + k];
        }
    }
    for (uint32_t t = 0; t < W; t++) {
        if (t >= lo && t < hi) continue;
        const uint32_t pt = t < L1 ? t : n_q + (t - L1);
        const uint64_t q = P[pt].q;
        uint64_t acc = 0;
#pragma unroll
        for (int ii = 0; ii < 4; ii++) {
            if (lo + ii >= hi) break;
            const uint64_t *wm = qhat_mod + 2 * (((uint64_t)j * alpha + ii) * W + t);
            acc = add_mod(acc, shoup(ys[ii], wm[0], wm[1], q), q);
        }
        e[(uint64_t)t * n] = acc;
    }
}

// Key inner product for R jobs of C ciphertexts.  Job r uses the switching key keys[r],
// stored sigma_{g_r}^{-1}-permuted, so sum_j ext_j[k] key'_j[k] is formed with coalesced
// reads and written to position sigma_{g_r}^{-1}(k) of the output, which equals
// sum_j sigma_{g_r}(ext_j) (.) key_j (the automorphism applied to the extended digits).
// The 2*dnum key words of a coefficient are loaded once and reused for all C ciphertexts.
// y = limb t of Q_l u P.
// OWN (one-limb digits): digit j's own limb t = j is read from own + ct * own_stride (the
// input's c1 in the NTT domain) instead of ext.
// MINB: CTAs per SM the register allocation is capped for (3 or 2); c_chunk: ciphertexts
// per thread (grid y = job x chunk; 0 = all C ciphertexts in one thread, the keys then
// read once per coefficient)
template <int MAXD, bool OWN, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ks_inner(const uint64_t *ext, int ext_per_job, const uint64_t *const *keys, const uint32_t *ginv,
                           uint64_t *out, uint32_t C, uint32_t L1, uint32_t W, uint32_t dnum, uint32_t n_q,
                           uint32_t nqp, uint32_t log_n, const DevPrime *P, const uint64_t *own,
                           uint64_t own_stride, const uint64_t *pc0, const uint64_t *pmod, uint32_t c_chunk) {
    pdl_enter();
    // grid y = job (varies before the limb, so the jobs of one limb run together and
    // share that limb's digit slice in L2) and chunk of ciphertexts, z = limb t of Q_l u P
    const uint32_t nch = c_chunk ? (C + c_chunk - 1) / c_chunk : 1;
    const uint32_t n = 1u << log_n, k = COEF(), r = blockIdx.y / nch, t = blockIdx.z;
    const uint32_t c_begin = c_chunk ? (blockIdx.y % nch) * c_chunk : 0;
    const uint32_t c_end = c_chunk ? min(C, c_begin + c_chunk) : C;
    const uint32_t pt = t < L1 ? t : n_q + (t - L1);
    const uint64_t q = P[pt].q, qinv = P[pt].qinv;
    const uint64_t key_plane = (uint64_t)nqp * n;
    const uint64_t *key = keys[r] + (uint64_t)pt * n + k;
    uint64_t k0[MAXD], k1[MAXD];
#pragma unroll
    for (int j = 0; j < MAXD; j++) {
        if (j < (int)dnum) {
            k0[j] = __ldg(key + (uint64_t)j * 2 * key_plane);
            k1[j] = __ldg(key + (uint64_t)j * 2 * key_plane + key_plane);
        }
    }
    const uint32_t g = ginv[r];
    const uint32_t kk = g == 1 ? k : auto_index(k, g, log_n);
    const uint64_t ext_ct = (uint64_t)dnum * W * n, out_ct = 2ull * W * n;
    for (uint32_t c = c_begin; c < c_end; c++) {
        const uint64_t cti = ext_per_job ? (uint64_t)r * C + c : c;
        const uint64_t *e = ext + cti * ext_ct + (uint64_t)t * n + k;
        uint64_t xs[MAXD];
#pragma unroll
        for (int j = 0; j < MAXD; j++)      // all digit loads issued before the products
            if (j < (int)dnum) xs[j] = (OWN && j == (int)t) ? own[cti * own_stride + (uint64_t)t * n + k]
                                                            : e[(uint64_t)j * W * n];
        u128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
            if (j < (int)dnum) {
                mac_raw(a0, xs[j], k0[j]);
                mac_raw(a1, xs[j], k1[j]);
                if ((j & 7) == 7) {
                    fold(a0, q);
                    fold(a1, q);
                }
            }
        }
        fold(a0, q);
        fold(a1, q);
        uint64_t v0 = mont_reduce(a0, q, qinv);
        const uint64_t v1 = mont_reduce(a1, q, qinv);
        uint64_t *o = out + ((uint64_t)r * C + c) * out_ct + (uint64_t)t * n + kk;
        // pc0 (outputs kept over Q_l u P): + P sigma_g(c0) = P c0[k] at position kk
        if (pc0 && t < L1) v0 = add_mod(v0, shoup(pc0[cti * own_stride + (uint64_t)t * n + k], pmod[2 * t],
                                                  pmod[2 * t + 1], q), q);
        o[0] = v0;
        o[(uint64_t)W * n] = v1;
    }
}

// The key inner product for one ciphertext whose extended digits all jobs share (hoisted
// rotations of a single input): a thread loads the digits of its coefficient once and runs RJ
// jobs (keys) on them; grid y = group of RJ jobs, z = limb.  Same sums as k_ks_inner.
template <int MAXD, bool OWN, int RJ>
__global__ void __launch_bounds__(256, 3) k_ks_inner_rj(const uint64_t *ext, const uint64_t *const *keys,
                                                        const uint32_t *ginv, uint64_t *out, uint32_t R, uint32_t L1,
                                                        uint32_t W, uint32_t dnum, uint32_t n_q, uint32_t nqp,
                                                        uint32_t log_n, const DevPrime *P, const uint64_t *own,
                                                        const uint64_t *pc0, const uint64_t *pmod) {
    pdl_enter();
    const uint32_t n = 1u << log_n, k = COEF(), r0 = blockIdx.y * RJ, t = blockIdx.z;
    const uint32_t pt = t < L1 ? t : n_q + (t - L1);
    const uint64_t q = P[pt].q, qinv = P[pt].qinv;
    const uint64_t key_plane = (uint64_t)nqp * n, out_ct = 2ull * W * n;
    uint64_t xs[MAXD];
    const uint64_t *e = ext + (uint64_t)t * n + k;
#pragma unroll
    for (int j = 0; j < MAXD; j++)
        if (j < (int)dnum) xs[j] = (OWN && j == (int)t) ? own[(uint64_t)t * n + k] : e[(uint64_t)j * W * n];
#pragma unroll 1
    for (int rr = 0; rr < RJ; rr++) {
        const uint32_t r = r0 + rr;
        if (r >= R) break;
        const uint64_t *key = keys[r] + (uint64_t)pt * n + k;
        uint64_t k0[MAXD], k1[MAXD];
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
            if (j < (int)dnum) {
                k0[j] = __ldg(key + (uint64_t)j * 2 * key_plane);
                k1[j] = __ldg(key + (uint64_t)j * 2 * key_plane + key_plane);
            }
        }
        u128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
            if (j < (int)dnum) {
                mac_raw(a0, xs[j], k0[j]);
                mac_raw(a1, xs[j], k1[j]);
                if ((j & 7) == 7) {
                    fold(a0, q);
                    fold(a1, q);
                }
            }
        }
        fold(a0, q);
        fold(a1, q);
        uint64_t v0 = mont_reduce(a0, q, qinv);
        const uint64_t v1 = mont_reduce(a1, q, qinv);
        const uint32_t g = ginv[r];
        const uint32_t kk = g == 1 ? k : auto_index(k, g, log_n);
        uint64_t *o = out + (uint64_t)r * out_ct + (uint64_t)t * n + kk;
        if (pc0 && t < L1) v0 = add_mod(v0, shoup(pc0[(uint64_t)t * n + k], pmod[2 * t], pmod[2 * t + 1], q), q);
        o[0] = v0;
        o[(uint64_t)W * n] = v1;
    }
}

// ---- 1-D bulk asynchronous copies (the TMA engine) completing on shared-memory mbarriers.
// A copy engine transfer keeps its bytes in flight without registers or L1 miss slots, which
// is what bounds the register-staged key reads of the shared-digit inner product at batch 1.
// Every wait is bounded: after kWaitLimit SM cycles (about a second) the CTA counts the
// timeout in g_wait_timeouts, waits (bounded again) for its own copies and returns; the host
// reads the count with hear_async_status.
__device__ unsigned int g_wait_timeouts;
constexpr long long kWaitLimit = 2000000000ll;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// the barrier's initialisation visible to the copy engine (the async proxy)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// wait for the phase of parity `parity` to complete; false after `limit` SM cycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// k_ks_inner_rj with the keys streamed by the copy engine: a CTA owns kBlock coefficients of
// limb t for RJ jobs; the 2 dnum key planes of a job (kBlock contiguous words each) come into
// one of two shared-memory buffers as bulk copies, the next job's keys landing while the
// current job's products run.  Same sums and outputs as k_ks_inner_rj.  Dynamic shared
// memory: 2 buffers x 2 dnum x kBlock words.
template <int MAXD, bool OWN, int RJ>
__global__ void __launch_bounds__(256, 3) k_ks_inner_rj_bulk(const uint64_t *ext, const uint64_t *const *keys,
                                                             const uint32_t *ginv, uint64_t *out, uint32_t R,
                                                             uint32_t L1, uint32_t W, uint32_t dnum, uint32_t n_q,
                                                             uint32_t nqp, uint32_t log_n, const DevPrime *P,
                                                             const uint64_t *own, const uint64_t *pc0,
                                                             const uint64_t *pmod) {
    extern __shared__ __align__(128) uint64_t skey[];
    __shared__ __align__(8) uint64_t bars[2];
    pdl_enter();
    const uint32_t n = 1u << log_n, k = COEF(), r0 = blockIdx.y * RJ, t = blockIdx.z;
    const uint32_t k_base = blockIdx.x * kBlock;
    const uint32_t pt = t < L1 ? t : n_q + (t - L1);
    const uint64_t q = P[pt].q, qinv = P[pt].qinv;
    const uint64_t key_plane = (uint64_t)nqp * n, out_ct = 2ull * W * n;
    const uint32_t planes = 2 * dnum, jobs = min((uint32_t)RJ, R - r0);
    // thread 0: the keys of job r0 + rr into buffer rr & 1
    auto issue = [&](uint32_t rr) {
        const uint32_t b = rr & 1, bar = smem_addr(&bars[b]);
        const uint64_t *src = keys[r0 + rr] + (uint64_t)pt * n + k_base;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, planes * kBlock * 8);
        for (uint32_t p = 0; p < planes; p++)
            bulk_g2s(smem_addr(skey + ((uint64_t)b * planes + p) * kBlock), src + (uint64_t)p * key_plane, kBlock * 8,
                     bar);
    };
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bars[0]), 1);
        mbar_init(smem_addr(&bars[1]), 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        issue(0);
        if (jobs > 1) issue(1);
    }
    uint64_t xs[MAXD];
    const uint64_t *e = ext + (uint64_t)t * n + k;
#pragma unroll
    for (int j = 0; j < MAXD; j++)
        if (j < (int)dnum) xs[j] = (OWN && j == (int)t) ? own[(uint64_t)t * n + k] : e[(uint64_t)j * W * n];
#pragma unroll 1
    for (uint32_t rr = 0; rr < jobs; rr++) {
        const uint32_t b = rr & 1;
        if (!__syncthreads_and(mbar_wait(smem_addr(&bars[b]), (rr >> 1) & 1, kWaitLimit))) {
            if (threadIdx.x == 0) {     // give up: count it, let the copies in flight land, return
                atomicAdd(&g_wait_timeouts, 1u);
                mbar_wait(smem_addr(&bars[b]), (rr >> 1) & 1, kWaitLimit);
                if (rr + 1 < jobs) mbar_wait(smem_addr(&bars[b ^ 1]), ((rr + 1) >> 1) & 1, kWaitLimit);
            }
            return;
        }
        const uint64_t *sk = skey + (uint64_t)b * planes * kBlock + threadIdx.x;
        uint64_t k0[MAXD], k1[MAXD];
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
            if (j < (int)dnum) {
                k0[j] = sk[(2u * j) * kBlock];
                k1[j] = sk[(2u * j + 1) * kBlock];
            }
        }
        __syncthreads();                // buffer b is read: refill it with job rr + 2
        if (threadIdx.x == 0 && rr + 2 < jobs) issue(rr + 2);
        u128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int j = 0; j < MAXD; j++) {
            if (j < (int)dnum) {
                mac_raw(a0, xs[j], k0[j]);
                mac_raw(a1, xs[j], k1[j]);
                if ((j & 7) == 7) {
                    fold(a0, q);
                    fold(a1, q);
                }
            }
        }
        fold(a0, q);
        fold(a1, q);
        uint64_t v0 = mont_reduce(a0, q, qinv);
        const uint64_t v1 = mont_reduce(a1, q, qinv);
        const uint32_t r = r0 + rr, g = ginv[r];
        const uint32_t kk = g == 1 ? k : auto_index(k, g, log_n);
        uint64_t *o = out + (uint64_t)r * out_ct + (uint64_t)t * n + kk;
        if (pc0 && t < L1) v0 = add_mod(v0, shoup(pc0[(uint64_t)t * n + k], pmod[2 * t], pmod[2 * t + 1], q), q);
        o[0] = v0;
        o[(uint64_t)W * n] = v1;
    }
}

// A wait that nothing completes: one CTA initialises a barrier, expects one arrival that
// never comes and waits with a limit of `limit` cycles; *status = 1 if the wait ran out (and
// the timeout was counted), 0 if it completed.
__global__ void k_wait_probe(long long limit, uint32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    pdl_enter();
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait(smem_addr(&bar), 0, limit);
        if (!ok) atomicAdd(&g_wait_timeouts, 1u);
        *status = ok ? 0u : 1u;
    }
}

// P x over Q_l u P: limb t < L1 is [P]_{q_t} x_t (pmod = (value, Shoup) pairs), the special
// limbs are zero.  y = limb t of W, z = polynomial.
__global__ void k_scale_p_ext(const uint64_t *x, uint64_t *out, uint32_t L1, uint32_t W, const uint64_t *pmod,
                              const DevPrime *P, uint32_t n) {
    pdl_enter();
    const uint32_t t = blockIdx.y, g = blockIdx.z, k = COEF();
    uint64_t v = 0;
    if (t < L1) v = shoup(x[((uint64_t)g * L1 + t) * n + k], pmod[2 * t], pmod[2 * t + 1], P[t].q);
    out[((uint64_t)g * W + t) * n + k] = v;
}
// ModDown conversion, one thread per (group = y + z*gridDim.y, coefficient):
// y_k = [x_{p_k} * phat_inv_k]_{p_k} once, conv_i = sum_k y_k * [P/p_k]_{q_i} mod q_i for
// every i < L1 (x_P in the coefficient domain).
// the P limbs of group g: xp + g * xp_gstride + kk * n (coefficient domain)
__global__ void k_moddown_conv(const uint64_t *xp, uint64_t xp_gstride, uint64_t *tmp, uint32_t n_groups, uint32_t L1,
                               uint32_t K, uint32_t n_q, const uint64_t *phat_inv, const uint64_t *phat_mod,
                               const DevPrime *P, uint32_t n) {
    pdl_enter();
    const uint32_t g = limb_yz(), k = COEF();
    if (g >= n_groups) return;
    uint64_t ys[4] = {0, 0, 0, 0};
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
        if (kk < (int)K) {
            const DevPrime pk = P[n_q + kk];
            ys[kk] = shoup(xp[(uint64_t)g * xp_gstride + (uint64_t)kk * n + k], phat_inv[2 * kk], phat_inv[2 * kk + 1],
                           pk.q);
        }
    }
    for (uint32_t t = 0; t < L1; t++) {
        const uint64_t q = P[t].q;
        uint64_t s = 0;
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            if (kk < (int)K) {
                const uint64_t *w = phat_mod + 2 * ((uint64_t)kk * L1 + t);
                s = add_mod(s, shoup(ys[kk], w[0], w[1], q), q);
            }
        }
        tmp[((uint64_t)g * L1 + t) * n + k] = s;
    }
}

// out = (x_i - conv_i) * P^-1 (+ addend gathered through sigma_g); y = limb, z = group.
// acc_count > 1: x is the sum mod q_t of acc_count inputs, input r at acc + r * acc_cstride
__global__ void k_moddown_combine(const uint64_t *acc, const uint64_t *tmp, uint64_t *out, const uint64_t *addend,
                                  uint64_t add_stride, uint32_t add_mask, uint32_t add_shared, const uint32_t *gal,
                                  uint32_t cts_per_job, uint32_t L1, uint32_t W, const uint64_t *p_inv,
                                  const DevPrime *P, uint32_t log_n, uint32_t acc_count, uint64_t acc_cstride) {
    pdl_enter();
    const uint32_t n = 1u << log_n, k = COEF(), t = blockIdx.y, g = blockIdx.z;
    const DevPrime p = P[t];
    const uint64_t i = ((uint64_t)g * L1 + t) * n + k;
    const uint64_t ai = ((uint64_t)g * W + t) * n + k;
    uint64_t x = acc[ai];
    for (uint32_t r = 1; r < acc_count; r++) x = add_mod(x, acc[r * acc_cstride + ai], p.q);
    uint64_t v = shoup(x + p.q - tmp[i], p_inv[2 * t], p_inv[2 * t + 1], p.q);
    const uint32_t poly = g & 1, c = g >> 1;
    if (addend && (add_mask >> poly & 1)) {
        const uint32_t ga = gal ? gal[c / cts_per_job] : 1u;
        const uint32_t kk = ga == 1 ? k : auto_index(k, ga, log_n);
        const uint32_t ac = add_shared ? c % cts_per_job : c;
        v = add_mod(v, addend[(uint64_t)ac * add_stride + ((uint64_t)poly * L1 + t) * n + kk], p.q);
    }
    out[i] = v;
}

// y = limb t < l, z = polynomial
__global__ void k_rescale_combine(const uint64_t *in, const uint64_t *tmp, uint64_t *out, uint32_t L1,
                                  const uint64_t *ql_inv, const DevPrime *P, uint32_t n) {
    pdl_enter();
    const uint32_t l = L1 - 1, k = COEF(), t = blockIdx.y, g = blockIdx.z;
    const DevPrime p = P[t];
    const uint64_t i = ((uint64_t)g * l + t) * n + k;
    const uint64_t x = in[((uint64_t)g * L1 + t) * n + k];
    out[i] = shoup(x + p.q - tmp[i], ql_inv[2 * t], ql_inv[2 * t + 1], p.q);
}

// split a count over grid y/z (y <= 65535)
inline void split_yz(uint32_t count, uint32_t &ny, uint32_t &nz) {
    if (count == 0) throw Error(HEAR_E_INVAL, "empty launch");
    ny = count < 65535 ? count : 65535;
    nz = (count + ny - 1) / ny;
    if (nz > 65535) throw Error(HEAR_E_UNSUPPORTED, "launch too large");
}

void check_yz(uint32_t y, uint32_t z) {
    if (y == 0 || z == 0) throw Error(HEAR_E_INVAL, "empty launch");
    if (y > 65535 || z > 65535) throw Error(HEAR_E_UNSUPPORTED, "launch too large");
}

}  // namespace

// launch with the profiler bracket; the stage name is the kernel's, `bytes` its algorithmic
// HBM traffic (each residue it must read or write, once)
// the launch form of table `tab` for a launch of `n` (ciphertexts or jobs): forced, or the
// context's tuned table (0 = the default form)
uint32_t ks_form(const hear_context *c, int tab, uint32_t n) {
    if (c->ks_force >= 0) return (uint32_t)c->ks_force % kKsVariants[tab];
    return c->ks_choice[tab][ks_bucket(n)] % kKsVariants[tab];
}

#define LAUNCH3(kernel, grid, block, st, bytes, ...)                                      \
    do {                                                                                  \
        ProfScope ps__(c, #kernel, st, (double)(bytes));                                   \
        launch(kernel, grid, block, 0, st, __VA_ARGS__);                                   \
    } while (0)

void to_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_to_mont, grid3(c->n, ny, nz), kBlock, s, 16.0 * n_limbs * c->n, d, n_limbs, m, c->dev_primes(), c->n, 1);
}
void from_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_to_mont, grid3(c->n, ny, nz), kBlock, s, 16.0 * n_limbs * c->n, d, n_limbs, m, c->dev_primes(), c->n, 0);
}
void pointwise_mont(const hear_context *c, uint32_t n_limbs, LimbMap m, const uint64_t *a, const uint64_t *b_mont,
                    uint64_t *out, cudaStream_t st) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_pointwise_mont, grid3(c->n, ny, nz), kBlock, st, 24.0 * n_limbs * c->n, a, b_mont, out, n_limbs, m,
            c->dev_primes(), c->n);
}
void small_to_limbs(const hear_context *c, const int8_t *e, uint64_t *out, uint32_t n_limbs, LimbMap m,
                    cudaStream_t s) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_small_to_limbs, grid3(c->n, ny, nz), kBlock, s, 8.0 * n_limbs * c->n, e, out, n_limbs, m,
            c->dev_primes(), c->n);
}
void i64_to_limbs(const hear_context *c, const int64_t *v, uint64_t *out, uint32_t n_limbs, LimbMap m,
                  cudaStream_t s) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_i64_to_limbs, grid3(c->n, ny, nz), kBlock, s, 8.0 * n_limbs * c->n, v, out, n_limbs, m,
            c->dev_primes(), c->n, 0ull);
}
void i64_to_limbs_batch(const hear_context *c, const int64_t *v, uint64_t *out, uint32_t n_polys, uint32_t level,
                        cudaStream_t s) {
    uint32_t ny, nz;
    const uint32_t n_limbs = n_polys * (level + 1);
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_i64_to_limbs, grid3(c->n, ny, nz), kBlock, s, 8.0 * n_limbs * c->n + 8.0 * n_polys * c->n, v, out,
            n_limbs, map_q(level, c->n_q), c->dev_primes(), c->n, (uint64_t)c->n);
}
void sample_small(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index, SmallKind kind,
                  int8_t *out, cudaStream_t s) {
    LAUNCH3(k_sample_small, dim3((c->n / 8 + kBlock - 1) / kBlock), kBlock, s, (double)c->n, seed, purpose, index,
            c->n, (int)kind, c->d_cdt.u64(), (uint32_t)c->cdt.size(), out);
}
void sample_uniform(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index_base, uint64_t *out,
                    uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    uint32_t ny, nz;
    split_yz(n_limbs, ny, nz);
    LAUNCH3(k_sample_uniform, dim3((c->n / 4 + kBlock - 1) / kBlock, ny, nz), kBlock, s, 8.0 * n_limbs * c->n, seed,
            purpose, index_base, out, n_limbs, m, c->dev_primes(), c->n);
}
void pk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, uint64_t *b,
                cudaStream_t st) {
    LAUNCH3(k_pk_combine, grid3(c->n, c->n_q, 1), kBlock, st, 32.0 * c->n_q * c->n, a, s_mont, e, b,
            c->dev_primes(), c->n);
}
void swk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e,
                 const uint64_t *sp_mont, const uint64_t *p_mod, uint32_t digit, uint64_t *b, cudaStream_t st) {
    uint32_t lo = digit * c->alpha, hi = std::min(lo + c->alpha, c->n_q);
    LAUNCH3(k_swk_combine, grid3(c->n, c->nqp(), 1), kBlock, st, 40.0 * c->nqp() * c->n, a, s_mont, e, sp_mont,
            p_mod, lo, hi, c->dev_primes(), c->n, b);
}
void encrypt_combine(const hear_context *c, const uint64_t *v, const uint64_t *e0, const uint64_t *e1,
                     const uint64_t *m, const uint64_t *pk_mont, uint64_t *ct, cudaStream_t st) {
    const uint64_t limbs = (uint64_t)c->n_q * c->n;
    LAUNCH3(k_encrypt_combine, grid3(c->n, c->n_q, 1), kBlock, st, 72.0 * limbs, v, e0, e1, m, pk_mont, ct, limbs,
            c->dev_primes(), c->n);
}
void decrypt_combine(const hear_context *c, uint32_t level, const uint64_t *ct, const uint64_t *s_mont,
                     uint64_t *out, cudaStream_t st) {
    const uint64_t limbs = (uint64_t)(level + 1) * c->n;
    LAUNCH3(k_decrypt_combine, grid3(c->n, level + 1, 1), kBlock, st, 32.0 * limbs, ct, s_mont, out, limbs,
            c->dev_primes(), c->n);
}
void add_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, const uint64_t *b,
            uint64_t *out, cudaStream_t st) {
    check_yz(level + 1, n_polys_total);
    LAUNCH3(k_add, grid3(c->n, level + 1, n_polys_total), kBlock, st, 24.0 * n_polys_total * (level + 1) * c->n,
            a, b, out, level + 1, c->dev_primes(), c->n);
}
void sum_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, uint64_t stride,
            uint32_t cnt, uint64_t *out, cudaStream_t st) {
    check_yz(level + 1, n_polys_total);
    LAUNCH3(k_sum, grid3(c->n, level + 1, n_polys_total), kBlock, st,
            8.0 * (cnt + 1) * n_polys_total * (level + 1) * c->n, a, stride, cnt, (const uint64_t *)nullptr, out,
            level + 1, c->dev_primes(), c->n);
}
void sum_add_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, uint64_t stride,
                uint32_t cnt, const uint64_t *base, uint64_t *out, cudaStream_t st) {
    check_yz(level + 1, n_polys_total);
    LAUNCH3(k_sum, grid3(c->n, level + 1, n_polys_total), kBlock, st,
            8.0 * (cnt + 2) * n_polys_total * (level + 1) * c->n, a, stride, cnt, base, out, level + 1,
            c->dev_primes(), c->n);
}
void tensor_ct(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *a, const uint64_t *b,
               uint64_t *out3, cudaStream_t st) {
    check_yz(level + 1, n_ct);
    LAUNCH3(k_tensor, grid3(c->n, level + 1, n_ct), kBlock, st, 56.0 * n_ct * (level + 1) * c->n, a, b, out3,
            level + 1, c->dev_primes(), c->n);
}
void automorphism(const hear_context *c, uint32_t level, uint32_t n_polys_total, uint32_t galois,
                  const uint64_t *in, uint64_t *out, cudaStream_t st) {
    uint32_t limbs = n_polys_total * (level + 1), ny, nz;
    split_yz(limbs, ny, nz);
    LAUNCH3(k_automorphism, grid3(c->n, ny, nz), kBlock, st, 16.0 * limbs * c->n, in, out, limbs, galois, c->log_n);
}
#define LC_SPLIT(C, LIMBS)                                                                                        \
    do {                                                                                                         \
        ProfScope ps__(c, "k_lincomb_split<" #C ">", st, bytes);                                                 \
        launch(k_lincomb_split<C>, gs, 256, 0, st, LIMBS, n1, n2, baby, pt, out, c->dev_primes(), c->n, L1,     \
               c->n_q);                                                                                          \
    } while (0)
// the k_lincomb form of table 2 for n_ct ciphertexts: 0 -> 4 accumulators, 1 -> 8, 2 -> 2, 3 -> 1,
// 4 -> baby steps split over the warps (k_lincomb_split, up to 4 ciphertexts; 4 accumulators above)
#define LINCOMB_FORMS(LIMBS)                                                                                     \
    do {                                                                                                         \
        const dim3 gs(c->n / 32, LIMBS);                                                                         \
        uint32_t form__ = ks_form(c, 2, n_ct);                                                                   \
        if (form__ == 4 && n_ct > 4) form__ = 0;                                                                 \
        switch (form__) {                                                                                        \
        case 4:                                                                                                  \
            switch (n_ct) {                                                                                      \
            case 1: LC_SPLIT(1, LIMBS); break;                                           \
            case 2: LC_SPLIT(2, LIMBS); break;                                           \
            case 3: LC_SPLIT(3, LIMBS); break;                                           \
            default: LC_SPLIT(4, LIMBS);                                                 \
            }                                                                                                    \
            break;                                                                                               \
        case 1: LAUNCH3(k_lincomb<8>, grid, 256, st, bytes, LIMBS, n_ct, n1, n2, baby, pt, out, c->dev_primes(), \
                        c->n, jw, L1, c->n_q); break;                                                            \
        case 2: LAUNCH3(k_lincomb<2>, grid, 256, st, bytes, LIMBS, n_ct, n1, n2, baby, pt, out, c->dev_primes(), \
                        c->n, jw, L1, c->n_q); break;                                                            \
        case 3: LAUNCH3(k_lincomb<1>, grid, 256, st, bytes, LIMBS, n_ct, n1, n2, baby, pt, out, c->dev_primes(), \
                        c->n, jw, L1, c->n_q); break;                                                            \
        default: LAUNCH3(k_lincomb<4>, grid, 256, st, bytes, LIMBS, n_ct, n1, n2, baby, pt, out,                 \
                         c->dev_primes(), c->n, jw, L1, c->n_q);                                                 \
        }                                                                                                        \
    } while (0)

void lincomb(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t n1, uint32_t n2, const uint64_t *baby,
             const uint64_t *pt, uint64_t *out, cudaStream_t st) {
    const uint32_t L1 = level + 1;
    dim3 grid((2 * n_ct + 7) / 8, c->n / 32, L1);
    HEAR_REQUIRE(grid.x < (1u << 31) && L1 <= 65535, HEAR_E_UNSUPPORTED, "launch too large");
    // algorithmic: every baby ciphertext, every plaintext and every output once
    const double bytes = 8.0 * L1 * c->n * (2.0 * n_ct * n1 + (double)n1 * n2 + 2.0 * n_ct * n2);
    const uint32_t jw = 2 * n_ct <= 4 ? 8 / (2 * n_ct) : 1;
    LINCOMB_FORMS(L1);
}
void lincomb_ext(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t n1, uint32_t n2, const uint64_t *baby,
                 const uint64_t *pt, uint64_t *out, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K;
    dim3 grid((2 * n_ct + 7) / 8, c->n / 32, W);
    HEAR_REQUIRE(grid.x < (1u << 31), HEAR_E_UNSUPPORTED, "launch too large");
    const double bytes = 8.0 * W * c->n * (2.0 * n_ct * n1 + (double)n1 * n2 + 2.0 * n_ct * n2);
    const uint32_t jw = 2 * n_ct <= 4 ? 8 / (2 * n_ct) : 1;
    LINCOMB_FORMS(W);
}
void mulplain(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *ct, const uint64_t *pt,
              uint64_t *out, cudaStream_t st) {
    check_yz(2 * (level + 1), n_ct);
    LAUNCH3(k_mulplain, grid3(c->n, 2 * (level + 1), n_ct), kBlock, st, 8.0 * (4.0 * n_ct + 1) * (level + 1) * c->n,
            ct, pt, out, level + 1, c->dev_primes(), c->n, n_ct);
}
void mulplain_grouped(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t cts_per_pt, const uint64_t *ct,
                      const uint64_t *pt, uint64_t *out, cudaStream_t st) {
    check_yz(2 * (level + 1), n_ct);
    HEAR_REQUIRE(cts_per_pt >= 1, HEAR_E_INVAL, "cts_per_pt must be positive");
    const double n_pt = (n_ct + cts_per_pt - 1) / cts_per_pt;
    LAUNCH3(k_mulplain, grid3(c->n, 2 * (level + 1), n_ct), kBlock, st,
            8.0 * (4.0 * n_ct + n_pt) * (level + 1) * c->n, ct, pt, out, level + 1, c->dev_primes(), c->n, cts_per_pt);
}
void add_plain(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t cts_per_pt, uint64_t *ct,
               const uint64_t *pt, cudaStream_t st) {
    check_yz(level + 1, n_ct);
    HEAR_REQUIRE(cts_per_pt >= 1, HEAR_E_INVAL, "cts_per_pt must be positive");
    const double n_pt = (n_ct + cts_per_pt - 1) / cts_per_pt;
    LAUNCH3(k_add_plain, grid3(c->n, level + 1, n_ct), kBlock, st, 8.0 * (2.0 * n_ct + n_pt) * (level + 1) * c->n, ct,
            pt, level + 1, c->dev_primes(), c->n, cts_per_pt);
}

void modup(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *c1, uint64_t c1_stride,
           uint64_t *ext, uint64_t *tmp, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level);
    const LevelConsts &lc = *c->levels[level];
    HEAR_REQUIRE(c->alpha <= 4, HEAR_E_UNSUPPORTED, "at most 4 special primes");
    // coefficient-domain copy of the digit limbs (the inverse NTT reads c1 in place of a copy)
    ntt_inverse_from(c, c1, c1_stride, tmp, n_ct * L1, map_q(level, c->n_q), st);
    LimbMap m = map_qp(level, c->n_q, c->K);
    m.skip_dnum = dnum;
    m.alpha = c->alpha;
    if (c->alpha == 1) {
        // one-limb digits: the extension of digit j to limb t is [a_j]_t, folded into the
        // forward transform's load; the digit's own limb stays in c1 (ks_inner reads it there)
        ntt_forward_pro(c, ext, n_ct * dnum * W, m, tmp, c->n, st);
        return;
    }
    check_yz(dnum, n_ct);
    LAUNCH3(k_modup_conv, grid3(c->n, dnum, n_ct), kBlock, st, 8.0 * n_ct * ((double)L1 + (double)dnum * W) * c->n,
            c1, c1_stride, tmp, ext, L1, W, dnum, c->alpha, c->n_q, lc.d.u64() + lc.off_qhat_inv,
            lc.d.u64() + lc.off_qhat_mod, c->dev_primes(), c->n);
    ntt_forward(c, ext, n_ct * dnum * W, m, st);
}

void ks_inner(const hear_context *c, uint32_t level, uint32_t R, uint32_t C, const uint64_t *ext, bool ext_per_job,
              const uint64_t *const *d_keys, const uint32_t *d_ginv, uint64_t *out, const uint64_t *c1,
              uint64_t c1_stride, cudaStream_t st, const uint64_t *pmod) {
    const uint64_t *own = c->alpha == 1 ? c1 : nullptr;
    // with pmod: the outputs stay over Q_l u P and receive P sigma_g(c0), c0 = c1 - one plane
    const uint64_t *pc0 = pmod ? c1 - (uint64_t)(level + 1) * c->n : nullptr;
    const uint32_t L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level);
    const double dn = dnum, wn = (double)W * c->n * 8.0;
    // algorithmic: each key once, each extended digit once (per job if not shared), each output once
    const double bytes = R * 2.0 * dn * wn + (ext_per_job ? (double)R * C : (double)C) * dn * wn + R * C * 2.0 * wn;
    // the form of the k_ks_inner launch: register cap (3 CTAs per SM, or 2 with no spills) x
    // ciphertexts per thread (all, or chunks of 4: more CTAs, keys read once per chunk)
    const uint32_t form = ks_form(c, 0, C);
    const uint32_t c_chunk = (form & 2) && C > 4 ? 4 : 0;
    const uint32_t nch = c_chunk ? (C + c_chunk - 1) / c_chunk : 1;
    check_yz(R * nch, W);
    const dim3 grid = grid3(c->n, R * nch, W);
#define KS_LAUNCH(NAME, D, O, MB)                                                                                 \
    do {                                                                                                          \
        ProfScope ps__(c, NAME, st, bytes);                                                                       \
        launch(k_ks_inner<D, O, MB>, grid, kBlock, 0, st, ext, (int)ext_per_job, d_keys, d_ginv, out, C, L1, W,   \
               dnum, c->n_q, c->nqp(), c->log_n, c->dev_primes(), own, c1_stride, pc0, pmod, c_chunk);            \
    } while (0)
#define KS_RJ(RJ)                                                                                                 \
    do {                                                                                                          \
        const dim3 g4(c->n / kBlock, (R + RJ - 1) / RJ, W);                                                      \
        ProfScope ps__(c, "k_ks_inner<8>", st, bytes);                                                            \
        if (own)                                                                                                  \
            launch(k_ks_inner_rj<8, true, RJ>, g4, kBlock, 0, st, ext, d_keys, d_ginv, out, R, L1, W, dnum,       \
                   c->n_q, c->nqp(), c->log_n, c->dev_primes(), own, pc0, pmod);                                  \
        else                                                                                                      \
            launch(k_ks_inner_rj<8, false, RJ>, g4, kBlock, 0, st, ext, d_keys, d_ginv, out, R, L1, W, dnum,      \
                   c->n_q, c->nqp(), c->log_n, c->dev_primes(), own, pc0, pmod);                                  \
    } while (0)
#define KS_RJ_BULK(RJ)                                                                                            \
    do {                                                                                                          \
        const dim3 g4(c->n / kBlock, (R + RJ - 1) / RJ, W);                                                      \
        const size_t smem = 2ull * 2 * dnum * kBlock * 8;                                                         \
        ProfScope ps__(c, "k_ks_inner<8>", st, bytes);                                                            \
        if (own)                                                                                                  \
            launch(k_ks_inner_rj_bulk<8, true, RJ>, g4, kBlock, smem, st, ext, d_keys, d_ginv, out, R, L1, W,     \
                   dnum, c->n_q, c->nqp(), c->log_n, c->dev_primes(), own, pc0, pmod);                            \
        else                                                                                                      \
            launch(k_ks_inner_rj_bulk<8, false, RJ>, g4, kBlock, smem, st, ext, d_keys, d_ginv, out, R, L1, W,    \
                   dnum, c->n_q, c->nqp(), c->log_n, c->dev_primes(), own, pc0, pmod);                            \
    } while (0)
    if (C == 1 && !ext_per_job && R >= 2 && dnum <= 8) {
        // one ciphertext whose digits all jobs share: RJ jobs per thread (4, 2 or 8), or RJ
        // jobs per CTA with the keys streamed by bulk copies (4 or 8)
        switch (ks_form(c, 1, R)) {
        case 1: KS_RJ(2); break;
        case 2: KS_RJ(8); break;
        case 3: KS_RJ_BULK(4); break;
        case 4: KS_RJ_BULK(8); break;
        default: KS_RJ(4);
        }
        HEAR_CHECK_CUDA(cudaGetLastError());
        return;
    }
    if (dnum <= 8) {
        const bool mb2 = form & 1;
        if (own && mb2) KS_LAUNCH("k_ks_inner<8>", 8, true, 2);
        else if (own) KS_LAUNCH("k_ks_inner<8>", 8, true, 3);
        else if (mb2) KS_LAUNCH("k_ks_inner<8>", 8, false, 2);
        else KS_LAUNCH("k_ks_inner<8>", 8, false, 3);
    } else if (dnum <= 16) {
        if (own) KS_LAUNCH("k_ks_inner<16>", 16, true, 3);
        else KS_LAUNCH("k_ks_inner<16>", 16, false, 3);
    } else {
        if (own) KS_LAUNCH("k_ks_inner<48>", 48, true, 3);
        else KS_LAUNCH("k_ks_inner<48>", 48, false, 3);
    }
#undef KS_LAUNCH
#undef KS_RJ
#undef KS_RJ_BULK
}

// dynamic shared memory of the bulk-copy inner products (64 KB at 8 digits) on the current device
void ks_bulk_setup() {
    const int smem = 2 * 2 * 8 * kBlock * 8;
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_ks_inner_rj_bulk<8, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_ks_inner_rj_bulk<8, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_ks_inner_rj_bulk<8, true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_ks_inner_rj_bulk<8, false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
}

uint32_t async_timeouts(bool clear) {
    uint32_t v = 0;
    HEAR_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)));
    if (clear && v) {
        const uint32_t z = 0;
        HEAR_CHECK_CUDA(cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof(z)));
    }
    return v;
}

uint32_t wait_probe(long long limit_cycles, cudaStream_t st) {
    DevBuf d(4, st);
    launch(k_wait_probe, dim3(1), dim3(32), 0, st, limit_cycles, static_cast<uint32_t *>(d.p));
    uint32_t v = 0;
    HEAR_CHECK_CUDA(cudaMemcpyAsync(&v, d.p, 4, cudaMemcpyDeviceToHost, st));
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    return v;
}

void scale_p_ext(const hear_context *c, uint32_t level, uint32_t n_polys, const uint64_t *x, uint64_t *out,
                 const uint64_t *pmod, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K;
    check_yz(W, n_polys);
    LAUNCH3(k_scale_p_ext, grid3(c->n, W, n_polys), kBlock, st, 8.0 * n_polys * ((double)L1 + W) * c->n, x, out, L1,
            W, pmod, c->dev_primes(), c->n);
}
void moddown(const hear_context *c, uint32_t level, uint32_t n_ct, uint64_t *acc, uint64_t *out,
             const uint64_t *addend, uint64_t add_stride, uint32_t add_mask, bool add_shared, const uint32_t *d_gal,
             uint32_t cts_per_job, uint64_t *tmp, cudaStream_t st, uint32_t acc_count, uint64_t acc_cstride) {
    const uint32_t L1 = level + 1, W = L1 + c->K, groups = n_ct * 2;
    const LevelConsts &lc = *c->levels[level];
    HEAR_REQUIRE(c->K <= 4, HEAR_E_UNSUPPORTED, "at most 4 special primes");
    HEAR_REQUIRE(acc_count >= 1, HEAR_E_INVAL, "ModDown of no input");
    // the P limbs in the coefficient domain: in place (one input) or, for a sum of inputs,
    // the inverse transform of their sum into a buffer of its own
    const uint64_t *xp = acc + (uint64_t)L1 * c->n;
    uint64_t xp_gstride = (uint64_t)W * c->n;
    DevBuf psum;
    if (acc_count == 1) {
        LimbMap pm;
        pm.per_group = c->K;
        pm.q_count = 0;
        pm.n_q = c->n_q;
        pm.group_stride = (uint64_t)W * c->n;
        ntt_inverse(c, acc + (uint64_t)L1 * c->n, groups * c->K, pm, st);
    } else {
        LimbMap pm;
        pm.per_group = c->K;
        pm.q_count = 0;
        pm.n_q = c->n_q;
        psum = DevBuf((size_t)groups * c->K * c->n * 8, st);
        ntt_inverse_from(c, acc + (uint64_t)L1 * c->n, (uint64_t)W * c->n, psum.u64(), groups * c->K, pm, st, acc_count,
                         acc_cstride);
        xp = psum.u64();
        xp_gstride = (uint64_t)c->K * c->n;
    }
    if (c->K == 1) {
        // one special prime: the conversion P -> q_t is [x_P]_t, folded into the load of the
        // forward transform
        ntt_forward_pro(c, tmp, groups * L1, map_q(level, c->n_q), xp, xp_gstride, st);
    } else {
        uint32_t ny, nz;
        split_yz(groups, ny, nz);
        LAUNCH3(k_moddown_conv, grid3(c->n, ny, nz), kBlock, st, 8.0 * groups * ((double)c->K + L1) * c->n, xp,
                xp_gstride, tmp, groups, L1, c->K, c->n_q, lc.d.u64() + lc.off_phat_inv, lc.d.u64() + lc.off_phat_mod,
                c->dev_primes(), c->n);
        ntt_forward(c, tmp, groups * L1, map_q(level, c->n_q), st);
    }
    check_yz(L1, groups);
    LAUNCH3(k_moddown_combine, grid3(c->n, L1, groups), kBlock, st,
            8.0 * groups * L1 * c->n * (2.0 + acc_count + (addend ? 1.0 : 0.0)), acc, tmp, out, addend, add_stride,
            add_mask, (uint32_t)add_shared, d_gal, cts_per_job, L1, W, lc.d.u64() + lc.off_p_inv, c->dev_primes(),
            c->log_n, acc_count, acc_cstride);
}

void rescale(const hear_context *c, uint32_t level, uint32_t n_polys, uint64_t *in, uint64_t *out, uint64_t *tmp,
             cudaStream_t st) {
    const uint32_t L1 = level + 1;
    const LevelConsts &lc = *c->levels[level];
    LimbMap lm;
    lm.per_group = 1;
    lm.q_base = level;
    lm.q_count = 1;
    lm.n_q = c->n_q;
    lm.group_stride = (uint64_t)L1 * c->n;
    ntt_inverse(c, in + (uint64_t)level * c->n, n_polys, lm, st);
    // the centred lift of the last limb to the other limbs, folded into the forward
    // transform's load
    ntt_forward_pro(c, tmp, n_polys * level, map_q(level - 1, c->n_q), in + (uint64_t)level * c->n,
                    (uint64_t)L1 * c->n, st, c->primes[level]);
    check_yz(level, n_polys);
    LAUNCH3(k_rescale_combine, grid3(c->n, level, n_polys), kBlock, st, 24.0 * n_polys * level * c->n, in, tmp, out,
            L1, lc.d.u64() + lc.off_ql_inv, c->dev_primes(), c->n);
}


// Time every launch form of the key-switch inner product and the BSGS inner sums on
// synthetic operands at the top level (the values do not change the work) for batches of
// 1, 2, 4, .. max_ct ciphertexts (inner products over 8 jobs; shared-digit products over
// 2 .. 16 jobs; inner sums over 32 x 4 baby / giant steps up to 4 ciphertexts, 8 x 8
// above), each as a replayed CUDA graph of `iters` launches, and record the fastest form
// per bucket.  Buckets above the tuned range keep the largest tuned bucket's form.
void ks_tune(hear_context *c, uint32_t max_ct, int iters, float *ms_out) {
    HEAR_REQUIRE(max_ct >= 1 && max_ct <= 64 && iters >= 1, HEAR_E_INVAL, "bad tuning range");
    cudaStream_t st = c->stream;
    const uint32_t level = c->L, L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level), n = c->n;
    const uint32_t R = 8, RMAX = 16;
    // inner sums: 32 baby x 4 giant steps for up to 4 ciphertexts (the shape of an FC layer of
    // 128 diagonals at batch 1, where the warp-split form applies), 8 x 8 above
    auto bsgs = [](uint32_t m) { return m <= 4 ? std::make_pair(32u, 4u) : std::make_pair(8u, 8u); };
    const uint64_t baby_planes = std::max<uint64_t>(32ull * 4, 8ull * max_ct);     // n1 x ciphertexts
    const uint64_t pt_planes = 32ull * 4;                                          // n1 x n2 (>= 8 x 8)
    const uint64_t sum_planes = std::max<uint64_t>(4ull * 4, 8ull * max_ct);       // n2 x ciphertexts
    const uint64_t plane = (uint64_t)n;
    const uint64_t key_words = (uint64_t)c->dnum_max() * 2 * c->nqp() * plane;
    DevBuf keys(RMAX * key_words * 8, st);
    const uint64_t n_src = std::max(max_ct, R);   // ciphertexts whose digits are read
    DevBuf ext(n_src * dnum * W * plane * 8, st);
    DevBuf c1(n_src * 2 * L1 * plane * 8, st);
    DevBuf out((uint64_t)std::max(max_ct * R, RMAX) * 2 * W * plane * 8, st);
    DevBuf baby(baby_planes * 2 * L1 * plane * 8, st);
    DevBuf pts(pt_planes * L1 * plane * 8, st);
    DevBuf sums(sum_planes * 2 * L1 * plane * 8, st);
    for (DevBuf *b : {&keys, &ext, &c1, &out, &baby, &pts, &sums}) HEAR_CHECK_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, st));
    std::vector<const uint64_t *> kp(RMAX);
    std::vector<uint32_t> gi(RMAX);
    uint64_t g = 1;
    for (uint32_t r = 0; r < RMAX; r++) {
        kp[r] = keys.u64() + r * key_words;
        g = g * 5 % (2ull * n);
        gi[r] = (uint32_t)g;
    }
    DevBuf d_kp(RMAX * sizeof(void *), st), d_gi(RMAX * 4, st);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(d_kp.p, kp.data(), RMAX * sizeof(void *), cudaMemcpyHostToDevice, st));
    HEAR_CHECK_CUDA(cudaMemcpyAsync(d_gi.p, gi.data(), RMAX * 4, cudaMemcpyHostToDevice, st));
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
    const uint64_t *const *dk = static_cast<const uint64_t *const *>(d_kp.p);
    const uint32_t *dg = static_cast<const uint32_t *>(d_gi.p);
    cudaEvent_t e0, e1;
    HEAR_CHECK_CUDA(cudaEventCreate(&e0));
    HEAR_CHECK_CUDA(cudaEventCreate(&e1));
    // ms of one launch of fn, timed as the second replay of a graph of `iters` launches
    auto time_graph = [&](const std::function<void()> &fn) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        HEAR_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            for (int i = 0; i < iters; i++) fn();
        } catch (...) {
            cudaStreamEndCapture(st, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        HEAR_CHECK_CUDA(cudaStreamEndCapture(st, &graph));
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        HEAR_CHECK_CUDA(e);
        float ms = 0;
        e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaGraphExecDestroy(exec);
        HEAR_CHECK_CUDA(e);
        return ms / iters;
    };
    const int saved = c->ks_force;
    try {
        for (int tab = 0; tab < kKsTables; tab++) {
            uint32_t last = 0;
            for (uint32_t b = 0; b < (uint32_t)kKsBuckets; b++) {
                const uint32_t m = 1u << b;
                if (tab == 1 ? (m < 2 || m > RMAX) : m > max_ct) continue;
                float best = 0;
                int best_v = 0;
                for (int v = 0; v < kKsVariants[tab]; v++) {
                    c->ks_force = v;
                    float ms = 0;
                    if (tab == 0)   // C = m ciphertexts per job (one ciphertext: digits per job)
                        ms = time_graph([&] {
                            ks_inner(c, level, R, m, ext.u64(), m == 1, dk, dg, out.u64(), c1.u64(),
                                     2ull * L1 * plane, st);
                        });
                    else if (tab == 1)   // one ciphertext, m jobs sharing its digits
                        ms = time_graph([&] {
                            ks_inner(c, level, m, 1, ext.u64(), false, dk, dg, out.u64(), c1.u64(), 2ull * L1 * plane, st);
                        });
                    else
                        ms = time_graph([&] {
                            lincomb(c, level, m, bsgs(m).first, bsgs(m).second, baby.u64(), pts.u64(), sums.u64(), st);
                        });
                    if (ms_out) ms_out[((size_t)tab * kKsBuckets + b) * kKsMaxForms + v] = ms;
                    if (v == 0 || ms < best) {
                        best = ms;
                        best_v = v;
                    }
                }
                c->ks_choice[tab][b] = (uint8_t)best_v;
                last = b;
            }
            for (uint32_t b = last + 1; b < (uint32_t)kKsBuckets; b++) c->ks_choice[tab][b] = c->ks_choice[tab][last];
        }
    } catch (...) {
        c->ks_force = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    c->ks_force = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace hear
