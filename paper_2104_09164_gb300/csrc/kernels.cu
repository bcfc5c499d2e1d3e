// kernels.cu -- elementwise, sampling and basis-conversion kernels of RNS-CKKS on sm_103a.
//
// All kernels are HBM-streaming: one thread per 64-bit residue (grid-stride), coalesced
// along the coefficient index.  The NTT domain ordering is that of ntt.cu: index i holds
// the evaluation at psi^(2 brv(i) + 1).
#include "kernels.cuh"
#include "modarith.cuh"

namespace hear {
namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(uint64_t total) {
    uint64_t g = (total + kBlock - 1) / kBlock;
    return (unsigned)(g > 0x7fffffffULL ? 0x7fffffffULL : (g ? g : 1));
}

#define GRID_STRIDE(i, total) for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (total); \
                                   i += (uint64_t)gridDim.x * blockDim.x)

// NTT-domain index of sigma_g: out[i] = in[perm(i)]
__device__ __forceinline__ uint32_t auto_index(uint32_t i, uint32_t galois, uint32_t log_n) {
    const uint32_t n2 = 2u << log_n;
    uint32_t e = 2 * (__brev(i) >> (32 - log_n)) + 1;
    uint32_t e2 = (uint32_t)(((uint64_t)e * galois) & (n2 - 1));
    return __brev((e2 - 1) >> 1) >> (32 - log_n);
}

// ------------------------------------------------------------------ representation
__global__ void k_to_mont(uint64_t *d, uint32_t n_limbs, LimbMap m, const DevPrime *P, uint32_t n, int dir) {
    GRID_STRIDE(i, (uint64_t)n_limbs * n) {
        uint32_t b = (uint32_t)(i / n), k = (uint32_t)(i % n), pi;
        if (!m.resolve(b, &pi)) continue;
        const DevPrime p = P[pi];
        uint64_t &x = d[m.offset(b, n) + k];
        x = dir ? mont_mul(x, p.r2, p.q, p.qinv) : mont_mul(x, 1, p.q, p.qinv);
    }
}

__global__ void k_pointwise_mont(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t n_limbs, LimbMap m,
                                 const DevPrime *P, uint32_t n) {
    GRID_STRIDE(i, (uint64_t)n_limbs * n) {
        uint32_t bb = (uint32_t)(i / n), k = (uint32_t)(i % n), pi;
        if (!m.resolve(bb, &pi)) continue;
        const DevPrime p = P[pi];
        uint64_t off = m.offset(bb, n) + k;
        out[off] = mont_mul(a[off], b[off], p.q, p.qinv);
    }
}

__global__ void k_small_to_limbs(const int8_t *e, uint64_t *out, uint32_t n_limbs, LimbMap m, const DevPrime *P,
                                 uint32_t n) {
    GRID_STRIDE(i, (uint64_t)n_limbs * n) {
        uint32_t b = (uint32_t)(i / n), k = (uint32_t)(i % n), pi;
        if (!m.resolve(b, &pi)) continue;
        int v = e[k];
        uint64_t q = P[pi].q;
        out[m.offset(b, n) + k] = v < 0 ? q - (uint64_t)(-v) : (uint64_t)v;
    }
}

__global__ void k_i64_to_limbs(const int64_t *v, uint64_t *out, uint32_t n_limbs, LimbMap m, const DevPrime *P,
                               uint32_t n) {
    GRID_STRIDE(i, (uint64_t)n_limbs * n) {
        uint32_t b = (uint32_t)(i / n), k = (uint32_t)(i % n), pi;
        if (!m.resolve(b, &pi)) continue;
        const DevPrime p = P[pi];
        int64_t x = v[k];
        uint64_t mag = x < 0 ? (uint64_t)0 - (uint64_t)x : (uint64_t)x;
        uint64_t r = reduce64(mag, p);
        out[m.offset(b, n) + k] = (x < 0) ? neg_mod(r, p.q) : r;
    }
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
    GRID_STRIDE(blk, (uint64_t)n / 8) {
        uint64_t w[8];
        chacha_words(seed, purpose, index, (uint32_t)blk, w);
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
}

// uniform residues: coefficient k of limb b is (w_{2k+1} 2^64 + w_{2k}) mod q, stream index
// index_base | prime(b)
__global__ void k_sample_uniform(uint64_t seed, uint32_t purpose, uint64_t index_base, uint64_t *out,
                                 uint32_t n_limbs, LimbMap m, const DevPrime *P, uint32_t n) {
    const uint32_t blocks_per_limb = n / 4;
    GRID_STRIDE(i, (uint64_t)n_limbs * blocks_per_limb) {
        uint32_t b = (uint32_t)(i / blocks_per_limb), blk = (uint32_t)(i % blocks_per_limb), pi;
        if (!m.resolve(b, &pi)) continue;
        const DevPrime p = P[pi];
        uint64_t w[8];
        chacha_words(seed, purpose, index_base | pi, blk, w);
        uint64_t *o = out + m.offset(b, n) + (uint64_t)blk * 4;
#pragma unroll
        for (int j = 0; j < 4; j++) o[j] = barrett_reduce(u128{w[2 * j], w[2 * j + 1]}, p.q, p.ratio_hi, p.ratio_lo);
    }
}

// ------------------------------------------------------------------ keys and encryption
__global__ void k_pk_combine(const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, uint64_t *b,
                             uint32_t n_q, const DevPrime *P, uint32_t n) {
    GRID_STRIDE(i, (uint64_t)n_q * n) {
        const DevPrime p = P[i / n];
        uint64_t as = mont_mul(a[i], s_mont[i], p.q, p.qinv);
        b[i] = sub_mod(e[i], as, p.q);
    }
}

__global__ void k_swk_combine(const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, const uint64_t *sp_mont,
                              const uint64_t *p_mod, uint32_t lo, uint32_t hi, uint32_t nqp, const DevPrime *P,
                              uint32_t n, uint64_t *b) {
    GRID_STRIDE(i, (uint64_t)nqp * n) {
        uint32_t t = (uint32_t)(i / n);
        const DevPrime p = P[t];
        uint64_t v = sub_mod(e[i], mont_mul(a[i], s_mont[i], p.q, p.qinv), p.q);
        if (t >= lo && t < hi) v = add_mod(v, mont_mul(p_mod[t], sp_mont[i], p.q, p.qinv), p.q);
        b[i] = v;
    }
}

__global__ void k_encrypt_combine(const uint64_t *v, const uint64_t *e0, const uint64_t *e1, const uint64_t *m,
                                  const uint64_t *pk_mont, uint64_t *ct, uint32_t n_q, const DevPrime *P,
                                  uint32_t n) {
    const uint64_t limbs = (uint64_t)n_q * n;
    GRID_STRIDE(i, limbs) {
        const DevPrime p = P[i / n];
        uint64_t c0 = add_mod(add_mod(mont_mul(v[i], pk_mont[i], p.q, p.qinv), e0[i], p.q), m[i], p.q);
        uint64_t c1 = add_mod(mont_mul(v[i], pk_mont[limbs + i], p.q, p.qinv), e1[i], p.q);
        ct[i] = c0;
        ct[limbs + i] = c1;
    }
}

__global__ void k_decrypt_combine(const uint64_t *ct, const uint64_t *s_mont, uint64_t *out, uint32_t L1,
                                  const DevPrime *P, uint32_t n) {
    const uint64_t limbs = (uint64_t)L1 * n;
    GRID_STRIDE(i, limbs) {
        const DevPrime p = P[i / n];
        out[i] = add_mod(ct[i], mont_mul(ct[limbs + i], s_mont[i], p.q, p.qinv), p.q);
    }
}

// ------------------------------------------------------------------ ciphertext arithmetic
__global__ void k_add(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t L1, uint64_t total,
                      const DevPrime *P, uint32_t n) {
    GRID_STRIDE(i, total) {
        uint32_t t = (uint32_t)((i / n) % L1);
        out[i] = add_mod(a[i], b[i], P[t].q);
    }
}

__global__ void k_tensor(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t L1, uint32_t n_ct,
                         const DevPrime *P, uint32_t n) {
    const uint64_t plane = (uint64_t)L1 * n;
    GRID_STRIDE(i, (uint64_t)n_ct * plane) {
        uint64_t c = i / plane, r = i % plane;
        const DevPrime p = P[r / n];
        const uint64_t *ac = a + c * 2 * plane, *bc = b + c * 2 * plane;
        uint64_t *oc = out + c * 3 * plane;
        uint64_t a0 = ac[r], a1 = ac[plane + r], b0 = bc[r], b1 = bc[plane + r];
        oc[r] = mul_mod(a0, b0, p);
        u128 s = mul_wide(a0, b1);
        add_to(s, mul_wide(a1, b0));
        oc[plane + r] = barrett_reduce(s, p.q, p.ratio_hi, p.ratio_lo);
        oc[2 * plane + r] = mul_mod(a1, b1, p);
    }
}

__global__ void k_automorphism(const uint64_t *in, uint64_t *out, uint64_t total, uint32_t galois, uint32_t log_n) {
    const uint32_t n = 1u << log_n;
    GRID_STRIDE(i, total) {
        uint64_t base = i & ~(uint64_t)(n - 1);
        uint32_t k = (uint32_t)(i & (n - 1));
        out[i] = in[base + auto_index(k, galois, log_n)];
    }
}

// lazily accumulate x*y into acc keeping acc.hi < q (so the final Montgomery reduce is valid)
__device__ __forceinline__ void mac_lazy(u128 &acc, uint64_t x, uint64_t y, uint64_t q) {
    add_to(acc, mul_wide(x, y));
    if (acc.hi >= q) acc.hi -= q;
}

template <int JB>
__global__ void k_lincomb(uint32_t L1, uint32_t n_ct, uint32_t n_in, uint32_t n_out, uint32_t j0,
                          const uint64_t *const *in, const uint64_t *const *pt, uint64_t *const *out,
                          const DevPrime *P, uint32_t n) {
    const uint64_t plane = (uint64_t)L1 * n;          // one polynomial
    GRID_STRIDE(i, (uint64_t)n_ct * plane) {
        uint64_t c = i / plane, r = i % plane;
        const DevPrime p = P[r / n];
        u128 acc0[JB], acc1[JB];
#pragma unroll
        for (int jj = 0; jj < JB; jj++) acc0[jj] = acc1[jj] = u128{0, 0};
        for (uint32_t b = 0; b < n_in; b++) {
            const uint64_t *src = in[b] + c * 2 * plane;
            uint64_t x0 = src[r], x1 = src[plane + r];
#pragma unroll
            for (int jj = 0; jj < JB; jj++) {
                uint32_t j = j0 + jj;
                if (j >= n_out) break;
                const uint64_t *w = pt[j * n_in + b];
                if (!w) continue;
                uint64_t wv = w[r];
                mac_lazy(acc0[jj], x0, wv, p.q);
                mac_lazy(acc1[jj], x1, wv, p.q);
            }
        }
#pragma unroll
        for (int jj = 0; jj < JB; jj++) {
            uint32_t j = j0 + jj;
            if (j >= n_out) break;
            uint64_t *dst = out[j] + c * 2 * plane;
            dst[r] = mont_reduce(acc0[jj], p.q, p.qinv);
            dst[plane + r] = mont_reduce(acc1[jj], p.q, p.qinv);
        }
    }
}

__global__ void k_mulplain(const uint64_t *ct, const uint64_t *pt, uint64_t *out, uint32_t L1, uint32_t n_ct,
                           const DevPrime *P, uint32_t n) {
    const uint64_t plane = (uint64_t)L1 * n;
    GRID_STRIDE(i, (uint64_t)n_ct * 2 * plane) {
        uint64_t r = i % plane;
        const DevPrime p = P[r / n];
        out[i] = mont_mul(ct[i], pt[r], p.q, p.qinv);
    }
}

// ------------------------------------------------------------------ key switching
// ext[c][j][t][k]: limbs t in I_j copy c1 (NTT domain); other limbs get the basis
// conversion of the (scaled) coefficient-domain digit limbs y (NTT applied afterwards).
__global__ void k_modup_conv(const uint64_t *c1, uint64_t c1_stride, const uint64_t *y, uint64_t *ext,
                             uint32_t L1, uint32_t W, uint32_t dnum, uint32_t alpha, uint32_t n_q,
                             const uint64_t *qhat_inv, const uint64_t *qhat_mod, const DevPrime *P, uint32_t n,
                             uint32_t n_ct) {
    GRID_STRIDE(i, (uint64_t)n_ct * dnum * W * n) {
        uint32_t k = (uint32_t)(i % n);
        uint64_t rest = i / n;
        uint32_t t = (uint32_t)(rest % W);
        rest /= W;
        uint32_t j = (uint32_t)(rest % dnum);
        uint32_t c = (uint32_t)(rest / dnum);
        uint32_t lo = j * alpha, hi = min(lo + alpha, L1);
        if (t >= lo && t < hi) {
            ext[i] = c1[c * c1_stride + (uint64_t)t * n + k];
            continue;
        }
        uint32_t pt = t < L1 ? t : n_q + (t - L1);
        const DevPrime p = P[pt];
        uint64_t acc = 0;
        for (uint32_t src = lo; src < hi; src++) {
            const DevPrime ps = P[src];
            uint64_t a = y[((uint64_t)c * L1 + src) * n + k];
            uint64_t yi = shoup(a, qhat_inv[2 * src], qhat_inv[2 * src + 1], ps.q);
            const uint64_t *wm = qhat_mod + 2 * (((uint64_t)j * alpha + (src - lo)) * W + t);
            acc = add_mod(acc, shoup(yi, wm[0], wm[1], p.q), p.q);
        }
        ext[i] = acc;
    }
}

__global__ void k_ks_inner(const uint64_t *ext, const uint64_t *const *keys, const uint32_t *galois,
                           uint64_t *out, uint32_t L1, uint32_t W, uint32_t dnum, uint32_t n_q, uint32_t nqp,
                           uint32_t log_n, const DevPrime *P, uint32_t n_ct) {
    const uint32_t n = 1u << log_n;
    GRID_STRIDE(i, (uint64_t)n_ct * W * n) {
        uint32_t k = (uint32_t)(i % n);
        uint32_t t = (uint32_t)((i / n) % W);
        uint32_t c = (uint32_t)(i / ((uint64_t)W * n));
        uint32_t pt = t < L1 ? t : n_q + (t - L1);
        const DevPrime p = P[pt];
        uint32_t g = galois ? galois[c] : 1u;
        uint32_t kk = g == 1 ? k : auto_index(k, g, log_n);
        const uint64_t *key = keys[c];
        const uint64_t key_plane = (uint64_t)nqp * n;
        u128 a0{0, 0}, a1{0, 0};
        for (uint32_t j = 0; j < dnum; j++) {
            uint64_t x = ext[(((uint64_t)c * dnum + j) * W + t) * n + kk];
            const uint64_t *kj = key + (uint64_t)j * 2 * key_plane + (uint64_t)pt * n + k;
            mac_lazy(a0, x, kj[0], p.q);
            mac_lazy(a1, x, kj[key_plane], p.q);
        }
        uint64_t *o = out + (uint64_t)c * 2 * W * n + (uint64_t)t * n + k;
        o[0] = mont_reduce(a0, p.q, p.qinv);
        o[(uint64_t)W * n] = mont_reduce(a1, p.q, p.qinv);
    }
}

// conv_i = sum_k [x_{p_k} * phat_inv_k]_{p_k} * phat_mod[k][i] mod q_i (x_P coefficient domain)
__global__ void k_moddown_conv(const uint64_t *acc, uint64_t *tmp, uint32_t L1, uint32_t W, uint32_t K,
                               uint32_t n_q, const uint64_t *phat_inv, const uint64_t *phat_mod,
                               const DevPrime *P, uint32_t n, uint32_t n_groups) {
    GRID_STRIDE(i, (uint64_t)n_groups * L1 * n) {
        uint32_t k = (uint32_t)(i % n);
        uint32_t t = (uint32_t)((i / n) % L1);
        uint32_t g = (uint32_t)(i / ((uint64_t)L1 * n));
        const DevPrime p = P[t];
        uint64_t s = 0;
        for (uint32_t kk = 0; kk < K; kk++) {
            const DevPrime pk = P[n_q + kk];
            uint64_t x = acc[((uint64_t)g * W + L1 + kk) * n + k];
            uint64_t y = shoup(x, phat_inv[2 * kk], phat_inv[2 * kk + 1], pk.q);
            const uint64_t *w = phat_mod + 2 * ((uint64_t)kk * L1 + t);
            s = add_mod(s, shoup(y, w[0], w[1], p.q), p.q);
        }
        tmp[i] = s;
    }
}

__global__ void k_moddown_combine(const uint64_t *acc, const uint64_t *tmp, uint64_t *out, const uint64_t *addend,
                                  uint64_t add_stride, uint32_t add_mask, const uint32_t *galois, uint32_t L1, uint32_t W,
                                  const uint64_t *p_inv, const DevPrime *P, uint32_t log_n, uint32_t n_groups) {
    const uint32_t n = 1u << log_n;
    GRID_STRIDE(i, (uint64_t)n_groups * L1 * n) {
        uint32_t k = (uint32_t)(i % n);
        uint32_t t = (uint32_t)((i / n) % L1);
        uint32_t g = (uint32_t)(i / ((uint64_t)L1 * n));
        const DevPrime p = P[t];
        uint64_t x = acc[((uint64_t)g * W + t) * n + k];
        uint64_t v = shoup(x + p.q - tmp[i], p_inv[2 * t], p_inv[2 * t + 1], p.q);
        uint32_t poly = g & 1, c = g >> 1;
        if (addend && (add_mask >> poly & 1)) {
            uint32_t gal = galois ? galois[c] : 1u;
            uint32_t kk = gal == 1 ? k : auto_index(k, gal, log_n);
            v = add_mod(v, addend[(uint64_t)c * add_stride + ((uint64_t)poly * L1 + t) * n + kk], p.q);
        }
        out[i] = v;
    }
}

// w_i = [c_l]_centred mod q_i for the coefficient-domain last limb c_l
__global__ void k_rescale_lift(const uint64_t *in, uint64_t *tmp, uint32_t L1, const DevPrime *P, uint32_t n,
                               uint32_t n_polys) {
    const uint32_t l = L1 - 1;
    const uint64_t ql = P[l].q, half = (ql - 1) / 2;
    GRID_STRIDE(i, (uint64_t)n_polys * l * n) {
        uint32_t k = (uint32_t)(i % n);
        uint32_t t = (uint32_t)((i / n) % l);
        uint32_t g = (uint32_t)(i / ((uint64_t)l * n));
        const DevPrime p = P[t];
        uint64_t v = in[((uint64_t)g * L1 + l) * n + k];
        uint64_t w;
        if (v > half) w = neg_mod(reduce64(ql - v, p), p.q);
        else w = reduce64(v, p);
        tmp[i] = w;
    }
}

__global__ void k_rescale_combine(const uint64_t *in, const uint64_t *tmp, uint64_t *out, uint32_t L1,
                                  const uint64_t *ql_inv, const DevPrime *P, uint32_t n, uint32_t n_polys) {
    const uint32_t l = L1 - 1;
    GRID_STRIDE(i, (uint64_t)n_polys * l * n) {
        uint32_t k = (uint32_t)(i % n);
        uint32_t t = (uint32_t)((i / n) % l);
        uint32_t g = (uint32_t)(i / ((uint64_t)l * n));
        const DevPrime p = P[t];
        uint64_t x = in[((uint64_t)g * L1 + t) * n + k];
        out[i] = shoup(x + p.q - tmp[i], ql_inv[2 * t], ql_inv[2 * t + 1], p.q);
    }
}

}  // namespace

// launch with the profiler bracket; the stage name is the kernel's, the algorithmic bytes
// are those of one residue read or written per element unless a launcher says otherwise
#define LAUNCH_B(kernel, total, st, bytes, ...)                                           \
    do {                                                                                  \
        ProfScope ps__(c, #kernel, st, (double)(bytes));                                   \
        kernel<<<grid_for(total), kBlock, 0, st>>>(__VA_ARGS__);                           \
        HEAR_CHECK_CUDA(cudaGetLastError());                                               \
    } while (0)
#define LAUNCH(kernel, total, st, ...) LAUNCH_B(kernel, total, st, 16.0 * (double)(total), __VA_ARGS__)

void to_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    LAUNCH(k_to_mont, (uint64_t)n_limbs * c->n, s, d, n_limbs, m, c->dev_primes(), c->n, 1);
}
void from_mont(const hear_context *c, uint64_t *d, uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    LAUNCH(k_to_mont, (uint64_t)n_limbs * c->n, s, d, n_limbs, m, c->dev_primes(), c->n, 0);
}
void pointwise_mont(const hear_context *c, uint32_t n_limbs, LimbMap m, const uint64_t *a, const uint64_t *b_mont,
                    uint64_t *out, cudaStream_t st) {
    LAUNCH(k_pointwise_mont, (uint64_t)n_limbs * c->n, st, a, b_mont, out, n_limbs, m, c->dev_primes(), c->n);
}
void small_to_limbs(const hear_context *c, const int8_t *e, uint64_t *out, uint32_t n_limbs, LimbMap m,
                    cudaStream_t s) {
    LAUNCH(k_small_to_limbs, (uint64_t)n_limbs * c->n, s, e, out, n_limbs, m, c->dev_primes(), c->n);
}
void i64_to_limbs(const hear_context *c, const int64_t *v, uint64_t *out, uint32_t n_limbs, LimbMap m,
                  cudaStream_t s) {
    LAUNCH(k_i64_to_limbs, (uint64_t)n_limbs * c->n, s, v, out, n_limbs, m, c->dev_primes(), c->n);
}
void sample_small(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index, SmallKind kind,
                  int8_t *out, cudaStream_t s) {
    LAUNCH(k_sample_small, (uint64_t)c->n / 8, s, seed, purpose, index, c->n, (int)kind, c->d_cdt.u64(),
           (uint32_t)c->cdt.size(), out);
}
void sample_uniform(const hear_context *c, uint64_t seed, uint32_t purpose, uint64_t index_base, uint64_t *out,
                    uint32_t n_limbs, LimbMap m, cudaStream_t s) {
    LAUNCH(k_sample_uniform, (uint64_t)n_limbs * (c->n / 4), s, seed, purpose, index_base, out, n_limbs, m,
           c->dev_primes(), c->n);
}
void pk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e, uint64_t *b,
                cudaStream_t st) {
    LAUNCH(k_pk_combine, (uint64_t)c->n_q * c->n, st, a, s_mont, e, b, c->n_q, c->dev_primes(), c->n);
}
void swk_combine(const hear_context *c, const uint64_t *a, const uint64_t *s_mont, const uint64_t *e,
                 const uint64_t *sp_mont, const uint64_t *p_mod, uint32_t digit, uint64_t *b, cudaStream_t st) {
    uint32_t lo = digit * c->alpha, hi = std::min(lo + c->alpha, c->n_q);
    LAUNCH(k_swk_combine, (uint64_t)c->nqp() * c->n, st, a, s_mont, e, sp_mont, p_mod, lo, hi, c->nqp(),
           c->dev_primes(), c->n, b);
}
void encrypt_combine(const hear_context *c, const uint64_t *v, const uint64_t *e0, const uint64_t *e1,
                     const uint64_t *m, const uint64_t *pk_mont, uint64_t *ct, cudaStream_t st) {
    LAUNCH(k_encrypt_combine, (uint64_t)c->n_q * c->n, st, v, e0, e1, m, pk_mont, ct, c->n_q, c->dev_primes(),
           c->n);
}
void decrypt_combine(const hear_context *c, uint32_t level, const uint64_t *ct, const uint64_t *s_mont,
                     uint64_t *out, cudaStream_t st) {
    LAUNCH(k_decrypt_combine, (uint64_t)(level + 1) * c->n, st, ct, s_mont, out, level + 1, c->dev_primes(),
           c->n);
}
void add_ct(const hear_context *c, uint32_t level, uint32_t n_polys_total, const uint64_t *a, const uint64_t *b,
            uint64_t *out, cudaStream_t st) {
    uint64_t total = (uint64_t)n_polys_total * (level + 1) * c->n;
    LAUNCH(k_add, total, st, a, b, out, level + 1, total, c->dev_primes(), c->n);
}
void tensor_ct(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *a, const uint64_t *b,
               uint64_t *out3, cudaStream_t st) {
    LAUNCH(k_tensor, (uint64_t)n_ct * (level + 1) * c->n, st, a, b, out3, level + 1, n_ct, c->dev_primes(), c->n);
}
void automorphism(const hear_context *c, uint32_t level, uint32_t n_polys_total, uint32_t galois,
                  const uint64_t *in, uint64_t *out, cudaStream_t st) {
    uint64_t total = (uint64_t)n_polys_total * (level + 1) * c->n;
    LAUNCH(k_automorphism, total, st, in, out, total, galois, c->log_n);
}
void lincomb(const hear_context *c, uint32_t level, uint32_t n_ct, uint32_t n_in, uint32_t n_out,
             const uint64_t *const *d_in, const uint64_t *const *d_pt, uint64_t *const *d_out, cudaStream_t st) {
    constexpr int JB = 4;
    for (uint32_t j0 = 0; j0 < n_out; j0 += JB)
        LAUNCH(k_lincomb<JB>, (uint64_t)n_ct * (level + 1) * c->n, st, level + 1, n_ct, n_in, n_out, j0, d_in,
               d_pt, d_out, c->dev_primes(), c->n);
}
void mulplain(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *ct, const uint64_t *pt,
              uint64_t *out, cudaStream_t st) {
    LAUNCH(k_mulplain, (uint64_t)n_ct * 2 * (level + 1) * c->n, st, ct, pt, out, level + 1, n_ct, c->dev_primes(),
           c->n);
}

void modup(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *c1, uint64_t c1_stride,
           uint64_t *ext, uint64_t *tmp, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K, dnum = c->dnum(level);
    const LevelConsts &lc = *c->levels[level];
    // coefficient-domain copy of the digit limbs
    for (uint32_t i = 0; i < n_ct; i++)
        HEAR_CHECK_CUDA(cudaMemcpyAsync(tmp + (uint64_t)i * L1 * c->n, c1 + i * c1_stride,
                                        (size_t)L1 * c->n * 8, cudaMemcpyDeviceToDevice, st));
    ntt_inverse(c, tmp, n_ct * L1, map_q(level, c->n_q), st);
    LAUNCH(k_modup_conv, (uint64_t)n_ct * dnum * W * c->n, st, c1, c1_stride, tmp, ext, L1, W, dnum, c->alpha,
           c->n_q, lc.d.u64() + lc.off_qhat_inv, lc.d.u64() + lc.off_qhat_mod, c->dev_primes(), c->n, n_ct);
    LimbMap m = map_qp(level, c->n_q, c->K);
    m.skip_dnum = dnum;
    m.alpha = c->alpha;
    ntt_forward(c, ext, n_ct * dnum * W, m, st);
}

void ks_inner(const hear_context *c, uint32_t level, uint32_t n_ct, const uint64_t *ext,
              const uint64_t *const *d_keys, const uint32_t *d_galois, uint64_t *out, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K;
    const double dn = c->dnum(level), wn = (double)W * c->n * 8.0;
    // keys are read once per distinct key; the batch shares them when n_ct > 1 and the key is common
    LAUNCH_B(k_ks_inner, (uint64_t)n_ct * W * c->n, st, 2.0 * dn * wn + n_ct * (dn + 2.0) * wn, ext, d_keys,
             d_galois, out, L1, W, c->dnum(level), c->n_q, c->nqp(), c->log_n, c->dev_primes(), n_ct);
}

void moddown(const hear_context *c, uint32_t level, uint32_t n_ct, uint64_t *acc, uint64_t *out,
             const uint64_t *addend, uint64_t add_stride, uint32_t add_mask, const uint32_t *d_galois,
             uint64_t *tmp, cudaStream_t st) {
    const uint32_t L1 = level + 1, W = L1 + c->K, groups = n_ct * 2;
    const LevelConsts &lc = *c->levels[level];
    LimbMap pm;
    pm.per_group = c->K;
    pm.q_count = 0;
    pm.n_q = c->n_q;
    pm.group_stride = (uint64_t)W * c->n;
    ntt_inverse(c, acc + (uint64_t)L1 * c->n, groups * c->K, pm, st);
    LAUNCH(k_moddown_conv, (uint64_t)groups * L1 * c->n, st, acc, tmp, L1, W, c->K, c->n_q,
           lc.d.u64() + lc.off_phat_inv, lc.d.u64() + lc.off_phat_mod, c->dev_primes(), c->n, groups);
    ntt_forward(c, tmp, groups * L1, map_q(level, c->n_q), st);
    LAUNCH(k_moddown_combine, (uint64_t)groups * L1 * c->n, st, acc, tmp, out, addend, add_stride, add_mask,
           d_galois, L1, W,
           lc.d.u64() + lc.off_p_inv, c->dev_primes(), c->log_n, groups);
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
    LAUNCH(k_rescale_lift, (uint64_t)n_polys * level * c->n, st, in, tmp, L1, c->dev_primes(), c->n, n_polys);
    ntt_forward(c, tmp, n_polys * level, map_q(level - 1, c->n_q), st);
    LAUNCH(k_rescale_combine, (uint64_t)n_polys * level * c->n, st, in, tmp, out, L1, lc.d.u64() + lc.off_ql_inv,
           c->dev_primes(), c->n, n_polys);
}

}  // namespace hear
