// internal.h -- shared declarations of the CUDA library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>
#include "hear.h"   // include/ is on the include path

namespace hear {

constexpr int kMaxPrimes = 48;

// Error carried to the C ABI boundary.
struct Error : std::runtime_error {
    hear_status code;
    Error(hear_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};
#define HEAR_CHECK_CUDA(expr)                                                              \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            throw ::hear::Error(HEAR_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)
#define HEAR_REQUIRE(cond, code, msg)                                                      \
    do {                                                                                   \
        if (!(cond)) throw ::hear::Error((code), (msg));                                   \
    } while (0)

// Per-prime constants, device resident.
struct DevPrime {
    uint64_t q;
    uint64_t qinv;       // q^-1 mod 2^64 (Montgomery)
    uint64_t r2;         // 2^128 mod q (into Montgomery form)
    uint64_t ratio_hi;   // floor(2^128 / q), high word (Barrett)
    uint64_t ratio_lo;   //                   low word
    uint64_t n_inv;      // N^-1 mod q
    uint64_t n_inv_sh;   // Shoup companion of n_inv
    uint64_t one_sh;     // Shoup companion of 1 = floor(2^64 / q)
};

// A caller-supplied device allocator (hear_set_allocator): alloc(bytes, stream, user) and
// free(ptr, stream, user).  While an ABI call of a context that has one runs, the calling
// thread's allocations go through it (see AllocScope), except inside a stream capture,
// whose memory the graph owns.
struct Allocator {
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*free)(void *, void *, void *) = nullptr;
    void *user = nullptr;
};
extern thread_local const Allocator *tl_allocator;
struct AllocScope {
    const Allocator *prev;
    explicit AllocScope(const Allocator *a) : prev(tl_allocator) { tl_allocator = (a && a->alloc) ? a : nullptr; }
    ~AllocScope() { tl_allocator = prev; }
};

// Device memory owned through the stream-ordered allocator (or the caller's allocator).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    void (*free_fn)(void *, void *, void *) = nullptr;   // set: p came from a caller's allocator
    void *free_user = nullptr;
    DevBuf() = default;
    DevBuf(size_t b, cudaStream_t st);
    ~DevBuf();
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
    DevBuf &operator=(DevBuf &&o) noexcept;
    uint64_t *u64() const { return static_cast<uint64_t *>(p); }
    void reset();
};

// Basis-conversion constants of one level (ModUp / ModDown / rescale), device resident.
// ModUp, digit j (source limbs i in I_j = [j*alpha, min((j+1)*alpha, l+1))):
//   y_i = a_i * qhat_inv_i mod q_i, conv_t = sum_i y_i * qhat_mod[j][i - j*alpha][t] mod t.
// ModDown: y_k = x_k * phat_inv_k mod p_k, conv_i = sum_k y_k * phat_mod[k][i] mod q_i,
//   out_i = (x_i - conv_i) * P^-1 mod q_i.
// Rescale (to l-1): out_i = (c_i - [c_l]_centred) * q_l^-1 mod q_i.
struct LevelConsts {
    uint32_t level = 0, dnum = 0, width = 0;  // width = l+1+K
    DevBuf d;                                  // all tables of this level, packed
    // offsets (in uint64 words) into d; each table entry is a (value, Shoup) pair
    size_t off_qhat_inv = 0;   // [l+1] pairs (mod the limb's own prime)
    size_t off_qhat_mod = 0;   // [dnum][alpha][width] pairs (mod target prime)
    size_t off_phat_inv = 0;   // [K] pairs
    size_t off_phat_mod = 0;   // [K][l+1] pairs
    size_t off_p_inv = 0;      // [l+1] pairs: P^-1 mod q_i
    size_t off_ql_inv = 0;     // [l] pairs: q_l^-1 mod q_i (rescale from level l)
    size_t off_nql_half = 0;   // unused
};

// Stage profiler: when enabled, every kernel launch of the context is bracketed by CUDA
// events on its stream and tagged with a stage name and its algorithmic HBM bytes.
struct Profiler {
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
        double bytes;
        uint32_t launches;
    };
    bool on = false;
    std::mutex mu;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> spare;
    cudaEvent_t get();
    void clear();
};

// total kernel launches issued by the library since it was loaded
extern std::atomic<uint64_t> g_launches;
extern std::atomic<uint64_t> g_pdl_launches;

}  // namespace hear

// ------------------------------------------------------------------ handles
// NTT launch variants (ntt.cu): two-pass wide tiles, two-pass narrow tiles, one-launch
// cluster form, two-pass tiny tiles (radix-4 units); kNttAuto = the default rule
enum : uint8_t { kNttWide = 0, kNttNarrow = 1, kNttFused = 2, kNttTiny = 3, kNttAuto = 255 };
constexpr int kNttVariants = 4;
constexpr int kNttBuckets = 16;   // launches of 1, 2-3, 4-7, .. limbs (log2 buckets)
inline uint32_t ntt_bucket(uint32_t n_limbs) {
    uint32_t b = 0;
    while ((2u << b) <= n_limbs && b + 1 < (uint32_t)kNttBuckets) b++;
    return b;
}

// launch forms of the key-switch inner product and the BSGS inner sums (kernels.cu), per
// log2 bucket of the batch: [0] k_ks_inner by ciphertexts per job (4 forms: register cap
// for 3 or 2 CTAs per SM x all ciphertexts per thread or chunks of 4), [1] k_ks_inner_rj by
// jobs (4, 2 or 8 jobs per thread; 4 or 8 jobs per CTA with the keys streamed by bulk
// copies), [2] k_lincomb by ciphertexts (4, 8, 2 or 1 accumulators per thread; the baby
// steps split over the warps for up to 4 ciphertexts); every form computes the same residues
constexpr int kKsTables = 3;
constexpr int kKsBuckets = 8;
constexpr int kKsMaxForms = 8;     // hear_ks_tune's ms_out: [kKsTables][kKsBuckets][kKsMaxForms]
constexpr int kKsVariants[kKsTables] = {4, 5, 5};
inline uint32_t ks_bucket(uint32_t n) {
    uint32_t b = 0;
    while ((2u << b) <= n && b + 1 < (uint32_t)kKsBuckets) b++;
    return b;
}

struct hear_context {
    int device = 0;
    int ks_force = -1;                        // debug: force one form in every table (-1 = tables)
    uint8_t ks_choice[kKsTables][kKsBuckets] = {};   // 0 = the default form
    hear::Allocator allocator;                // hear_set_allocator (none = the stream-ordered pool)
    int ntt_force = -1;                       // debug: force one NTT variant (-1 = table)
    uint8_t ntt_choice[2][kNttBuckets];       // [forward, inverse][limb bucket] -> variant
    uint32_t log_n = 0, n = 0, n_q = 0, n_p = 0, L = 0, K = 0, alpha = 0;
    double default_scale = 0, sigma = 0;
    std::vector<uint64_t> primes;          // n_q + n_p
    std::vector<uint64_t> psi;             // primitive 2N-th roots used by the tables
    std::vector<uint64_t> cdt;             // CDT thresholds
    cudaStream_t stream = nullptr;         // default stream of the context
    cudaMemPool_t pool = nullptr;
    hear::DevBuf d_primes;                 // DevPrime[n_q+n_p]
    hear::DevBuf d_tw;                     // [4][n_q+n_p][N]: fwd, fwd_sh, inv, inv_sh
    hear::DevBuf d_cdt;                    // CDT on device
    std::vector<std::unique_ptr<hear::LevelConsts>> levels;  // per level 0..L
    bool poisoned = false;
    mutable hear::Profiler prof;
    // device tables of key-switching jobs (key pointers, galois elements), keyed by content;
    // built outside stream capture and reused, so a captured evaluation uploads nothing
    mutable std::mutex tab_mu;
    mutable std::map<std::vector<uint64_t>, hear::DevBuf> job_tables;
    const hear::DevPrime *dev_primes() const { return static_cast<const hear::DevPrime *>(d_primes.p); }
    uint32_t nqp() const { return n_q + n_p; }
    uint32_t dnum(uint32_t level) const { return (level + 1 + alpha - 1) / alpha; }
    uint32_t dnum_max() const { return dnum(L); }
};

struct hear_secret_key {
    hear_context *ctx = nullptr;
    std::vector<int8_t> s;         // ternary coefficients
    hear::DevBuf s_mont;           // s in NTT + Montgomery form over all n_q+n_p primes
};

struct hear_public_key {
    hear_context *ctx = nullptr;
    hear::DevBuf pk_mont;          // [2][n_q][N] NTT + Montgomery form
};

struct hear_eval_keys {
    hear_context *ctx = nullptr;
    uint64_t serial = 0;           // unique per key set (graph plans are keyed by it)
    // galois element -> [dnum_max][2][n_q+n_p][N] NTT + Montgomery form; 1 = relin
    std::map<uint32_t, hear::DevBuf> keys;
    const uint64_t *key(uint32_t g) const {
        auto it = keys.find(g);
        return it == keys.end() ? nullptr : it->second.u64();
    }
};

struct hear_ciphertext {
    hear_context *ctx = nullptr;
    uint32_t level = 0, n_poly = 2;
    double scale = 1.0;
    hear::DevBuf d;                // [n_poly][level+1][N], NTT domain
};

namespace hear {

// ------------------------------------------------------------------ kernels (launchers)
// Limb maps: limb b of a launch lives in group g = b / per_group at position
// t = b % per_group, address data + g * group_stride + t * N, and has the prime
// q_base + t if t < q_count, else the special prime n_q + (t - q_count).
struct LimbMap {
    uint32_t per_group = 1;
    uint32_t q_base = 0;
    uint32_t q_count = 1;
    uint32_t n_q = 0;
    uint64_t group_stride = 0;   // words; 0 = per_group * N
    uint32_t skip_dnum = 0;      // if nonzero: group g is digit j = g % skip_dnum and limbs
    uint32_t alpha = 0;          //   t in [j*alpha, (j+1)*alpha) with t < q_count are skipped
    __host__ __device__ inline bool resolve(uint32_t b, uint32_t *prime) const {
        uint32_t t = b % per_group;
        if (skip_dnum) {
            uint32_t j = (b / per_group) % skip_dnum;
            if (t >= j * alpha && t < (j + 1) * alpha && t < q_count) return false;
        }
        *prime = t < q_count ? q_base + t : n_q + (t - q_count);
        return true;
    }
    __host__ __device__ inline uint64_t offset(uint32_t b, uint32_t n) const {
        uint32_t g = b / per_group, t = b % per_group;
        uint64_t gs = group_stride ? group_stride : (uint64_t)per_group * n;
        return g * gs + (uint64_t)t * n;
    }
};

// limbs of polynomials at level l (groups of l+1 limbs q_0..q_l)
inline LimbMap map_q(uint32_t level, uint32_t n_q) {
    LimbMap m; m.per_group = level + 1; m.q_count = level + 1; m.n_q = n_q; return m;
}
// limbs of polynomials over Q_l u P (groups of l+1+K limbs)
inline LimbMap map_qp(uint32_t level, uint32_t n_q, uint32_t K) {
    LimbMap m; m.per_group = level + 1 + K; m.q_count = level + 1; m.n_q = n_q; return m;
}

void ntt_forward(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, cudaStream_t s);
void ntt_inverse(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, cudaStream_t s);
// forward NTT whose input limb b (group g = b / per_group) is read from pro + g * pro_gstride
// (coefficient domain) and reduced mod limb b's prime (an extension by one source limb),
// centred mod pro_center first when that is nonzero; pro = null: ntt_forward
void ntt_forward_pro(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, const uint64_t *pro,
                     uint64_t pro_gstride, cudaStream_t s, uint64_t pro_center = 0);
// inverse NTT from src (limb b of group g at src + g * src_gstride + b' * N) into data (the
// layout of `map`, contiguous groups); src is left unchanged.  src_count > 1: the transform of
// the sum mod q of src_count sources, source r at src + r * src_cstride
void ntt_inverse_from(const hear_context *ctx, const uint64_t *src, uint64_t src_gstride, uint64_t *data,
                      uint32_t n_limbs, LimbMap map, cudaStream_t s, uint32_t src_count = 1,
                      uint64_t src_cstride = 0);
// butterflies per second of the transforms' register-resident arithmetic (forward or
// inverse) over the context's prime mix, iters rounds of four radix-16 stages per thread
double bfly_peak(const hear_context *ctx, bool fwd, uint32_t iters);
// fill ctx->ntt_choice by timing the launch variants (ms_out: [2][kNttBuckets][3] or null)
// ms_out: [2][kNttBuckets][kNttVariants] or null
void ntt_tune(hear_context *ctx, uint32_t max_limbs, int iters, float *ms_out);

// RAII bracket of one or more kernel launches for the profiler
struct ProfScope {
    const hear_context *c;
    const char *name;
    cudaStream_t s;
    double bytes;
    uint32_t launches;
    cudaEvent_t a = nullptr;
    ProfScope(const hear_context *ctx, const char *nm, cudaStream_t st, double algo_bytes, uint32_t n_launch = 1);
    ~ProfScope();
};

// The other launchers are declared in kernels.cuh.
}  // namespace hear
