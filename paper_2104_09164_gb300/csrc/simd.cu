// simd.cu -- slot-batched evaluation of the FC / x^2 networks on sm_103a.
//
// One clip per slot and one ciphertext per feature: an FC layer y_o = sum_i [w_oi] x_i
// multiplies the d_in input ciphertexts by plaintext scalars (the constant polynomial
// round(w q_l), i.e. the encoding of the constant slot vector w at scale q_l; Methods,
// "Non-convolutional layers", with every slot a different clip) and needs no rotation.  Per
// limb t this is a product of an M x K matrix of residues with a K x 2N matrix of residues,
// done here as a modular matrix product on the integer multiply-add pipe (the exact
// arithmetic rules the tensor cores out).  Each residue is cut into two pieces and the three
// partial products of Karatsuba's identity a0 b1 + a1 b0 = (a0 + a1)(b0 + b1) - a0 b0 - a1 b1
// are summed over K and reduced mod q_t once per output:
//  * primes below 2^42: 21-bit pieces, every partial product one 32 x 32 -> 64-bit
//    multiply-add (mad.wide.u32) into a 64-bit sum (K <= 2^19 products of < 2^44);
//  * primes below 2^62: 31-bit pieces, every partial product a multiply-low / multiply-high
//    pair added into a 96-bit sum by one carry chain.
// Both forms hold the multiply pipe the same number of cycles per partial product.
#include <cmath>
#include "simd.h"
#include "modarith.cuh"
#include "launch.cuh"

namespace hear {
namespace {

constexpr int kGemmThreads = 256;
constexpr uint32_t kMaxK = 1u << 19;     // K * 2^44 < 2^63
constexpr uint32_t kMpadUnit = 64;

// KIND 0: 21-bit pieces (q < 2^42), 64-bit sums; KIND 1: 31-bit pieces (q < 2^62), 96-bit
// sums.  Planes of pieces: a0, a1, a0 + a1.  A CTA tile of TM rows x TX columns (residues of
// one limb), RM rows x CM columns per thread (16 x 16 threads), KC inner indices per
// shared-memory round, MINB resident CTAs per SM.
template <int KIND> struct Gemm;
template <> struct Gemm<0> {
    static constexpr int BITS = 21, TM = 64, TX = 64, RM = 4, CM = 4, KC = 32, MINB = 2;
};
template <> struct Gemm<1> {
    static constexpr int BITS = 31, TM = 32, TX = 32, RM = 2, CM = 2, KC = 32, MINB = 2;
};
constexpr int kPlanes = 3;

struct LimbSet {
    uint32_t n;
    uint8_t t[kMaxPrimes];
};

// per limb: c[0] = 2^BITS, c[1] = 2^(2 BITS), c[2] = 2^64 mod q_t and their Shoup companions
struct PieceConsts {
    uint64_t c[4], c_sh[4];
};

// V consecutive words of shared memory (V = 2 or 4; 4V-byte aligned) into registers
template <int V>
__device__ __forceinline__ void load_vec(const uint32_t *s, uint32_t *r) {
    if constexpr (V == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(s);
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(s);
        r[0] = v.x;
        r[1] = v.y;
    }
}

template <int KIND>
__device__ __forceinline__ void split_pieces(uint64_t v, uint32_t *p) {
    constexpr int B = Gemm<KIND>::BITS;
    const uint32_t b0 = (uint32_t)v & ((1u << B) - 1), b1 = (uint32_t)(v >> B);
    p[0] = b0;
    p[1] = b1;
    p[2] = b0 + b1;
}

// (x2 x1 x0) += a * b: one carry chain of a multiply-low, a multiply-high and a carry add
__device__ __forceinline__ void mac96(uint32_t a, uint32_t b, uint32_t &x0, uint32_t &x1, uint32_t &x2) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(x0), "+r"(x1), "+r"(x2)
        : "r"(a), "r"(b));
}

// a 96-bit sum (x2 x1 x0) mod q
__device__ __forceinline__ uint64_t reduce96(uint32_t x0, uint32_t x1, uint32_t x2, const DevPrime &pr,
                                             const PieceConsts &k) {
    const uint64_t lo = ((uint64_t)x1 << 32) | x0;
    return add_mod(shoup(lo, 1, pr.one_sh, pr.q), shoup(x2, k.c[2], k.c_sh[2], pr.q), pr.q);
}

// the reduction of a thread's RM x CM sums mod q_t and their store
template <int KIND>
__device__ __forceinline__ void store_outputs(const uint64_t (&acc)[Gemm<KIND>::RM][Gemm<KIND>::CM][KIND == 0 ? kPlanes : 1],
                                              const uint32_t (&acw)[Gemm<KIND>::RM][Gemm<KIND>::CM][KIND == 1 ? 3 * kPlanes : 1],
                                              uint64_t *__restrict__ y, const DevPrime *__restrict__ P,
                                              const PieceConsts *__restrict__ pc, uint32_t t, uint32_t m0, uint32_t M,
                                              uint32_t poly, uint32_t L1, uint32_t n, uint32_t j0, uint32_t tx,
                                              uint32_t ty) {
    using G = Gemm<KIND>;
    constexpr int RM = G::RM, CM = G::CM;
    const DevPrime pr = P[t];
    const PieceConsts k = pc[t];
    const uint64_t q = pr.q;
#pragma unroll
    for (int r = 0; r < RM; r++) {
        const uint32_t m = m0 + ty * RM + r;
        if (m >= M) continue;
        uint64_t o[CM];
#pragma unroll
        for (int c = 0; c < CM; c++) {
            uint64_t v;
            if constexpr (KIND == 0) {   // s00 + (sm - s00 - s11) 2^21 + s11 2^42
                const uint64_t *s = acc[r][c];
                const uint64_t cross = s[2] - s[0] - s[1];
                v = add_mod(shoup(s[0], 1, pr.one_sh, q), shoup(cross, k.c[0], k.c_sh[0], q), q);
                v = add_mod(v, shoup(s[1], k.c[1], k.c_sh[1], q), q);
            } else {                     // the same with 96-bit sums and 2^31, 2^62
                const uint32_t *w = acw[r][c];
                uint32_t c0, c1, c2;     // cross = sm - s00 - s11 (never negative)
                asm("sub.cc.u32 %0, %3, %6;\n\t"
                    "subc.cc.u32 %1, %4, %7;\n\t"
                    "subc.u32 %2, %5, %8;"
                    : "=r"(c0), "=r"(c1), "=r"(c2)
                    : "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[0]), "r"(w[1]), "r"(w[2]));
                asm("sub.cc.u32 %0, %0, %3;\n\t"
                    "subc.cc.u32 %1, %1, %4;\n\t"
                    "subc.u32 %2, %2, %5;"
                    : "+r"(c0), "+r"(c1), "+r"(c2)
                    : "r"(w[3]), "r"(w[4]), "r"(w[5]));
                v = add_mod(reduce96(w[0], w[1], w[2], pr, k),
                            shoup(reduce96(c0, c1, c2, pr, k), k.c[0], k.c_sh[0], q), q);
                v = add_mod(v, shoup(reduce96(w[3], w[4], w[5], pr, k), k.c[1], k.c_sh[1], q), q);
            }
            o[c] = v;
        }
        ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(y + (((uint64_t)m * 2 + poly) * L1 + t) * n + j0 + tx * CM);
#pragma unroll
        for (int c = 0; c < CM; c += 2) dst[c / 2] = make_ulonglong2(o[c], o[c + 1]);
    }
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// y[m][poly][t][j] = sum_k A_t[m][k] x[k][poly][t][j] mod q_t for the limbs of `limbs`
// (blockIdx.y), rows m0 = blockIdx.z * TM .., columns (poly, j) = blockIdx.x * TX ..
// The global loads run one round ahead: while round k0 (KC inner indices) is computed from
// one pair of piece buffers, cp.async brings round k0 + KC's scalar pieces into the other
// scalar buffer and its raw residues into a staging buffer; after the round the staged
// residues are cut into the other residue-piece buffer.  Dynamic shared memory: 2 x 3 KC TM
// + 2 x 3 KC TX pieces (32-bit) + KC TX residues (64-bit).
template <int KIND>
__global__ void __launch_bounds__(kGemmThreads, Gemm<KIND>::MINB)
k_simd_fc(const uint64_t *__restrict__ x, uint64_t *__restrict__ y, const uint32_t *__restrict__ a,
               const uint64_t *__restrict__ a_off, const PieceConsts *__restrict__ pc, LimbSet limbs, uint32_t M,
               uint32_t Mpad, uint32_t K, uint32_t L1, uint32_t n, const DevPrime *__restrict__ P) {
    using G = Gemm<KIND>;
    constexpr int PL = kPlanes, TM = G::TM, TX = G::TX, RM = G::RM, CM = G::CM, KC = G::KC;
    constexpr int SA = PL * KC * TM, SB = PL * KC * TX;
    static_assert(TM == 16 * RM && TX == 16 * CM, "16 x 16 threads");
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *const sa_base = reinterpret_cast<uint32_t *>(smem);               // [2][PL][KC][TM]
    uint32_t *const sb_base = sa_base + 2 * SA;                                 // [2][PL][KC][TX]
    uint64_t *const sraw = reinterpret_cast<uint64_t *>(sb_base + 2 * SB);      // [KC][TX]
    pdl_enter();
    const uint32_t t = limbs.t[blockIdx.y];
    const uint32_t m0 = blockIdx.z * TM;
    const uint32_t col0 = blockIdx.x * TX;
    const uint32_t poly = col0 / n, j0 = col0 % n;
    const uint32_t tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const uint64_t xrow = 2ull * L1 * n;
    const uint64_t *xb = x + ((uint64_t)poly * L1 + t) * n + j0;
    const uint32_t *ab = a + a_off[t] + m0;

    // round k0: scalar pieces into scalar buffer b, raw residues into the staging buffer
    auto issue = [&](uint32_t k0, int b) {
        uint32_t *sa = sa_base + b * SA;
#pragma unroll 1
        for (int i = threadIdx.x; i < PL * KC * TM / 4; i += kGemmThreads) {
            const int p = i / (KC * TM / 4), rem = i % (KC * TM / 4);
            const int r = rem / (TM / 4), c4 = rem % (TM / 4);
            const bool ok = k0 + r < K;
            cp_async16(sa + (p * KC + r) * TM + c4 * 4, ok ? ab + ((uint64_t)p * K + k0 + r) * Mpad + c4 * 4 : ab,
                       ok ? 16u : 0u);
        }
#pragma unroll 1
        for (int i = threadIdx.x; i < KC * TX / 2; i += kGemmThreads) {
            const int r = i / (TX / 2), c2 = i % (TX / 2);
            const bool ok = k0 + r < K;
            cp_async16(sraw + r * TX + 2 * c2, ok ? xb + (uint64_t)(k0 + r) * xrow + 2 * c2 : xb, ok ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // the staged residues cut into residue-piece buffer b (each thread its own residues)
    auto cut = [&](int b) {
        uint32_t *sb = sb_base + b * SB;
#pragma unroll 1
        for (int i = threadIdx.x; i < KC * TX; i += kGemmThreads) {
            uint32_t pcs[PL];
            split_pieces<KIND>(sraw[i], pcs);
#pragma unroll
            for (int p = 0; p < PL; p++) sb[p * KC * TX + i] = pcs[p];
        }
    };

    uint64_t acc[RM][CM][KIND == 0 ? PL : 1];
    uint32_t acw[RM][CM][KIND == 1 ? 3 * PL : 1];
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
        for (int c = 0; c < CM; c++) {
#pragma unroll
            for (int p = 0; p < (KIND == 0 ? PL : 1); p++) acc[r][c][p] = 0;
#pragma unroll
            for (int p = 0; p < (KIND == 1 ? 3 * PL : 1); p++) acw[r][c][p] = 0;
        }

    issue(0, 0);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    cut(0);
    int b = 0;
    for (uint32_t k0 = 0; k0 < K; k0 += KC, b ^= 1) {
        __syncthreads();                                  // buffers b are complete, sraw is free
        const bool more = k0 + KC < K;
        if (more) issue(k0 + KC, b ^ 1);
        const uint32_t *sa = sa_base + b * SA;
        const uint32_t *sb = sb_base + b * SB;
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
            uint32_t av[PL][RM], bv[PL][CM];
#pragma unroll
            for (int p = 0; p < PL; p++) {
                load_vec<CM>(&sb[(p * KC + kk) * TX + tx * CM], bv[p]);
                load_vec<RM>(&sa[(p * KC + kk) * TM + ty * RM], av[p]);
            }
#pragma unroll
            for (int r = 0; r < RM; r++)
#pragma unroll
                for (int c = 0; c < CM; c++)
#pragma unroll
                    for (int p = 0; p < PL; p++) {
                        if constexpr (KIND == 0)
                            acc[r][c][p] += (uint64_t)av[p][r] * bv[p][c];
                        else
                            mac96(av[p][r], bv[p][c], acw[r][c][3 * p], acw[r][c][3 * p + 1], acw[r][c][3 * p + 2]);
                    }
        }
        if (more) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");   // round k0 + KC has landed
            __syncthreads();                                       // ... for every thread's copies
            cut(b ^ 1);
        }
    }
    store_outputs<KIND>(acc, acw, y, P, pc, t, m0, M, poly, L1, n, j0, tx, ty);
}
// dynamic shared memory of k_simd_fc (112 KB for KIND 0, 56 KB for KIND 1)
template <int KIND> constexpr size_t gemm_smem() {
    return 2ull * kPlanes * Gemm<KIND>::KC * (Gemm<KIND>::TM + Gemm<KIND>::TX) * 4 +
           8ull * Gemm<KIND>::KC * Gemm<KIND>::TX;
}

// Throughput of the integer multiply-add forms on this GPU: every thread runs 8 independent
// chains of `iters` multiply-adds (kind 0: mad.wide.u32, 32 x 32 -> 64 bits plus a 64-bit
// addend, the GEMM's step; kind 1: mad.lo.u32).  Each step multiplies a word of the next
// chain's accumulator, so no product is loop-invariant and no operand overlaps its own
// destination; one word per thread keeps the chains live.
template <int KIND>
__global__ void __launch_bounds__(256) k_imad_peak(uint32_t seed, uint32_t iters, uint64_t *out) {
    pdl_enter();
    uint64_t acc[8];
    uint32_t acc32[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        acc[i] = seed + threadIdx.x * 8 + i;
        acc32[i] = (uint32_t)acc[i];
    }
    const uint32_t b = (seed ^ (blockIdx.x * 2654435761u)) | 1u;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if constexpr (KIND == 0)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;"
                             : "+l"(acc[i])
                             : "r"((uint32_t)(acc[(i + 1) & 7] >> 32)), "r"(b));
            else
                asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(acc32[i]) : "r"(acc32[(i + 1) & 7]), "r"(b));
        }
    }
    uint64_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) x ^= acc[i] ^ acc32[i];
    out[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

uint64_t pow2_mod(uint32_t e, uint64_t q) {
    unsigned __int128 r = 1;
    for (uint32_t i = 0; i < e; i++) r = (r * 2) % q;
    return (uint64_t)r;
}
uint64_t shoup_companion(uint64_t w, uint64_t q) { return (uint64_t)(((unsigned __int128)w << 64) / q); }

// residue kind of a prime: 0 = 21-bit pieces (q < 2^42), 1 = 31-bit pieces (q < 2^62)
int kind_of(uint64_t q) {
    HEAR_REQUIRE(q < (1ull << 62), HEAR_E_UNSUPPORTED, "prime above 2^62");
    return q < (1ull << 42) ? 0 : 1;
}

// the scalars of an M x K weight matrix (row-major, rows beyond M zero) at scale q_level,
// cut into pieces per limb t <= level: planes a0, a1, a0 + a1, each [K][Mpad]
void build_matrix(hear_context *c, hear_simd_model::Layer &L, const std::vector<double> &W, uint32_t level,
                  cudaStream_t st) {
    const uint32_t L1 = level + 1, M = L.M, K = L.K;
    L.Mpad = (M + kMpadUnit - 1) / kMpadUnit * kMpadUnit;
    const uint64_t ql = c->primes[level];
    std::vector<int64_t> sc((size_t)M * K);
    for (size_t i = 0; i < sc.size(); i++) sc[i] = round_scalar(W[i], ql);
    const uint64_t per_limb = (uint64_t)kPlanes * K * L.Mpad;
    std::vector<uint64_t> off(L1);
    for (uint32_t t = 0; t < L1; t++) {
        off[t] = t * per_limb;
        (kind_of(c->primes[t]) == 0 ? L.limbs_narrow : L.limbs_wide).push_back((uint8_t)t);
    }
    std::vector<uint32_t> A(L1 * per_limb, 0u);
    std::vector<PieceConsts> pcs(L1);
    for (uint32_t t = 0; t < L1; t++) {
        const uint64_t q = c->primes[t];
        const uint32_t bits = kind_of(q) == 0 ? Gemm<0>::BITS : Gemm<1>::BITS;
        uint32_t *base = A.data() + off[t];
        for (uint32_t m = 0; m < M; m++)
            for (uint32_t k = 0; k < K; k++) {
                const int64_t s = sc[(size_t)m * K + k];
                const uint64_t r = s >= 0 ? (uint64_t)s % q : (q - (uint64_t)(-(s + 1)) % q - 1) % q;
                const uint32_t a0 = (uint32_t)(r & ((1ull << bits) - 1)), a1 = (uint32_t)(r >> bits);
                const uint32_t pv[kPlanes] = {a0, a1, a0 + a1};
                for (int p = 0; p < kPlanes; p++) base[((uint64_t)p * K + k) * L.Mpad + m] = pv[p];
            }
        const uint32_t e[4] = {bits, 2 * bits, 64, 0};
        for (int i = 0; i < 4; i++) {
            pcs[t].c[i] = pow2_mod(e[i], q);
            pcs[t].c_sh[i] = shoup_companion(pcs[t].c[i], q);
        }
    }
    L.a = DevBuf(A.size() * 4, st);
    L.a_off = DevBuf(L1 * 8, st);
    L.consts = DevBuf(L1 * sizeof(PieceConsts), st);
    HEAR_CHECK_CUDA(cudaMemcpyAsync(L.a.p, A.data(), A.size() * 4, cudaMemcpyHostToDevice, st));
    HEAR_CHECK_CUDA(cudaMemcpyAsync(L.a_off.p, off.data(), L1 * 8, cudaMemcpyHostToDevice, st));
    HEAR_CHECK_CUDA(cudaMemcpyAsync(L.consts.p, pcs.data(), L1 * sizeof(PieceConsts), cudaMemcpyHostToDevice, st));
    HEAR_CHECK_CUDA(cudaStreamSynchronize(st));
}

template <int KIND>
void launch_gemm(const hear_context *c, const hear_simd_model::Layer &L, const std::vector<uint8_t> &limbs,
                 uint32_t L1, const uint64_t *x, uint64_t *y, cudaStream_t st) {
    if (limbs.empty()) return;
    LimbSet s{};
    s.n = (uint32_t)limbs.size();
    for (uint32_t i = 0; i < s.n; i++) s.t[i] = limbs[i];
    launch(k_simd_fc<KIND>, dim3(2 * c->n / Gemm<KIND>::TX, s.n, L.Mpad / Gemm<KIND>::TM), kGemmThreads,
           gemm_smem<KIND>(), st, x, y, static_cast<const uint32_t *>(L.a.p), static_cast<const uint64_t *>(L.a_off.p),
           static_cast<const PieceConsts *>(L.consts.p), s, L.M, L.Mpad, L.K, L1, c->n, c->dev_primes());
}

// Y [M][2][l+1][N] = scalars (.) X [K][2][l+1][N]
void gemm(const hear_context *c, const hear_simd_model::Layer &L, uint32_t level, const uint64_t *x, uint64_t *y,
          cudaStream_t st) {
    const uint32_t L1 = level + 1;
    const double bytes = 8.0 * (double)c->n * 2 * L1 * (L.K + L.M);
    ProfScope ps(c, "k_simd_fc", st, bytes, (L.limbs_narrow.empty() ? 0 : 1) + (L.limbs_wide.empty() ? 0 : 1));
    launch_gemm<0>(c, L, L.limbs_narrow, L1, x, y, st);
    launch_gemm<1>(c, L, L.limbs_wide, L1, x, y, st);
}

}  // namespace

double imad_peak(hear_context *c, int kind, uint32_t iters) {
    HEAR_REQUIRE(kind == 0 || kind == 1, HEAR_E_INVAL, "kind must be 0 (mad.wide.u32) or 1 (mad.lo.u32)");
    HEAR_REQUIRE(iters >= 1 && iters <= (1u << 20), HEAR_E_INVAL, "iters must be in [1, 2^20]");
    int sms = 0;
    HEAR_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const uint32_t blocks = (uint32_t)sms * 8, threads = 256;
    cudaStream_t st = c->stream;
    DevBuf out((size_t)blocks * threads * 8, st);
    auto run = [&](uint32_t it) {
        if (kind == 0) launch(k_imad_peak<0>, blocks, threads, 0, st, 12345u, it, out.u64());
        else launch(k_imad_peak<1>, blocks, threads, 0, st, 12345u, it, out.u64());
    };
    run(iters);   // warm-up
    cudaEvent_t e0, e1;
    HEAR_CHECK_CUDA(cudaEventCreate(&e0));
    HEAR_CHECK_CUDA(cudaEventCreate(&e1));
    HEAR_CHECK_CUDA(cudaEventRecord(e0, st));
    run(iters);
    HEAR_CHECK_CUDA(cudaEventRecord(e1, st));
    HEAR_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)blocks * threads * 8.0 * iters / (ms / 1e3);
}

int64_t round_scalar(double w, uint64_t q) {
    HEAR_REQUIRE(std::isfinite(w), HEAR_E_INVAL, "weight is not finite");
    if (w == 0.0) return 0;
    int e = 0;
    const double fr = std::frexp(std::fabs(w), &e);            // |w| = fr 2^e, fr in [1/2, 1)
    const uint64_t mant = (uint64_t)std::ldexp(fr, 53);        // |w| = mant 2^(e - 53), exact
    const int sh = e - 53;
    const unsigned __int128 pq = (unsigned __int128)mant * q;  // < 2^114
    unsigned __int128 r;
    HEAR_REQUIRE(sh < 0, HEAR_E_INVAL, "weight too large for the scale");   // |w| >= 2^53
    if (-sh > 115) {
        r = 0;                                                  // |w q| < 1/4
    } else {
        r = (pq + ((unsigned __int128)1 << (-sh - 1))) >> (-sh);   // half away from zero
    }
    HEAR_REQUIRE((r >> 62) == 0, HEAR_E_INVAL, "weight too large for the scale");
    return w < 0 ? -(int64_t)r : (int64_t)r;
}

void simd_setup() {
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_simd_fc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem<0>()));
    HEAR_CHECK_CUDA(cudaFuncSetAttribute(k_simd_fc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem<1>()));
}

hear_simd_model *simd_model_create(hear_context *c, const hear_layer_desc *layers, size_t n_layers,
                                   uint32_t level) {
    HEAR_REQUIRE(layers && n_layers > 0, HEAR_E_INVAL, "no layers");
    HEAR_REQUIRE(level >= 1 && level <= c->L, HEAR_E_LEVEL, "start level outside [1, L]");
    auto m = std::make_unique<hear_simd_model>();
    m->ctx = c;
    m->level_in = level;
    cudaStream_t st = c->stream;
    uint32_t dim = 0;
    for (size_t li = 0; li < n_layers; li++) {
        const hear_layer_desc &d = layers[li];
        hear_simd_model::Layer L;
        L.kind = d.kind;
        L.level_in = level;
        if (li == 0) {
            HEAR_REQUIRE(d.kind != HEAR_LAYER_SQUARE, HEAR_E_INVAL, "the first layer must be linear");
            dim = d.d_in;
            m->d_in = dim;
        }
        L.n_in = dim;
        if (d.kind == HEAR_LAYER_FC || d.kind == HEAR_LAYER_FC_SQ_FC) {
            HEAR_REQUIRE(d.w && d.d_in == dim && d.d_out >= 1, HEAR_E_INVAL, "FC input dimension mismatch");
            HEAR_REQUIRE(!d.bias, HEAR_E_UNSUPPORTED, "bias is not supported");
            HEAR_REQUIRE(d.d_in >= 1 && d.d_in <= kMaxK, HEAR_E_UNSUPPORTED, "FC input dimension above 2^19");
        }
        if (d.kind == HEAR_LAYER_FC) {
            HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
            L.M = d.d_out;
            L.K = d.d_in;
            std::vector<double> W(d.w, d.w + (size_t)d.d_out * d.d_in);
            build_matrix(c, L, W, level, st);
            level -= 1;
            dim = d.d_out;
        } else if (d.kind == HEAR_LAYER_SQUARE) {
            HEAR_REQUIRE(level >= 1, HEAR_E_LEVEL, "not enough levels for the network");
            level -= 1;
        } else if (d.kind == HEAR_LAYER_FC_SQ_FC) {
            HEAR_REQUIRE(d.w2 && d.d_out2 >= 1, HEAR_E_INVAL, "FC_SQ_FC needs its second matrix");
            HEAR_REQUIRE(level >= 2, HEAR_E_LEVEL, "not enough levels for the network");
            const uint32_t d1 = d.d_out, d2 = d.d_out2, K = d.d_in;
            L.d1 = d1;
            L.d2 = d2;
            L.M = 2 * d1 * d2;
            L.K = K;
            std::vector<double> W((size_t)L.M * K);
            for (uint32_t r = 0; r < d1; r++)
                for (uint32_t cc = 0; cc < d2; cc++)
                    for (uint32_t i = 0; i < K; i++) {
                        const double w1 = d.w[(size_t)r * K + i];
                        W[((size_t)r * d2 + cc) * K + i] = w1;
                        W[((size_t)d1 * d2 + r * d2 + cc) * K + i] = d.w2[(size_t)cc * d1 + r] * w1;
                    }
            build_matrix(c, L, W, level, st);
            level -= 2;
            dim = d2;
        } else {
            throw Error(HEAR_E_INVAL, "unknown layer kind");
        }
        L.n_out = dim;
        L.level_out = level;
        m->layers.push_back(std::move(L));
    }
    m->d_out = dim;
    m->level_out = level;
    return m.release();
}

DevBuf simd_evaluate(const hear_simd_model *m, const hear_eval_keys *evk, const uint64_t *x, double scale_in,
                     double *scale_out, cudaStream_t st) {
    hear_context *c = m->ctx;
    const uint32_t n = c->n;
    DevBuf cur;
    const uint64_t *xin = x;
    double scale = scale_in;
    for (const hear_simd_model::Layer &L : m->layers) {
        const uint32_t level = L.level_in;
        const uint64_t plane = (uint64_t)(level + 1) * n, plane1 = (uint64_t)level * n;
        DevBuf next;
        if (L.kind == HEAR_LAYER_FC) {
            DevBuf Y((size_t)L.M * 2 * plane * 8, st), tmp((size_t)L.M * 2 * plane1 * 8, st);
            gemm(c, L, level, xin, Y.u64(), st);
            next = DevBuf((size_t)L.M * 2 * plane1 * 8, st);
            rescale(c, level, 2 * L.M, Y.u64(), next.u64(), tmp.u64(), st);
            const double ql = (double)c->primes[level];
            scale = scale * ql / ql;
        } else if (L.kind == HEAR_LAYER_SQUARE) {
            const uint64_t *rk = evk->key(1);
            HEAR_REQUIRE(rk, HEAR_E_NOKEY, "missing relinearisation key");
            DevBuf prod((size_t)L.n_in * 2 * plane * 8, st), tmp((size_t)L.n_in * 2 * plane1 * 8, st);
            mul_relin(c, level, L.n_in, xin, xin, rk, prod.u64(), st);
            next = DevBuf((size_t)L.n_in * 2 * plane1 * 8, st);
            rescale(c, level, 2 * L.n_in, prod.u64(), next.u64(), tmp.u64(), st);
            scale = scale * scale / (double)c->primes[level];
        } else {
            // y_r and u_(c,r) one level down, then sum_r y_r u_(c,r) as degree-2
            // ciphertexts, one relinearisation and one rescale per output
            const uint64_t *rk = evk->key(1);
            HEAR_REQUIRE(rk, HEAR_E_NOKEY, "missing relinearisation key");
            const uint32_t P2 = L.d1 * L.d2, lv = level - 1;
            const uint64_t p1 = plane1, p2 = (uint64_t)lv * n;
            DevBuf Y((size_t)L.M * 2 * plane * 8, st), Z((size_t)L.M * 2 * p1 * 8, st),
                tmp((size_t)L.M * 2 * p1 * 8, st);
            gemm(c, L, level, xin, Y.u64(), st);
            rescale(c, level, 2 * L.M, Y.u64(), Z.u64(), tmp.u64(), st);
            const double ql = (double)c->primes[level];
            const double s1 = scale * ql / ql;
            DevBuf T((size_t)P2 * 3 * p1 * 8, st), S((size_t)L.d2 * 3 * p1 * 8, st);
            tensor_ct(c, lv, P2, Z.u64(), Z.u64() + (uint64_t)P2 * 2 * p1, T.u64(), st);
            // T is ordered (r, c): sum over r = stride d2 degree-2 ciphertexts
            sum_ct(c, lv, 3 * L.d2, T.u64(), (uint64_t)L.d2 * 3 * p1, L.d1, S.u64(), st);
            DevBuf R((size_t)L.d2 * 2 * p1 * 8, st), tmp2((size_t)L.d2 * 2 * p2 * 8, st);
            relin3(c, lv, L.d2, S.u64(), rk, R.u64(), st);
            next = DevBuf((size_t)L.d2 * 2 * p2 * 8, st);
            rescale(c, lv, 2 * L.d2, R.u64(), next.u64(), tmp2.u64(), st);
            scale = s1 * s1 / (double)c->primes[lv];
        }
        cur = std::move(next);
        xin = cur.u64();
    }
    *scale_out = scale;
    return cur;
}

}  // namespace hear
