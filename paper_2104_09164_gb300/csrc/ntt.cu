// ntt.cu -- batched negacyclic NTT / inverse NTT over word-size primes on sm_103a.
//
// Forward: Cooley-Tukey, natural-order input, bit-reversed output, twiddle table
// fwd[k] = psi^brv(k) (psi a primitive 2N-th root); output index i holds the evaluation
// a(psi^(2 brv(i) + 1)).  Inverse: Gentleman-Sande with inv[k] = psi^-brv(k), bit-reversed
// input, natural output, times N^-1.  The NTT of the input ciphertext limbs is the
// "NTT conversion" the paper shares across rotations by hoisting (Methods, "Algorithmic
// and cryptographic optimizations", item (i)).
//
// Layout: N = 2^a * 2^b.  Pass A runs stages 0..a-1 on strided sub-problems (column c:
// elements c + u*2^b, u < 2^a), pass B runs stages a..logN-1 on contiguous blocks of 2^b.
// A CTA stages a 2048- or 4096-word tile in shared memory (XOR-swizzled, bank-conflict
// free); each pass runs in two register rounds, each thread applying three or four stages
// at a time to 8 or 16 words (radix-2^3 / 2^4 units), with Harvey lazy butterflies
// (values kept in [0, 4q) forward and [0, 2q) inverse) and Shoup products by the
// precomputed twiddle companions.
#include "internal.h"
#include "modarith.cuh"

namespace hear {
namespace {

constexpr int kThreads = 256;

struct PassArgs {
    uint64_t small_below;    // primes below this skip the per-stage corrections
    uint64_t *data;
    uint32_t n_limbs;
    uint32_t log_n;
    LimbMap map;
    const DevPrime *primes;
    const uint64_t *tw;      // twiddle table [n_primes][N]
    const uint64_t *tw_sh;   // Shoup companions
    uint32_t n;              // N
};

// Shared-memory word of logical tile index i: the low four bits are XORed with bits 3..6 and
// 4..7, which makes every unit access pattern below bank-conflict free (two wavefronts per
// warp-wide 64-bit access) and keeps each 16-word block in place.
__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ ((i >> 3) & 15u) ^ ((i >> 4) & 15u); }

// Stage split of a pass of LOGR stages into register units of 2^W0 and 2^W1 words, and the
// tile (words per CTA) of the wide variant; the narrow variant (for launches with too few
// CTAs to fill the GPU) uses a quarter of the tile with a quarter of the threads.
template <int LOGR> struct Split;
template <> struct Split<5> { static constexpr int W0 = 3, W1 = 2, TILE = 2048; };
template <> struct Split<6> { static constexpr int W0 = 3, W1 = 3, TILE = 2048; };
template <> struct Split<7> { static constexpr int W0 = 4, W1 = 3, TILE = 4096; };
template <> struct Split<8> { static constexpr int W0 = 4, W1 = 4, TILE = 4096; };
template <int LOGR, bool NARROW> struct Tile {
    static constexpr int WORDS = NARROW ? Split<LOGR>::TILE / 4 : Split<LOGR>::TILE;
    static constexpr int THREADS = NARROW ? kThreads / 4 : kThreads;
};

// One group of W stages on a tile: forward stages LS0, LS0+1, ..; inverse LS0, LS0-1, ...
// Each thread holds the 2^W words of a unit in registers.  In the stage i of the group the
// unit's butterflies use only 2^i (forward) or 2^(W-1-i) (inverse) distinct twiddles, which
// are loaded once.  PASSA: sub-problems are the TILE/R columns of an R x (TILE/R) tile
// (logical index u*NSP + sp); else TILE/R contiguous blocks of R words (sp*R + u).
// RED = false (primes small enough, see ntt_forward / ntt_inverse): no per-stage
// corrections.  Forward values then grow by at most 2q per stage; inverse sums double per
// stage, so the subtraction adds 2^done * q, done = inverse stages applied before this one
// (DONE0 before this pass).
template <int LOGR, int W, int LS0, bool FWD, bool PASSA, int TILE, bool RED, int DONE0>
__device__ __forceinline__ void stage_group(uint64_t *s, uint32_t s_off, uint32_t blk_base,
                                            const uint64_t *__restrict__ tw,
                                            const uint64_t *__restrict__ tws, uint64_t q) {
    constexpr int R = 1 << LOGR;
    constexpr int E = 1 << W;
    constexpr int NSP = TILE / R;
    constexpr int UPS = R >> W;
    constexpr int P_LO = FWD ? (LOGR - LS0 - W) : (LOGR - 1 - LS0);
    constexpr uint32_t LOWMASK = (1u << P_LO) - 1;
    const uint64_t two_q = 2 * q;
    for (int id = threadIdx.x; id < NSP * UPS; id += blockDim.x) {
        int sp, ub;
        if (PASSA) { sp = id % NSP; ub = id / NSP; }
        else       { ub = id % UPS; sp = id / UPS; }
        const uint32_t u_base = (((uint32_t)ub & ~LOWMASK) << W) | ((uint32_t)ub & LOWMASK);
        uint64_t x[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint32_t u = u_base + (e << P_LO);
            x[e] = s[swz(PASSA ? (u * NSP + sp) : (sp * R + u))];
        }
        const uint32_t blk = PASSA ? 0u : (blk_base + sp);
#pragma unroll
        for (int i = 0; i < W; i++) {
            const int ls = FWD ? (LS0 + i) : (LS0 - i);
            const int half = FWD ? (E >> (i + 1)) : (1 << i);
            const uint32_t base = (1u << (s_off + ls)) + (blk << ls) + (u_base >> (LOGR - ls));
            // pair p = (e, e + half); its twiddle index m is nondecreasing in p, so a
            // twiddle is loaded when m changes (all indices are compile-time constants)
            uint64_t w = 0, wsh = 0;
#pragma unroll
            for (int p = 0; p < E / 2; p++) {
                const int e = FWD ? ((p / half) * 2 * half + (p % half)) : (((p >> i) << (i + 1)) | (p & (half - 1)));
                const int m = FWD ? (e >> (W - i)) : (p >> i);
                const int pe = FWD ? (((p - 1) / half) * 2 * half + ((p - 1) % half)) : 0;
                const int pm = p == 0 ? -1 : (FWD ? (pe >> (W - i)) : ((p - 1) >> i));
                if (m != pm) {
                    w = __ldg(tw + base + m);
                    wsh = __ldg(tws + base + m);
                }
                uint64_t X = x[e], Y = x[e + half];
                if (FWD) {
                    if (RED) X = X >= two_q ? X - two_q : X;
                    const uint64_t T = shoup_lazy(Y, w, wsh, q);
                    x[e] = X + T;
                    x[e + half] = X - T + two_q;
                } else if (RED) {
                    const uint64_t S = X + Y;
                    x[e] = S >= two_q ? S - two_q : S;
                    x[e + half] = shoup_lazy(X - Y + two_q, w, wsh, q);
                } else {
                    const int done = DONE0 + (LOGR - 1 - ls);
                    x[e] = X + Y;
                    x[e + half] = shoup_lazy(X - Y + (q << done), w, wsh, q);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint32_t u = u_base + (e << P_LO);
            s[swz(PASSA ? (u * NSP + sp) : (sp * R + u))] = x[e];
        }
    }
}

template <int LOGR, bool FWD, bool PASSA, int TILE, bool RED, int DONE0>
__device__ __forceinline__ void all_groups(uint64_t *s, uint32_t s_off, uint32_t blk_base,
                                           const uint64_t *tw, const uint64_t *tws, uint64_t q) {
    constexpr int W0 = Split<LOGR>::W0, W1 = Split<LOGR>::W1;
    stage_group<LOGR, W0, FWD ? 0 : LOGR - 1, FWD, PASSA, TILE, RED, DONE0>(s, s_off, blk_base, tw, tws, q);
    __syncthreads();
    stage_group<LOGR, W1, FWD ? W0 : LOGR - 1 - W0, FWD, PASSA, TILE, RED, DONE0>(s, s_off, blk_base, tw, tws, q);
    __syncthreads();
}

// Pass A: strided columns, stages 0..LOGR-1 (forward) or LOGR-1..0 (inverse, + N^-1).
template <int LOGR, bool FWD, bool NARROW, int DONE0>
__global__ void __launch_bounds__(Tile<LOGR, NARROW>::THREADS, NARROW ? 8 : 3) ntt_pass_a(PassArgs a) {
    constexpr int TILE = Tile<LOGR, NARROW>::WORDS;
    __shared__ uint64_t s[TILE];
    constexpr int R = 1 << LOGR;
    constexpr int C = TILE / R;
    const uint32_t tiles = a.n / TILE;
    const uint32_t limb = blockIdx.x / tiles;
    const uint32_t tile = blockIdx.x % tiles;
    uint32_t pi;
    if (limb >= a.n_limbs || !a.map.resolve(limb, &pi)) return;
    const DevPrime P = a.primes[pi];
    uint64_t *g = a.data + a.map.offset(limb, a.n);
    const uint32_t cols = a.n >> LOGR;
    const uint32_t c0 = tile * C;
    for (int i = threadIdx.x; i < TILE; i += blockDim.x) {
        const int u = i / C, c = i % C;
        s[swz(i)] = g[c0 + c + (size_t)u * cols];
    }
    __syncthreads();
    const uint64_t *tw = a.tw + (size_t)pi * a.n, *tws = a.tw_sh + (size_t)pi * a.n;
    if (P.q < a.small_below) all_groups<LOGR, FWD, true, TILE, false, DONE0>(s, 0, 0, tw, tws, P.q);
    else all_groups<LOGR, FWD, true, TILE, true, DONE0>(s, 0, 0, tw, tws, P.q);
    for (int i = threadIdx.x; i < TILE; i += blockDim.x) {
        const int u = i / C, c = i % C;
        uint64_t v = s[swz(i)];
        if (!FWD) {
            v = shoup_lazy(v, P.n_inv, P.n_inv_sh, P.q);
            v = v >= P.q ? v - P.q : v;
        }
        g[c0 + c + (size_t)u * cols] = v;
    }
}

// Pass B: contiguous blocks of R words, stages s_off..s_off+LOGR-1.
template <int LOGR, bool FWD, bool NARROW>
__global__ void __launch_bounds__(Tile<LOGR, NARROW>::THREADS, NARROW ? 8 : 3) ntt_pass_b(PassArgs a, uint32_t s_off) {
    constexpr int TILE = Tile<LOGR, NARROW>::WORDS;
    __shared__ uint64_t s[TILE];
    constexpr int R = 1 << LOGR;
    constexpr int S = TILE / R;
    const uint32_t tiles = a.n / TILE;
    const uint32_t limb = blockIdx.x / tiles;
    const uint32_t tile = blockIdx.x % tiles;
    uint32_t pi;
    if (limb >= a.n_limbs || !a.map.resolve(limb, &pi)) return;
    const DevPrime P = a.primes[pi];
    uint64_t *g = a.data + a.map.offset(limb, a.n) + (size_t)tile * TILE;
    for (int i = threadIdx.x; i < TILE / 2; i += blockDim.x) {
        const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(g)[i];
        s[swz(2 * i)] = v.x;
        s[swz(2 * i + 1)] = v.y;
    }
    __syncthreads();
    const uint64_t *tw = a.tw + (size_t)pi * a.n, *tws = a.tw_sh + (size_t)pi * a.n;
    const bool small = P.q < a.small_below;
    if (small) all_groups<LOGR, FWD, false, TILE, false, 0>(s, s_off, tile * S, tw, tws, P.q);
    else all_groups<LOGR, FWD, false, TILE, true, 0>(s, s_off, tile * S, tw, tws, P.q);
    const uint64_t q = P.q, two_q = 2 * q;
    for (int i = threadIdx.x; i < TILE / 2; i += blockDim.x) {
        ulonglong2 v;
        v.x = s[swz(2 * i)];
        v.y = s[swz(2 * i + 1)];
        if (FWD && small) {     // values below (1 + 2 logN) q: one Shoup reduction
            v.x = shoup(v.x, 1, P.one_sh, q);
            v.y = shoup(v.y, 1, P.one_sh, q);
        } else if (FWD) {
            v.x = v.x >= two_q ? v.x - two_q : v.x;
            v.x = v.x >= q ? v.x - q : v.x;
            v.y = v.y >= two_q ? v.y - two_q : v.y;
            v.y = v.y >= q ? v.y - q : v.y;
        }
        reinterpret_cast<ulonglong2 *>(g)[i] = v;
    }
}

// a launch whose wide tiles would not give every SM two CTAs runs the narrow variant
constexpr uint32_t kNarrowBelow = 2 * 152;

template <int A, int B, bool NARROW>
void launch_fwd_t(const PassArgs &a, cudaStream_t st) {
    ntt_pass_a<A, true, NARROW, 0><<<a.n_limbs * (a.n / Tile<A, NARROW>::WORDS), Tile<A, NARROW>::THREADS, 0, st>>>(a);
    ntt_pass_b<B, true, NARROW><<<a.n_limbs * (a.n / Tile<B, NARROW>::WORDS), Tile<B, NARROW>::THREADS, 0, st>>>(a, A);
}
template <int A, int B, bool NARROW>
void launch_inv_t(const PassArgs &a, cudaStream_t st) {
    ntt_pass_b<B, false, NARROW><<<a.n_limbs * (a.n / Tile<B, NARROW>::WORDS), Tile<B, NARROW>::THREADS, 0, st>>>(a, A);
    ntt_pass_a<A, false, NARROW, B><<<a.n_limbs * (a.n / Tile<A, NARROW>::WORDS), Tile<A, NARROW>::THREADS, 0, st>>>(a);
}
template <int A, int B>
void launch_fwd(const PassArgs &a, cudaStream_t st) {
    if (a.n_limbs * (a.n / Split<A>::TILE) < kNarrowBelow) launch_fwd_t<A, B, true>(a, st);
    else launch_fwd_t<A, B, false>(a, st);
}
template <int A, int B>
void launch_inv(const PassArgs &a, cudaStream_t st) {
    if (a.n_limbs * (a.n / Split<A>::TILE) < kNarrowBelow) launch_inv_t<A, B, true>(a, st);
    else launch_inv_t<A, B, false>(a, st);
}

PassArgs make_args(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, bool fwd) {
    PassArgs a;
    a.data = data;
    a.n_limbs = n_limbs;
    a.log_n = ctx->log_n;
    a.n = ctx->n;
    a.map = map;
    a.primes = ctx->dev_primes();
    const size_t plane = (size_t)ctx->nqp() * ctx->n;
    const uint64_t *base = ctx->d_tw.u64();
    a.tw = base + (fwd ? 0 : 2 * plane);
    a.tw_sh = base + (fwd ? plane : 3 * plane);
    // forward: values stay below (1 + 2 logN) q < 2^64 for q < 2^58; inverse: below
    // 2^(logN+1) q < 2^64 for q < 2^(63 - logN)
    a.small_below = fwd ? (1ull << 58) : (1ull << (63 - ctx->log_n));
    return a;
}

}  // namespace

// algorithmic bytes of one NTT over the limbs a launch transforms: each residue read once
// and written once
double ntt_bytes(const hear_context *ctx, uint32_t n_limbs, const LimbMap &map) {
    uint32_t active = 0, pi;
    for (uint32_t b = 0; b < n_limbs; b++) active += map.resolve(b, &pi) ? 1 : 0;
    return 16.0 * (double)ctx->n * active;
}

void ntt_forward(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, cudaStream_t s) {
    if (n_limbs == 0) return;
    ProfScope ps(ctx, "ntt_fwd", s, ntt_bytes(ctx, n_limbs, map), 2);
    PassArgs a = make_args(ctx, data, n_limbs, map, true);
    switch (ctx->log_n) {
    case 11: launch_fwd<6, 5>(a, s); break;
    case 12: launch_fwd<6, 6>(a, s); break;
    case 13: launch_fwd<7, 6>(a, s); break;
    case 14: launch_fwd<7, 7>(a, s); break;
    case 15: launch_fwd<8, 7>(a, s); break;
    case 16: launch_fwd<8, 8>(a, s); break;
    default: throw Error(HEAR_E_UNSUPPORTED, "log_n outside [11, 16]");
    }
    HEAR_CHECK_CUDA(cudaGetLastError());
}

void ntt_inverse(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, cudaStream_t s) {
    if (n_limbs == 0) return;
    ProfScope ps(ctx, "ntt_inv", s, ntt_bytes(ctx, n_limbs, map), 2);
    PassArgs a = make_args(ctx, data, n_limbs, map, false);
    switch (ctx->log_n) {
    case 11: launch_inv<6, 5>(a, s); break;
    case 12: launch_inv<6, 6>(a, s); break;
    case 13: launch_inv<7, 6>(a, s); break;
    case 14: launch_inv<7, 7>(a, s); break;
    case 15: launch_inv<8, 7>(a, s); break;
    case 16: launch_inv<8, 8>(a, s); break;
    default: throw Error(HEAR_E_UNSUPPORTED, "log_n outside [11, 16]");
    }
    HEAR_CHECK_CUDA(cudaGetLastError());
}

}  // namespace hear
