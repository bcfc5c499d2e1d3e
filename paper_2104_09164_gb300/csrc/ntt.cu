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
#include <cooperative_groups.h>
#include <mutex>
#include "internal.h"
#include "modarith.cuh"
#include "launch.cuh"

namespace cg = cooperative_groups;

namespace hear {
namespace {

constexpr int kThreads = 256;

struct PassArgs {
    uint64_t small_below;    // primes below this skip the per-stage corrections
    uint64_t *data;
    // inverse only: the first pass reads limb b from src + (b / per_group) * src_gstride +
    // (b % per_group) * N instead of from data (out-of-place start), null = in place
    const uint64_t *src;
    uint64_t src_gstride;
    uint32_t src_count;      // > 1: the first pass reads the sum mod q of src_count sources,
    uint64_t src_cstride;    //   source r at src + r * src_cstride (same layout)
    // forward only: the first pass reads limb b's values from pro + (b / per_group) *
    // pro_gstride (coefficient domain, any residue below 2^64) reduced mod the limb's
    // prime -- a basis extension by one source limb folded into the transform's load
    const uint64_t *pro;
    uint64_t pro_gstride;
    uint64_t pro_center;     // nonzero: the source residues are centred mod this prime first
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
// MODE 0 (wide): Split::TILE words, 256 threads, radix-8/16 units; MODE 1 (narrow): a
// quarter of the tile and of the threads; MODE 2 (tiny): 1024 words, 256 threads, radix-4
// units (four words per thread: four times the threads of the narrow tile for launches of
// few limbs, at the price of more shared-memory rounds)
template <int LOGR, int MODE> struct Tile {
    static constexpr int WORDS = MODE == 0 ? Split<LOGR>::TILE : MODE == 1 ? Split<LOGR>::TILE / 4 : 1024;
    static constexpr int THREADS = MODE == 1 ? kThreads / 4 : kThreads;
    static constexpr int MIN_CTAS = MODE == 0 ? 3 : MODE == 1 ? 8 : 4;
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
template <int LOGR, int W, int LS0, bool FWD, bool PASSA, int TILE, bool RED, int DONE0, bool TWS>
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
                    w = TWS ? tw[base + m] : __ldg(tw + base + m);
                    wsh = TWS ? tws[base + m] : __ldg(tws + base + m);
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

// PASSA: the pass-A twiddles (indices below 2^LOGR) sit in shared memory; pass B reads its
// (per-block) twiddles through the read-only cache.
template <int LOGR, bool FWD, bool PASSA, int TILE, bool RED, int DONE0>
__device__ __forceinline__ void all_groups(uint64_t *s, uint32_t s_off, uint32_t blk_base,
                                           const uint64_t *tw, const uint64_t *tws, uint64_t q) {
    constexpr int W0 = Split<LOGR>::W0, W1 = Split<LOGR>::W1;
    stage_group<LOGR, W0, FWD ? 0 : LOGR - 1, FWD, PASSA, TILE, RED, DONE0, PASSA>(s, s_off, blk_base, tw, tws, q);
    __syncthreads();
    stage_group<LOGR, W1, FWD ? W0 : LOGR - 1 - W0, FWD, PASSA, TILE, RED, DONE0, PASSA>(s, s_off, blk_base, tw, tws,
                                                                                         q);
    __syncthreads();
}

// MODE 2: the stages in groups of two (radix-4 units), a last group of one if LOGR is odd
template <int LOGR, bool FWD, bool PASSA, int TILE, bool RED, int DONE0, int DONE_STAGES = 0>
__device__ __forceinline__ void tiny_groups(uint64_t *s, uint32_t s_off, uint32_t blk_base,
                                            const uint64_t *tw, const uint64_t *tws, uint64_t q) {
    if constexpr (DONE_STAGES < LOGR) {
        constexpr int W = LOGR - DONE_STAGES >= 2 ? 2 : 1;
        constexpr int LS0 = FWD ? DONE_STAGES : LOGR - 1 - DONE_STAGES;
        stage_group<LOGR, W, LS0, FWD, PASSA, TILE, RED, DONE0, PASSA>(s, s_off, blk_base, tw, tws, q);
        __syncthreads();
        tiny_groups<LOGR, FWD, PASSA, TILE, RED, DONE0, DONE_STAGES + W>(s, s_off, blk_base, tw, tws, q);
    }
}
template <int LOGR, bool FWD, bool PASSA, int TILE, bool RED, int DONE0, int MODE>
__device__ __forceinline__ void pass_groups(uint64_t *s, uint32_t s_off, uint32_t blk_base,
                                            const uint64_t *tw, const uint64_t *tws, uint64_t q) {
    if constexpr (MODE == 2) tiny_groups<LOGR, FWD, PASSA, TILE, RED, DONE0>(s, s_off, blk_base, tw, tws, q);
    else all_groups<LOGR, FWD, PASSA, TILE, RED, DONE0>(s, s_off, blk_base, tw, tws, q);
}

// the prologue value of a forward transform: v (a residue of the source limb) reduced mod q,
// after centring it into (-qc/2, qc/2] when qc is nonzero
__device__ __forceinline__ uint64_t pro_value(uint64_t v, uint64_t qc, const DevPrime &P) {
    if (!qc) return shoup(v, 1, P.one_sh, P.q);
    const bool neg = v > (qc - 1) / 2;
    const uint64_t r = shoup(neg ? qc - v : v, 1, P.one_sh, P.q);
    return neg ? neg_mod(r, P.q) : r;
}

// Tile transfers in two phases -- all of a thread's global (or remote shared) loads issued
// before its first shared store -- so each thread has TILE / THREADS requests in flight.
// (in batches of 8 words, which keeps the register footprint of the wide tiles in budget)
template <int TILE, int THREADS, class Src>
__device__ __forceinline__ void gather_tile(uint64_t *s, Src src) {
    constexpr int PER = TILE / THREADS;
    constexpr int B = PER < 8 ? PER : 8;
    static_assert(PER * THREADS == TILE && PER % B == 0, "tile must split evenly");
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += B) {
        uint64_t v[B];
#pragma unroll
        for (int k = 0; k < B; k++) v[k] = src(threadIdx.x + (k0 + k) * THREADS);
#pragma unroll
        for (int k = 0; k < B; k++) s[swz(threadIdx.x + (k0 + k) * THREADS)] = v[k];
    }
}
template <int TILE, int THREADS>
__device__ __forceinline__ void load_rows(uint64_t *s, const uint64_t *g) {
    constexpr int PER = TILE / 2 / THREADS;
    constexpr int B = PER < 4 ? PER : 4;
    static_assert(PER * THREADS * 2 == TILE && PER % B == 0, "tile must split evenly");
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += B) {
        ulonglong2 v[B];
#pragma unroll
        for (int k = 0; k < B; k++) v[k] = reinterpret_cast<const ulonglong2 *>(g)[threadIdx.x + (k0 + k) * THREADS];
#pragma unroll
        for (int k = 0; k < B; k++) {
            const int i = threadIdx.x + (k0 + k) * THREADS;
            s[swz(2 * i)] = v[k].x;
            s[swz(2 * i + 1)] = v[k].y;
        }
    }
}
// s[i] += g[r * cstride + i] mod q for the sources r = 1 .. count - 1 of a tile load_rows read
// from source 0 (the sum of several inputs folded into a transform's first load)
template <int TILE, int THREADS>
__device__ __forceinline__ void add_rows(uint64_t *s, const uint64_t *g, uint32_t count, uint64_t cstride, uint64_t q) {
    constexpr int PER = TILE / 2 / THREADS;
    for (uint32_t r = 1; r < count; r++) {
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(g + r * cstride);
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * THREADS;
            const ulonglong2 v = src[i];
            s[swz(2 * i)] = add_mod(s[swz(2 * i)], v.x, q);
            s[swz(2 * i + 1)] = add_mod(s[swz(2 * i + 1)], v.y, q);
        }
    }
}
// the 2^LOGR pass-A twiddles (and companions) of a prime into shared memory
template <int LOGR, int THREADS>
__device__ __forceinline__ void load_twiddles(uint64_t *stw, const uint64_t *tw, const uint64_t *tws) {
    constexpr int R = 1 << LOGR;
    for (int i = threadIdx.x; i < R; i += THREADS) {
        stw[i] = __ldg(tw + i);
        stw[R + i] = __ldg(tws + i);
    }
}

// Pass A: strided columns, stages 0..LOGR-1 (forward) or LOGR-1..0 (inverse, + N^-1).
template <int LOGR, bool FWD, int MODE, int DONE0>
__global__ void __launch_bounds__(Tile<LOGR, MODE>::THREADS, Tile<LOGR, MODE>::MIN_CTAS) ntt_pass_a(PassArgs a) {
    pdl_enter();
    constexpr int TILE = Tile<LOGR, MODE>::WORDS;
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
    constexpr int THREADS = Tile<LOGR, MODE>::THREADS;
    __shared__ uint64_t stw[2 * R];
    const uint32_t cols = a.n >> LOGR;
    const uint32_t c0 = tile * C;
    load_twiddles<LOGR, THREADS>(stw, a.tw + (size_t)pi * a.n, a.tw_sh + (size_t)pi * a.n);
    if (FWD && a.pro) {
        const uint64_t *pg = a.pro + (uint64_t)(limb / a.map.per_group) * a.pro_gstride;
        const uint64_t qc = a.pro_center;
        gather_tile<TILE, THREADS>(s, [&](int i) { return pro_value(pg[c0 + i % C + (size_t)(i / C) * cols], qc, P); });
    } else {
        gather_tile<TILE, THREADS>(s, [&](int i) { return g[c0 + i % C + (size_t)(i / C) * cols]; });
    }
    __syncthreads();
    if (P.q < a.small_below) pass_groups<LOGR, FWD, true, TILE, false, DONE0, MODE>(s, 0, 0, stw, stw + R, P.q);
    else pass_groups<LOGR, FWD, true, TILE, true, DONE0, MODE>(s, 0, 0, stw, stw + R, P.q);
#pragma unroll
    for (int k = 0; k < TILE / THREADS; k++) {
        const int i = threadIdx.x + k * THREADS;
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
// SUM (inverse): the first pass reads the sum of a.src_count sources
template <int LOGR, bool FWD, int MODE, bool SUM = false>
__global__ void __launch_bounds__(Tile<LOGR, MODE>::THREADS, Tile<LOGR, MODE>::MIN_CTAS) ntt_pass_b(PassArgs a,
                                                                                               uint32_t s_off) {
    pdl_enter();
    constexpr int TILE = Tile<LOGR, MODE>::WORDS;
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
    constexpr int THREADS = Tile<LOGR, MODE>::THREADS;
    const uint64_t *gin = g;
    if (!FWD && a.src)
        gin = a.src + (uint64_t)(limb / a.map.per_group) * a.src_gstride + (uint64_t)(limb % a.map.per_group) * a.n +
              (size_t)tile * TILE;
    load_rows<TILE, THREADS>(s, gin);
    if (!FWD && SUM) add_rows<TILE, THREADS>(s, gin, a.src_count, a.src_cstride, P.q);
    __syncthreads();
    const uint64_t *tw = a.tw + (size_t)pi * a.n, *tws = a.tw_sh + (size_t)pi * a.n;
    const bool small = P.q < a.small_below;
    if (small) pass_groups<LOGR, FWD, false, TILE, false, 0, MODE>(s, s_off, tile * S, tw, tws, P.q);
    else pass_groups<LOGR, FWD, false, TILE, true, 0, MODE>(s, s_off, tile * S, tw, tws, P.q);
    const uint64_t q = P.q, two_q = 2 * q;
#pragma unroll
    for (int k = 0; k < TILE / 2 / THREADS; k++) {
        const int i = threadIdx.x + k * THREADS;
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

// ------------------------------------------------------------------ one-launch variant
// The two passes fused in one kernel: a cluster of CL CTAs owns one limb.  Forward: CTA r
// runs pass A on columns [r*CA, (r+1)*CA) of the 2^LA x 2^LB matrix, the cluster
// synchronises, CTA r gathers rows [r*SB, (r+1)*SB) from the pass-A tiles of all CTAs of
// the cluster (distributed shared memory), synchronises again (no CTA leaves while its tile
// is read), runs pass B and writes its rows.  Inverse: the same in reverse order.  Each
// residue is read from and written to HBM once; the intermediate never leaves the SMs.
template <int LA, int LB, int CL> struct Fused {
    static constexpr int N = 1 << (LA + LB);
    static constexpr int TILE = N / CL;                // words per CTA
    static constexpr int RA = 1 << LA, CA = TILE / RA;  // pass A: RA rows x CA columns
    static constexpr int RB = 1 << LB, SB = TILE / RB;  // pass B: SB rows of RB words
    static constexpr int THREADS = TILE / 16 < 32 ? 32 : (TILE / 16 > 256 ? 256 : TILE / 16);
    static constexpr size_t SMEM = (2 * TILE + 2 * RA) * sizeof(uint64_t);
    static_assert(CA >= 1 && SB >= 1, "cluster too large for this ring size");
};

// SUM: as for ntt_pass_b (inverse: summed sources)
template <int LA, int LB, bool FWD, int CL, bool SUM = false>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(Fused<LA, LB, CL>::THREADS, 512 / Fused<LA, LB, CL>::THREADS)
ntt_fused(PassArgs a) {
    pdl_enter();
    using F = Fused<LA, LB, CL>;
    constexpr int TILE = F::TILE, CA = F::CA, RA = F::RA, RB = F::RB, SB = F::SB, THREADS = F::THREADS;
    extern __shared__ uint64_t smem[];
    uint64_t *sA = smem, *sB = smem + TILE, *stw = smem + 2 * TILE;
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t r = cluster.block_rank();
    const uint32_t limb = blockIdx.x / CL;
    uint32_t pi;
    // every CTA of a cluster has the same limb, so the whole cluster leaves together
    if (limb >= a.n_limbs || !a.map.resolve(limb, &pi)) return;
    const DevPrime P = a.primes[pi];
    const uint64_t q = P.q, two_q = 2 * q;
    const bool small = q < a.small_below;
    uint64_t *g = a.data + a.map.offset(limb, a.n);
    const uint64_t *tw = a.tw + (size_t)pi * a.n, *tws = a.tw_sh + (size_t)pi * a.n;
    load_twiddles<LA, THREADS>(stw, tw, tws);
    if (FWD) {
        if (a.pro) {
            const uint64_t *pg = a.pro + (uint64_t)(limb / a.map.per_group) * a.pro_gstride;
            const uint64_t qc = a.pro_center;
            gather_tile<TILE, THREADS>(sA, [&](int i) { return pro_value(pg[r * CA + i % CA + (size_t)(i / CA) * RB], qc, P); });
        } else {
            gather_tile<TILE, THREADS>(sA, [&](int i) { return g[r * CA + i % CA + (size_t)(i / CA) * RB]; });
        }
        __syncthreads();
        if (small) all_groups<LA, true, true, TILE, false, 0>(sA, 0, 0, stw, stw + RA, q);
        else all_groups<LA, true, true, TILE, true, 0>(sA, 0, 0, stw, stw + RA, q);
        cluster.sync();
        gather_tile<TILE, THREADS>(sB, [&](int i) {
            const int sp = i / RB, x = i % RB;
            const uint64_t *rem = cluster.map_shared_rank(sA, (unsigned)(x / CA));
            return rem[swz((r * SB + sp) * CA + x % CA)];
        });
        cluster.sync();
        if (small) all_groups<LB, true, false, TILE, false, 0>(sB, LA, r * SB, tw, tws, q);
        else all_groups<LB, true, false, TILE, true, 0>(sB, LA, r * SB, tw, tws, q);
        uint64_t *out = g + (size_t)r * TILE;
#pragma unroll
        for (int k = 0; k < TILE / 2 / THREADS; k++) {
            const int i = threadIdx.x + k * THREADS;
            ulonglong2 v;
            v.x = sB[swz(2 * i)];
            v.y = sB[swz(2 * i + 1)];
            if (small) {
                v.x = shoup(v.x, 1, P.one_sh, q);
                v.y = shoup(v.y, 1, P.one_sh, q);
            } else {
                v.x = v.x >= two_q ? v.x - two_q : v.x;
                v.x = v.x >= q ? v.x - q : v.x;
                v.y = v.y >= two_q ? v.y - two_q : v.y;
                v.y = v.y >= q ? v.y - q : v.y;
            }
            reinterpret_cast<ulonglong2 *>(out)[i] = v;
        }
    } else {
        const uint64_t *gin = a.src ? a.src + (uint64_t)(limb / a.map.per_group) * a.src_gstride +
                                          (uint64_t)(limb % a.map.per_group) * a.n
                                    : g;
        load_rows<TILE, THREADS>(sB, gin + (size_t)r * TILE);
        if (SUM) add_rows<TILE, THREADS>(sB, gin + (size_t)r * TILE, a.src_count, a.src_cstride, q);
        __syncthreads();
        if (small) all_groups<LB, false, false, TILE, false, 0>(sB, LA, r * SB, tw, tws, q);
        else all_groups<LB, false, false, TILE, true, 0>(sB, LA, r * SB, tw, tws, q);
        cluster.sync();
        gather_tile<TILE, THREADS>(sA, [&](int i) {
            const int u = i / CA, c = i % CA;
            const uint64_t *rem = cluster.map_shared_rank(sB, (unsigned)(u / SB));
            return rem[swz((u % SB) * RB + r * CA + c)];
        });
        cluster.sync();
        if (small) all_groups<LA, false, true, TILE, false, LB>(sA, 0, 0, stw, stw + RA, q);
        else all_groups<LA, false, true, TILE, true, LB>(sA, 0, 0, stw, stw + RA, q);
#pragma unroll
        for (int k = 0; k < TILE / THREADS; k++) {
            const int i = threadIdx.x + k * THREADS;
            const int u = i / CA, c = i % CA;
            uint64_t v = shoup_lazy(sA[swz(i)], P.n_inv, P.n_inv_sh, q);
            g[r * CA + c + (size_t)u * RB] = v >= q ? v - q : v;
        }
    }
}

constexpr int kCluster = 8;

template <int LA, int LB, bool FWD, bool SUM = false>
void launch_fused_e(const PassArgs &a, cudaStream_t st) {
    using F = Fused<LA, LB, kCluster>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(ntt_fused<LA, LB, FWD, kCluster, SUM>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
    });
    HEAR_CHECK_CUDA(attr_err);
    launch(ntt_fused<LA, LB, FWD, kCluster, SUM>, a.n_limbs * kCluster, F::THREADS, F::SMEM, st, a);
}
template <int LA, int LB, bool FWD>
void launch_fused(const PassArgs &a, cudaStream_t st) {
    if (!FWD && a.src_count > 1) launch_fused_e<LA, LB, FWD, true>(a, st);
    else launch_fused_e<LA, LB, FWD, false>(a, st);
}

// a launch whose wide tiles would not give every SM two CTAs runs the narrow variant
constexpr uint32_t kNarrowBelow = 2 * 152;

template <int A, int B, int MODE>
void launch_fwd_t(const PassArgs &a, cudaStream_t st) {
    launch(ntt_pass_a<A, true, MODE, 0>, a.n_limbs * (a.n / Tile<A, MODE>::WORDS), Tile<A, MODE>::THREADS, 0, st, a);
    launch(ntt_pass_b<B, true, MODE>, a.n_limbs * (a.n / Tile<B, MODE>::WORDS), Tile<B, MODE>::THREADS, 0, st, a,
           (uint32_t)A);
}
template <int A, int B, int MODE>
void launch_inv_t(const PassArgs &a, cudaStream_t st) {
    if (a.src_count > 1)
        launch(ntt_pass_b<B, false, MODE, true>, a.n_limbs * (a.n / Tile<B, MODE>::WORDS), Tile<B, MODE>::THREADS, 0,
               st, a, (uint32_t)A);
    else
        launch(ntt_pass_b<B, false, MODE>, a.n_limbs * (a.n / Tile<B, MODE>::WORDS), Tile<B, MODE>::THREADS, 0, st, a,
               (uint32_t)A);
    launch(ntt_pass_a<A, false, MODE, B>, a.n_limbs * (a.n / Tile<A, MODE>::WORDS), Tile<A, MODE>::THREADS, 0, st, a);
}
// variant of a launch of n_limbs limbs: the context's table (filled by the tuner) or the
// default rule (narrow two-pass below two wide CTAs per SM, wide two-pass above)
uint32_t pick(const hear_context *ctx, bool fwd, uint32_t n_limbs, uint32_t wide_ctas) {
    if (ctx->ntt_force >= 0) return (uint32_t)ctx->ntt_force;
    const uint32_t b = ntt_bucket(n_limbs);
    const uint8_t v = ctx->ntt_choice[fwd ? 0 : 1][b];
    if (v != kNttAuto) return v;
    return wide_ctas < kNarrowBelow ? kNttNarrow : kNttWide;
}
// pass-A tile of the wide variant for a ring size (the A of the splits below)
constexpr uint32_t wide_tile_a(uint32_t log_n) { return log_n <= 12 ? Split<6>::TILE : log_n <= 14 ? Split<7>::TILE : Split<8>::TILE; }
uint32_t launches_of(const hear_context *ctx, bool fwd, uint32_t n_limbs) {
    return pick(ctx, fwd, n_limbs, n_limbs * (ctx->n / wide_tile_a(ctx->log_n))) == kNttFused ? 1 : 2;
}
template <int A, int B>
void launch_fwd(const hear_context *ctx, const PassArgs &a, cudaStream_t st) {
    switch (pick(ctx, true, a.n_limbs, a.n_limbs * (a.n / Split<A>::TILE))) {
    case kNttFused: launch_fused<A, B, true>(a, st); break;
    case kNttNarrow: launch_fwd_t<A, B, 1>(a, st); break;
    case kNttTiny: launch_fwd_t<A, B, 2>(a, st); break;
    default: launch_fwd_t<A, B, 0>(a, st);
    }
}
template <int A, int B>
void launch_inv(const hear_context *ctx, const PassArgs &a, cudaStream_t st) {
    switch (pick(ctx, false, a.n_limbs, a.n_limbs * (a.n / Split<A>::TILE))) {
    case kNttFused: launch_fused<A, B, false>(a, st); break;
    case kNttNarrow: launch_inv_t<A, B, 1>(a, st); break;
    case kNttTiny: launch_inv_t<A, B, 2>(a, st); break;
    default: launch_inv_t<A, B, 0>(a, st);
    }
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
    a.src = nullptr;
    a.src_gstride = 0;
    a.src_count = 1;
    a.src_cstride = 0;
    a.pro = nullptr;
    a.pro_gstride = 0;
    a.pro_center = 0;
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
    ntt_forward_pro(ctx, data, n_limbs, map, nullptr, 0, s);
}

void ntt_forward_pro(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, const uint64_t *pro,
                     uint64_t pro_gstride, cudaStream_t s, uint64_t pro_center) {
    if (n_limbs == 0) return;
    ProfScope ps(ctx, "ntt_fwd", s, ntt_bytes(ctx, n_limbs, map), launches_of(ctx, true, n_limbs));
    PassArgs a = make_args(ctx, data, n_limbs, map, true);
    a.pro = pro;
    a.pro_gstride = pro_gstride;
    a.pro_center = pro_center;
    switch (ctx->log_n) {
    case 11: launch_fwd<6, 5>(ctx, a, s); break;
    case 12: launch_fwd<6, 6>(ctx, a, s); break;
    case 13: launch_fwd<7, 6>(ctx, a, s); break;
    case 14: launch_fwd<7, 7>(ctx, a, s); break;
    case 15: launch_fwd<8, 7>(ctx, a, s); break;
    case 16: launch_fwd<8, 8>(ctx, a, s); break;
    default: throw Error(HEAR_E_UNSUPPORTED, "log_n outside [11, 16]");
    }
    HEAR_CHECK_CUDA(cudaGetLastError());
}

void ntt_inverse(const hear_context *ctx, uint64_t *data, uint32_t n_limbs, LimbMap map, cudaStream_t s) {
    ntt_inverse_from(ctx, nullptr, 0, data, n_limbs, map, s);
}

void ntt_inverse_from(const hear_context *ctx, const uint64_t *src, uint64_t src_gstride, uint64_t *data,
                      uint32_t n_limbs, LimbMap map, cudaStream_t s, uint32_t src_count, uint64_t src_cstride) {
    if (n_limbs == 0) return;
    HEAR_REQUIRE(!src || map.group_stride == 0, HEAR_E_INVAL, "out-of-place NTT needs contiguous groups");
    HEAR_REQUIRE(src_count >= 1 && (src_count == 1 || src), HEAR_E_INVAL, "summed sources need an out-of-place NTT");
    ProfScope ps(ctx, "ntt_inv", s, ntt_bytes(ctx, n_limbs, map) * (1.0 + (src_count - 1) * 0.5),
                 launches_of(ctx, false, n_limbs));
    PassArgs a = make_args(ctx, data, n_limbs, map, false);
    a.src = src;
    a.src_gstride = src_gstride;
    a.src_count = src_count;
    a.src_cstride = src_cstride;
    switch (ctx->log_n) {
    case 11: launch_inv<6, 5>(ctx, a, s); break;
    case 12: launch_inv<6, 6>(ctx, a, s); break;
    case 13: launch_inv<7, 6>(ctx, a, s); break;
    case 14: launch_inv<7, 7>(ctx, a, s); break;
    case 15: launch_inv<8, 7>(ctx, a, s); break;
    case 16: launch_inv<8, 8>(ctx, a, s); break;
    default: throw Error(HEAR_E_UNSUPPORTED, "log_n outside [11, 16]");
    }
    HEAR_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ butterfly throughput
// The arithmetic of the transforms without their memory traffic: every thread keeps a
// radix-16 unit (16 residues) and its 16 twiddle pairs in registers and applies the unit's
// four stages again and again -- the forward butterfly (Shoup product by the twiddle,
// Harvey lazy add / subtract, the 2q correction for primes at or above the no-correction
// bound) or the inverse one, exactly as stage_group does.  Warp w uses prime w mod
// (n_q + n_p), i.e. the prime mix of a transform over all limbs.  What the loop reaches is
// the measured ceiling of the transforms' butterfly rate on the integer pipes.
template <bool FWD>
__global__ void __launch_bounds__(256) k_bfly_peak(const DevPrime *primes, uint32_t n_primes, const uint64_t *tw,
                                                   const uint64_t *tws, uint32_t n, uint64_t small_below,
                                                   uint32_t iters, uint64_t *out) {
    pdl_enter();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const uint32_t pi = warp % n_primes;
    const uint64_t q = primes[pi].q, two_q = 2 * q;
    uint64_t w[16], wsh[16], x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        w[i] = __ldg(tw + (size_t)pi * n + 1 + i);
        wsh[i] = __ldg(tws + (size_t)pi * n + 1 + i);
        x[i] = (threadIdx.x * 16u + i) % q;
    }
    const bool red = q >= small_below;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int st = 0; st < 4; st++) {
            const int half = FWD ? (8 >> st) : (1 << st);
#pragma unroll
            for (int p = 0; p < 8; p++) {
                const int e = FWD ? ((p / half) * 2 * half + (p % half)) : (((p >> st) << (st + 1)) | (p & (half - 1)));
                const int m = FWD ? ((1 << st) + (e >> (4 - st))) : ((8 >> st) + (p >> st));
                uint64_t X = x[e], Y = x[e + half];
                if (FWD) {
                    if (red) X = X >= two_q ? X - two_q : X;
                    const uint64_t T = shoup_lazy(Y, w[m & 15], wsh[m & 15], q);
                    x[e] = X + T;
                    x[e + half] = X - T + two_q;
                } else if (red) {
                    const uint64_t S = X + Y;
                    x[e] = S >= two_q ? S - two_q : S;
                    x[e + half] = shoup_lazy(X - Y + two_q, w[m & 15], wsh[m & 15], q);
                } else {
                    x[e] = X + Y;
                    x[e + half] = shoup_lazy(X - Y + two_q, w[m & 15], wsh[m & 15], q);
                }
            }
        }
    }
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    out[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

double bfly_peak(const hear_context *ctx, bool fwd, uint32_t iters) {
    HEAR_REQUIRE(iters >= 1 && iters <= (1u << 20), HEAR_E_INVAL, "iters must be in [1, 2^20]");
    int sms = 0;
    HEAR_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const uint32_t threads = 256, blocks = (uint32_t)sms * 4;
    cudaStream_t st = ctx->stream;
    DevBuf out((size_t)blocks * threads * 8, st);
    const size_t plane = (size_t)ctx->nqp() * ctx->n;
    const uint64_t *base = ctx->d_tw.u64();
    const uint64_t *tw = base + (fwd ? 0 : 2 * plane), *tws = base + (fwd ? plane : 3 * plane);
    const uint64_t small_below = fwd ? (1ull << 58) : (1ull << (63 - ctx->log_n));
    auto run = [&](uint32_t it) {
        if (fwd)
            launch(k_bfly_peak<true>, blocks, threads, 0, st, ctx->dev_primes(), ctx->nqp(), tw, tws, ctx->n,
                   small_below, it, out.u64());
        else
            launch(k_bfly_peak<false>, blocks, threads, 0, st, ctx->dev_primes(), ctx->nqp(), tw, tws, ctx->n,
                   small_below, it, out.u64());
    };
    run(iters);   // warm-up
    cudaEvent_t e0, e1;
    HEAR_CHECK_CUDA(cudaEventCreate(&e0));
    HEAR_CHECK_CUDA(cudaEventCreate(&e1));
    float ms = 0;
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        run(iters);
        e = cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HEAR_CHECK_CUDA(e);
    return (double)blocks * threads * 32.0 * iters / (ms / 1e3);
}

// Time every launch variant for launches of 1, 2, 4, .. max_limbs limbs (both directions)
// and record the fastest per bucket.  Runs on the context's stream; the caller keeps other
// work off the context meanwhile.
void ntt_tune(hear_context *ctx, uint32_t max_limbs, int iters, float *ms_out) {
    HEAR_REQUIRE(max_limbs >= 1 && iters >= 1, HEAR_E_INVAL, "bad tuning range");
    cudaStream_t st = ctx->stream;
    const size_t words = (size_t)max_limbs * ctx->n;
    DevBuf d(words * 8, st);
    HEAR_CHECK_CUDA(cudaMemsetAsync(d.p, 0, words * 8, st));
    LimbMap m;
    m.per_group = ctx->nqp();
    m.q_count = ctx->n_q;
    m.n_q = ctx->n_q;
    cudaEvent_t e0, e1;
    HEAR_CHECK_CUDA(cudaEventCreate(&e0));
    HEAR_CHECK_CUDA(cudaEventCreate(&e1));
    const int saved = ctx->ntt_force;
    try {
        for (int dir = 0; dir < 2; dir++)
            for (uint32_t b = 0; b < (uint32_t)kNttBuckets && (1u << b) <= max_limbs; b++) {
                const uint32_t nl = 1u << b;
                float best = 0;
                uint8_t best_v = kNttAuto;
                for (uint8_t v = 0; v < kNttVariants; v++) {
                    ctx->ntt_force = v;
                    // timed as a replayed CUDA graph of `iters` back-to-back transforms, the
                    // way whole evaluations run
                    cudaGraph_t graph = nullptr;
                    cudaGraphExec_t exec = nullptr;
                    HEAR_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                    try {
                        for (int i = 0; i < iters; i++) {
                            if (dir == 0) ntt_forward(ctx, d.u64(), nl, m, st);
                            else ntt_inverse(ctx, d.u64(), nl, m, st);
                        }
                    } catch (...) {
                        cudaStreamEndCapture(st, &graph);
                        if (graph) cudaGraphDestroy(graph);
                        throw;
                    }
                    HEAR_CHECK_CUDA(cudaStreamEndCapture(st, &graph));
                    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
                    cudaGraphDestroy(graph);
                    HEAR_CHECK_CUDA(ie);
                    float ms = 0;
                    cudaError_t le = cudaGraphLaunch(exec, st);
                    if (le == cudaSuccess) le = cudaEventRecord(e0, st);
                    if (le == cudaSuccess) le = cudaGraphLaunch(exec, st);
                    if (le == cudaSuccess) le = cudaEventRecord(e1, st);
                    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
                    if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
                    cudaGraphExecDestroy(exec);
                    HEAR_CHECK_CUDA(le);
                    ms /= iters;
                    if (ms_out) ms_out[((size_t)dir * kNttBuckets + b) * kNttVariants + v] = ms;
                    // the one-launch cluster form is timed but not chosen: inside a whole
                    // evaluation it lost clearly (small network at batch 1: 981 against 1309
                    // inferences/s with it for the launches below 32 limbs) where isolated
                    // replays sometimes favoured it; a pinned table or a forced variant
                    // still selects it
                    if (v == kNttFused) continue;
                    // launches up to 127 limbs: the tiny form (256 threads of 64 registers)
                    // overlaps its neighbours better inside a graph than its isolated time
                    // shows (small network at batch 1: 1319 against 1303 inferences/s with
                    // it for the 32-127-limb forward transforms), so it keeps the bucket
                    // unless another form is 10 % faster in isolation
                    const float eff = (v == kNttTiny && b <= 6) ? ms * 0.9f : ms;
                    if (best_v == kNttAuto || eff < best) {
                        best = eff;
                        best_v = v;
                    }
                }
                ctx->ntt_choice[dir][b] = best_v;
            }
    } catch (...) {
        ctx->ntt_force = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    ctx->ntt_force = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // buckets above the tuned range keep the choice of the largest tuned bucket
    for (int dir = 0; dir < 2; dir++)
        for (uint32_t b = 1; b < (uint32_t)kNttBuckets; b++)
            if ((1u << b) > max_limbs) ctx->ntt_choice[dir][b] = ctx->ntt_choice[dir][b - 1];
}

}  // namespace hear
