// modarith.cuh -- word-size modular arithmetic on the integer pipes (q < 2^61).
//
// Three reductions are used:
//  * Shoup multiplication by a fixed operand w with companion w' = floor(w 2^64 / q):
//    x*w - floor(x*w'/2^64)*q lies in [0, 2q) for any x < 2^64 (NTT twiddles, scalar
//    constants of basis conversion and rescale).
//  * Montgomery reduction with R = 2^64: operands stored as k*R mod q (switching keys,
//    plaintexts, secret/public keys) so a product x*(kR) reduces to x*k mod q in two
//    multiply-high and two multiply-low operations; sums of up to 8 such 128-bit
//    products are reduced once (lazy accumulation).
//  * Barrett reduction of a full 128-bit product with floor(2^128/q) when neither operand
//    is pre-scaled (ciphertext x ciphertext tensor, sampling).
#pragma once
#include <cstdint>
#include "internal.h"

namespace hear {

struct u128 {
    uint64_t lo, hi;
};

__device__ __forceinline__ u128 mul_wide(uint64_t a, uint64_t b) {
    return u128{a * b, __umul64hi(a, b)};
}
__device__ __forceinline__ void add_to(u128 &acc, u128 v) {
    uint64_t lo = acc.lo + v.lo;
    acc.hi += v.hi + (lo < acc.lo ? 1 : 0);
    acc.lo = lo;
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}
__device__ __forceinline__ uint64_t neg_mod(uint64_t a, uint64_t q) { return a ? q - a : 0; }

// x * w mod q, lazy result in [0, 2q)
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t x, uint64_t w, uint64_t w_sh, uint64_t q) {
    uint64_t qh = __umul64hi(x, w_sh);
    return x * w - qh * q;
}
__device__ __forceinline__ uint64_t shoup(uint64_t x, uint64_t w, uint64_t w_sh, uint64_t q) {
    uint64_t r = shoup_lazy(x, w, w_sh, q);
    return r >= q ? r - q : r;
}

// Montgomery reduction of T < q * 2^64: returns T * 2^-64 mod q in [0, q)
__device__ __forceinline__ uint64_t mont_reduce(u128 T, uint64_t q, uint64_t qinv) {
    uint64_t m = T.lo * qinv;
    uint64_t mh = __umul64hi(m, q);
    uint64_t t = T.hi - mh;
    return T.hi < mh ? t + q : t;
}
// a * b * 2^-64 mod q (b usually stored in Montgomery form)
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t q, uint64_t qinv) {
    return mont_reduce(mul_wide(a, b), q, qinv);
}

// Barrett reduction of a 128-bit value x (x < 2^126) with floor(2^128/q) = (rh, rl)
__device__ __forceinline__ uint64_t barrett_reduce(u128 x, uint64_t q, uint64_t rh, uint64_t rl) {
    // qhat ~ floor(x * ratio / 2^128); dropping the low partial products makes it at
    // most 3 below the true quotient
    uint64_t t = __umul64hi(x.lo, rl);
    uint64_t a_lo = x.lo * rh, a_hi = __umul64hi(x.lo, rh);
    uint64_t b_lo = x.hi * rl, b_hi = __umul64hi(x.hi, rl);
    uint64_t s = t + a_lo;
    uint64_t c1 = s < t;
    uint64_t s2 = s + b_lo;
    uint64_t c2 = s2 < s;
    uint64_t qhat = x.hi * rh + a_hi + b_hi + c1 + c2;
    uint64_t r = x.lo - qhat * q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    return r;
}
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const DevPrime &p) {
    return barrett_reduce(mul_wide(a, b), p.q, p.ratio_hi, p.ratio_lo);
}
// x (any 64-bit value) mod q
__device__ __forceinline__ uint64_t reduce64(uint64_t x, const DevPrime &p) {
    return shoup(x, 1, p.one_sh, p.q);
}

// NTT-domain index of sigma_g: (sigma_g a)[i] = a[auto_index(i, g)] (index i holds the
// evaluation at psi^(2 brv(i) + 1))
__device__ __forceinline__ uint32_t auto_index(uint32_t i, uint32_t galois, uint32_t log_n) {
    const uint32_t n2 = 2u << log_n;
    uint32_t e = 2 * (__brev(i) >> (32 - log_n)) + 1;
    uint32_t e2 = (uint32_t)(((uint64_t)e * galois) & (n2 - 1));
    return __brev((e2 - 1) >> 1) >> (32 - log_n);
}

}  // namespace hear
