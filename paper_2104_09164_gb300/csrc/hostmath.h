// hostmath.h -- host-side word-size modular arithmetic for parameter set-up.
#pragma once
#include <cstdint>

namespace hear {
namespace hm {

typedef unsigned __int128 u128;

inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }

inline uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

// q prime
inline uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a % q, q - 2, q); }

// floor(w * 2^64 / q)
inline uint64_t shoup_companion(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// q^-1 mod 2^64 for odd q (Newton iteration, each step doubles the correct bits)
inline uint64_t inv_2_64(uint64_t q) {
    uint64_t x = q;
    for (int i = 0; i < 6; i++) x *= 2 - q * x;
    return x;
}

// Miller-Rabin with the first twelve prime bases: deterministic below 3.3e24
inline bool is_prime(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (uint64_t a : small) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

}  // namespace hm
}  // namespace hear
