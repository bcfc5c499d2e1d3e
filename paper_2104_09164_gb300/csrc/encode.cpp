// encode.cpp -- CKKS encoding / decoding on the client side (host), and the CRT lift used
// by decryption.
//
// Encoding (CKKS canonical embedding): slot j of a plaintext polynomial m(X) is the value
// m(zeta^(5^j)), zeta = exp(i pi / N), j < N/2; real slot values imply the conjugate
// slots.  The inverse map used here:
//   m_k = (2/N) Re( exp(-i pi k / N) * F[k] ),   F = DFT_N(B),  B[(5^j mod 2N - 1)/2] = z_j,
// evaluated with a radix-2 FFT in double-double arithmetic (about 106-bit significands)
// so that round(scale * m_k) is the correctly rounded value of the exact real number
// unless that number lies within ~2^-60 of a half-integer (ties go away from zero).
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>
#include "encode.h"

namespace hear {
namespace {

// ---- double-double: value = hi + lo with |lo| <= ulp(hi)/2
struct DD {
    double hi, lo;
};
inline DD two_sum(double a, double b) {
    double s = a + b, v = s - a;
    return {s, (a - (s - v)) + (b - v)};
}
inline DD fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline DD operator+(DD a, DD b) {
    DD s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline DD operator-(DD a) { return {-a.hi, -a.lo}; }
inline DD operator-(DD a, DD b) { return a + (-b); }
inline DD operator*(DD a, DD b) {
    double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p, e);
}
inline DD mul_d(DD a, double b) {
    double p = a.hi * b;
    double e = std::fma(a.hi, b, -p) + a.lo * b;
    return fast_two_sum(p, e);
}
inline DD div_d(DD a, double b) {
    double q = a.hi / b;
    double p = q * b, pe = std::fma(q, b, -p);
    double r = ((a.hi - p) - pe + a.lo) / b;
    return fast_two_sum(q, r);
}

struct CDD {
    DD re, im;
};
inline CDD operator+(const CDD &a, const CDD &b) { return {a.re + b.re, a.im + b.im}; }
inline CDD operator-(const CDD &a, const CDD &b) { return {a.re - b.re, a.im - b.im}; }
inline CDD operator*(const CDD &a, const CDD &b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// pi/2 to double-double precision
const DD kHalfPi = {1.5707963267948966, 6.123233995736766e-17};

// sin and cos of x (|x| <= pi/4) by their power series, summed from the small end
void sincos_series(DD x, DD &s, DD &c) {
    const int K = 27;                        // x^27/27! < 2^-110 for |x| <= pi/4
    DD x2 = x * x;
    // Horner: sin x = x (1 - x^2/(2*3) (1 - x^2/(4*5) (1 - ...)))
    DD hs = {1.0, 0.0}, hc = {1.0, 0.0};
    for (int k = K; k >= 1; k--) {
        hs = DD{1.0, 0.0} - div_d(x2 * hs, (double)((2 * k) * (2 * k + 1)));
        hc = DD{1.0, 0.0} - div_d(x2 * hc, (double)((2 * k - 1) * (2 * k)));
    }
    s = x * hs;
    c = hc;
}

// exp(-2 pi i m / M) for a power of two M >= 8
CDD unit_root_neg(uint64_t m, uint64_t M) {
    m &= (M - 1);
    // angle theta = 2 pi m / M = (pi/2) * (4m / M); split into quarter turns
    const uint64_t quarter = M / 4;
    uint64_t qd = m / quarter, r = m % quarter;
    bool flip = 2 * r > quarter;            // reduce to [0, pi/4] with theta' = pi/2 - theta
    uint64_t rr = flip ? quarter - r : r;
    DD x = mul_d(kHalfPi, (double)rr / (double)quarter);
    DD s, c;
    sincos_series(x, s, c);
    if (flip) std::swap(s, c);
    DD cs, sn;   // cos and sin of the full angle
    switch (qd) {
    case 0: cs = c; sn = s; break;
    case 1: cs = -s; sn = c; break;
    case 2: cs = -c; sn = -s; break;
    default: cs = s; sn = -c; break;
    }
    return {cs, -sn};
}

}  // namespace

struct EncoderTables {
    uint32_t log_n = 0, n = 0;
    std::vector<CDD> tw;         // exp(-2 pi i m / N), m < N/2
    std::vector<CDD> twist;      // exp(-i pi k / N), k < N
    std::vector<uint32_t> slot;  // (5^j mod 2N - 1)/2
};

std::shared_ptr<EncoderTables> make_encoder_tables(uint32_t log_n) {
    auto t = std::make_shared<EncoderTables>();
    t->log_n = log_n;
    t->n = 1u << log_n;
    const uint32_t n = t->n;
    t->tw.resize(n / 2);
    t->twist.resize(n);
    for (uint32_t m = 0; m < n / 2; m++) t->tw[m] = unit_root_neg(m, n);
    for (uint32_t k = 0; k < n; k++) t->twist[k] = unit_root_neg(k, 2ull * n);
    t->slot.resize(n / 2);
    uint64_t g = 1;
    for (uint32_t j = 0; j < n / 2; j++) {
        t->slot[j] = (uint32_t)((g - 1) / 2);
        g = g * 5 % (2ull * n);
    }
    return t;
}

int encode_dd(const EncoderTables &T, const double *z, double scale, int64_t *m_out) {
    const uint32_t n = T.n, logn = T.log_n;
    std::vector<CDD> a(n, CDD{{0, 0}, {0, 0}});
    for (uint32_t j = 0; j < n / 2; j++) a[T.slot[j]].re = DD{z[j], 0.0};
    // bit-reversal permutation then iterative radix-2 decimation in time
    for (uint32_t i = 0; i < n; i++) {
        uint32_t r = 0;
        for (uint32_t b = 0; b < logn; b++) r |= ((i >> b) & 1u) << (logn - 1 - b);
        if (i < r) std::swap(a[i], a[r]);
    }
    for (uint32_t len = 2; len <= n; len <<= 1) {
        const uint32_t half = len >> 1, stride = n / len;
        for (uint32_t base = 0; base < n; base += len)
            for (uint32_t j = 0; j < half; j++) {
                CDD v = a[base + j + half] * T.tw[j * stride];
                CDD u = a[base + j];
                a[base + j] = u + v;
                a[base + j + half] = u - v;
            }
    }
    const double f = 2.0 * scale / (double)n;   // exact scaling by a power of two times scale
    int near = 0;
    for (uint32_t k = 0; k < n; k++) {
        CDD w = a[k] * T.twist[k];
        DD v = mul_d(w.re, f);
        double fl = std::floor(v.hi);
        double frac = (v.hi - fl) + v.lo;
        if (frac >= 1.0) { fl += 1.0; frac -= 1.0; }
        if (frac < 0.0) { fl -= 1.0; frac += 1.0; }
        if (std::fabs(frac - 0.5) < 0x1p-30) near++;
        double r = frac > 0.5 ? fl + 1.0 : (frac < 0.5 ? fl : (fl >= 0 ? fl + 1.0 : fl));
        m_out[k] = (int64_t)r;
    }
    return near;
}

void encode_many(const EncoderTables &T, const double *z, size_t count, const double *scales, int64_t *m_out) {
    const size_t n = T.n;
    unsigned hw = std::thread::hardware_concurrency();
    unsigned nt = (unsigned)std::min<size_t>(count, hw ? hw : 4);
    if (nt <= 1) {
        for (size_t i = 0; i < count; i++) encode_dd(T, z + i * (n / 2), scales[i], m_out + i * n);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            for (size_t i = t; i < count; i += nt) encode_dd(T, z + i * (n / 2), scales[i], m_out + i * n);
        });
    for (auto &x : th) x.join();
}

// z_j = Re sum_k v_k zeta^((2 u_j + 1) k) = Re sum_k (v_k e^{i pi k/N}) e^{2 pi i u_j k / N}
void decode_double(uint32_t log_n, const double *v, double *z) {
    const uint32_t n = 1u << log_n;
    const double pi = 3.14159265358979323846;
    std::vector<std::complex<double>> a(n);
    for (uint32_t k = 0; k < n; k++) a[k] = v[k] * std::polar(1.0, pi * k / n);
    for (uint32_t i = 0; i < n; i++) {
        uint32_t r = 0;
        for (uint32_t b = 0; b < log_n; b++) r |= ((i >> b) & 1u) << (log_n - 1 - b);
        if (i < r) std::swap(a[i], a[r]);
    }
    for (uint32_t len = 2; len <= n; len <<= 1) {
        const uint32_t half = len >> 1;
        for (uint32_t j = 0; j < half; j++) {
            std::complex<double> w = std::polar(1.0, 2 * pi * j / len);
            for (uint32_t base = 0; base < n; base += len) {
                std::complex<double> u = a[base + j], t = a[base + j + half] * w;
                a[base + j] = u + t;
                a[base + j + half] = u - t;
            }
        }
    }
    uint64_t g = 1;
    for (uint32_t j = 0; j < n / 2; j++) {
        z[j] = a[(g - 1) / 2].real();
        g = g * 5 % (2ull * n);
    }
}

// CRT lift of residues [L1][N] to the centred integer in (-Q/2, Q/2], times inv_scale.
void crt_to_double(const uint64_t *res, const uint64_t *primes, uint32_t L1, uint32_t n, double inv_scale,
                   double *out) {
    typedef unsigned __int128 u128;
    const uint32_t W = L1 + 1;
    // Q and Qhat_i = Q / q_i as little-endian word arrays
    std::vector<uint64_t> Q(W, 0);
    Q[0] = 1;
    auto mul_small = [&](std::vector<uint64_t> &x, uint64_t m) {
        u128 carry = 0;
        for (uint32_t w = 0; w < W; w++) {
            u128 v = (u128)x[w] * m + carry;
            x[w] = (uint64_t)v;
            carry = v >> 64;
        }
    };
    for (uint32_t i = 0; i < L1; i++) mul_small(Q, primes[i]);
    std::vector<std::vector<uint64_t>> qhat(L1, std::vector<uint64_t>(W, 0));
    std::vector<uint64_t> qhat_inv(L1);
    for (uint32_t i = 0; i < L1; i++) {
        qhat[i][0] = 1;
        uint64_t r = 1;
        for (uint32_t i2 = 0; i2 < L1; i2++)
            if (i2 != i) {
                mul_small(qhat[i], primes[i2]);
                r = hm::mulmod(r, primes[i2] % primes[i], primes[i]);
            }
        qhat_inv[i] = hm::invmod(r, primes[i]);
    }
    std::vector<uint64_t> half(W);   // floor(Q/2)
    for (uint32_t w = 0; w < W; w++) half[w] = (Q[w] >> 1) | (w + 1 < W ? Q[w + 1] << 63 : 0);
    auto geq = [&](const std::vector<uint64_t> &a, const std::vector<uint64_t> &b) {
        for (int w = (int)W - 1; w >= 0; w--)
            if (a[w] != b[w]) return a[w] > b[w];
        return true;
    };
    auto sub = [&](std::vector<uint64_t> &a, const std::vector<uint64_t> &b) {
        uint64_t borrow = 0;
        for (uint32_t w = 0; w < W; w++) {
            u128 d = (u128)a[w] - b[w] - borrow;
            a[w] = (uint64_t)d;
            borrow = (uint64_t)(d >> 64) ? 1 : 0;
        }
    };
    auto to_double = [&](const std::vector<uint64_t> &a) {
        double r = 0;
        for (int w = (int)W - 1; w >= 0; w--) r = r * 18446744073709551616.0 + (double)a[w];
        return r;
    };
    std::vector<uint64_t> x(W), t(W);
    for (uint32_t k = 0; k < n; k++) {
        std::fill(x.begin(), x.end(), 0);
        for (uint32_t i = 0; i < L1; i++) {
            uint64_t y = hm::mulmod(res[(size_t)i * n + k], qhat_inv[i], primes[i]);
            u128 carry = 0;
            for (uint32_t w = 0; w < W; w++) {
                u128 v = (u128)qhat[i][w] * y + x[w] + carry;
                x[w] = (uint64_t)v;
                carry = v >> 64;
            }
        }
        while (geq(x, Q)) sub(x, Q);
        if (geq(x, half) && !(x == half)) {
            t = Q;
            sub(t, x);
            out[k] = -to_double(t) * inv_scale;
        } else {
            out[k] = to_double(x) * inv_scale;
        }
    }
}

}  // namespace hear
