"""Pins of the CPU oracle against things other than itself: brute force, closed forms,
published test vectors, big-integer arithmetic and statistical properties.

Every check here runs on the CPU only (no GPU); each is chosen so that a plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import math
import os
import random

import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import P, _u32p, _u64p, _i8p, _i64p, _dp

HERE = os.path.dirname(os.path.abspath(__file__))


def lib():
    return O.lib()


# ----------------------------------------------------------------- helpers
def negacyclic_schoolbook(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(n):
            k = i + j
            v = ai * int(b[j])
            if k < n:
                out[k] += v
            else:
                out[k - n] -= v
    return [x % q for x in out] if q else out


def crt(res, qs):
    Q = 1
    for q in qs:
        Q *= q
    out = []
    for k in range(len(res[0])):
        x = 0
        for i, q in enumerate(qs):
            qh = Q // q
            x += (int(res[i][k]) * pow(qh % q, -1, q) % q) * qh
        out.append(x % Q)
    return out, Q


def centre(x, Q):
    return x - Q if x > Q // 2 else x


# ----------------------------------------------------------------- modular arithmetic, primes
def test_mulmod_matches_bigint():
    rng = random.Random(1)
    for bits in (31, 40, 50, 60, 61):
        q = (1 << bits) - 1 if bits == 61 else rng.getrandbits(bits) | (1 << (bits - 1)) | 1
        cases = [(0, 0), (1, q - 1), (q - 1, q - 1), (q - 1, 1), (q // 2, q - 2)]
        cases += [(rng.randrange(q), rng.randrange(q)) for _ in range(2000)]
        for a, b in cases:
            assert lib().or_mulmod(a, b, q) == a * b % q


def test_is_prime_vs_trial_division():
    def trial(n):
        if n < 2:
            return False
        i = 2
        while i * i <= n:
            if n % i == 0:
                return False
            i += 1
        return True
    for n in range(0, 20000):
        assert bool(lib().or_is_prime(n)) == trial(n), n
    # Mersenne numbers: 2^61-1 prime, 2^59-1 = 179951 * 3203431780337 composite
    assert lib().or_is_prime((1 << 61) - 1) == 1
    assert lib().or_is_prime((1 << 59) - 1) == 0
    # strong pseudoprime to bases 2,3,5,7 (3215031751 = 151*751*28351)
    assert lib().or_is_prime(3215031751) == 0


def test_prime_chain_rule():
    sympy = pytest.importorskip("sympy")
    for log_n, bits in ((12, [50, 40, 40, 50]), (14, [60] + [40] * 7 + [60]), (15, [60] + [40] * 14 + [60, 60])):
        b = np.array(bits, dtype=np.uint32)
        out = np.zeros(len(bits), dtype=np.uint64)
        assert lib().or_gen_primes(log_n, P(b, _u32p), len(bits), P(out)) == 0
        got = [int(x) for x in out]
        two_n = 2 << log_n
        assert len(set(got)) == len(got)
        for i, (q, bb) in enumerate(zip(got, bits)):
            assert sympy.isprime(q) and q % two_n == 1 and q < (1 << bb) and q.bit_length() == bb
            # no unused qualifying prime between q and 2^b
            c = q + two_n
            while c < (1 << bb):
                assert not (sympy.isprime(c) and c not in got[:i]), (i, c)
                c += two_n


# ----------------------------------------------------------------- NTT
@pytest.fixture(scope="module")
def tiny():
    return O.Oracle(6, [30, 31], [32], 3.2)


def test_ntt_is_evaluation_at_odd_powers(tiny):
    n = tiny.n
    psi = np.zeros(3, dtype=np.uint64)
    lib().or_ctx_psi(tiny.h, P(psi))
    rng = np.random.default_rng(3)
    for pi in range(3):
        q = tiny.primes[pi]
        ps = int(psi[pi])
        assert pow(ps, n, q) == q - 1          # primitive 2N-th root
        a = rng.integers(0, q, size=n, dtype=np.uint64)
        A = tiny.ntt_fwd(a[None], [pi])[0]
        for i in range(n):
            x = pow(ps, 2 * i + 1, q)
            val = 0
            for k in reversed(range(n)):
                val = (val * x + int(a[k])) % q
            assert int(A[i]) == val


@pytest.mark.parametrize("log_n", [4, 7, 10])
def test_ntt_product_matches_schoolbook(log_n):
    o = O.Oracle(log_n, [40, 50], [60], 3.2)
    n = o.n
    rng = np.random.default_rng(log_n)
    for pi, q in enumerate(o.primes):
        inputs = [
            (rng.integers(0, q, n, dtype=np.uint64), rng.integers(0, q, n, dtype=np.uint64)),
            (np.eye(1, n, 0, dtype=np.uint64)[0], rng.integers(0, q, n, dtype=np.uint64)),
            (np.full(n, q - 1, dtype=np.uint64), np.full(n, q - 1, dtype=np.uint64)),
            (np.eye(1, n, n - 1, dtype=np.uint64)[0], np.eye(1, n, n - 1, dtype=np.uint64)[0]),
        ]
        for a, b in inputs:
            A = o.ntt_fwd(a[None], [pi])[0]
            B = o.ntt_fwd(b[None], [pi])[0]
            C = np.array([int(x) * int(y) % q for x, y in zip(A, B)], dtype=np.uint64)
            c = o.ntt_inv(C[None], [pi])[0]
            if log_n <= 7 or pi == 0:
                assert [int(x) for x in c] == negacyclic_schoolbook(a, b, q)
            back = o.ntt_inv(A[None], [pi])[0]
            assert np.array_equal(back, a)


# ----------------------------------------------------------------- randomness
def _read_chacha_vectors():
    rows = []
    with open(os.path.join(HERE, "golden", "chacha20_rfc8439.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, ctr, nonce, block = line.split()
            rows.append((bytes.fromhex(key), int(ctr), bytes.fromhex(nonce), bytes.fromhex(block)))
    return rows


def test_chacha20_rfc8439_vectors():
    for key, ctr, nonce, block in _read_chacha_vectors():
        k = np.frombuffer(key, dtype="<u4").astype(np.uint32).copy()
        nn = np.frombuffer(nonce, dtype="<u4").astype(np.uint32).copy()
        out = np.zeros(16, dtype=np.uint32)
        lib().or_chacha20_block(P(k, _u32p), ctr, P(nn, _u32p), P(out, _u32p))
        assert out.astype("<u4").tobytes() == block


def test_stream_word_layout():
    seed, purpose, index = 0x0123456789ABCDEF, 7, (5 << 32) | 3
    w = np.zeros(20, dtype=np.uint64)
    lib().or_stream_words(seed, purpose, index, 0, 20, P(w))
    key = np.array([seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0], dtype=np.uint32)
    nonce = np.array([purpose, index & 0xFFFFFFFF, index >> 32], dtype=np.uint32)
    blocks = []
    for b in range(3):
        out = np.zeros(16, dtype=np.uint32)
        lib().or_chacha20_block(P(key, _u32p), b, P(nonce, _u32p), P(out, _u32p))
        blocks.append(out.astype("<u4").tobytes())
    stream = b"".join(blocks)
    assert w.astype("<u8").tobytes() == stream[:160]
    w2 = np.zeros(5, dtype=np.uint64)
    lib().or_stream_words(seed, purpose, index, 13, 5, P(w2))
    assert np.array_equal(w2, w[13:18])


def test_gaussian_sampler_statistics(tiny):
    n = 1 << 20
    e = np.zeros(n, dtype=np.int8)
    lib().or_sample_gauss(tiny.h, 99, 3, 0, n, P(e, _i8p))
    x = e.astype(np.float64)
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 3.2 ** 2) < 0.1            # sigma = 3.2
    assert np.abs(e).max() <= 19                    # tail cut at 6 sigma
    # symmetric and unimodal
    h = np.bincount(np.abs(e).astype(np.int64), minlength=20)
    assert all(h[i] >= h[i + 1] for i in range(1, 12))
    assert abs((e > 0).mean() - (e < 0).mean()) < 0.005
    # P(|e| = 0) of a discretised N(0, 3.2^2) is about 0.1247
    assert abs((e == 0).mean() - 0.1247) < 0.004
    # CDT shape
    t = np.zeros(64, dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint32)
    assert lib().or_cdt_table(tiny.h, P(t), 64, P(cnt, _u32p)) == 0
    T = [int(v) for v in t[:int(cnt[0])]]
    assert len(T) == 20 and T[-1] == 1 << 63 and all(a < b for a, b in zip(T, T[1:]))


def test_cdt_thresholds_against_exact_discretised_normal(tiny):
    """The CDT thresholds T_k = floor(S_k / S_19 * 2^63), S_k = sum over |x| <= k of
    exp(-x^2 / (2 sigma^2)), evaluated in 200-bit arithmetic.  The oracle (like the library)
    sums in double with libm exp, so its T_k may differ from the exact value in the low
    bits: relative error of S_k / S_19 at most about 40 roundings of 2^-53, i.e. below 2^16
    in absolute terms after the 2^63 scaling.  A wrong sigma, tail cut, missing factor 2
    or shifted index moves a threshold by far more than that."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    sigma = mpmath.mpf("3.2")
    B = int(mpmath.floor(6 * sigma))
    assert B == 19
    rho = [mpmath.exp(-mpmath.mpf(x) ** 2 / (2 * sigma ** 2)) for x in range(B + 1)]
    S = [rho[0] + 2 * sum(rho[1:k + 1]) for k in range(B + 1)]
    exact = [int(mpmath.floor(S[k] / S[B] * mpmath.mpf(2) ** 63)) for k in range(B)] + [1 << 63]
    t = np.zeros(64, dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint32)
    assert lib().or_cdt_table(tiny.h, P(t), 64, P(cnt, _u32p)) == 0
    T = [int(v) for v in t[:int(cnt[0])]]
    assert len(T) == B + 1
    diffs = [abs(a - b) for a, b in zip(T, exact)]
    assert max(diffs) < 1 << 16, diffs
    # the first threshold is P(e = 0) = 1 / S_19 (about 0.1247 of 2^63)
    assert abs(T[0] / 2.0 ** 63 - 0.12467) < 1e-4


def test_ternary_and_uniform_samplers():
    n = 300000
    s = np.zeros(n, dtype=np.int8)
    lib().or_sample_ternary(5, 1, 0, n, P(s, _i8p))
    for v in (-1, 0, 1):
        assert abs((s == v).mean() - 1 / 3) < 0.005
    q = (1 << 59) + 123
    u = np.zeros(n, dtype=np.uint64)
    lib().or_sample_uniform(5, 2, 1, q, n, P(u))
    assert int(u.max()) < q
    frac = u.astype(np.float64) / q
    hist = np.histogram(frac, bins=10, range=(0, 1))[0] / n
    assert np.all(np.abs(hist - 0.1) < 0.005)
    # uniform value = (w_{2k+1} 2^64 + w_{2k}) mod q
    w = np.zeros(8, dtype=np.uint64)
    lib().or_stream_words(5, 2, 1, 0, 8, P(w))
    for k in range(4):
        assert int(u[k]) == ((int(w[2 * k + 1]) << 64) | int(w[2 * k])) % q


# ----------------------------------------------------------------- encoding
def test_dd_cossin_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    for M in (8, 64, 1 << 16):
        for m in list(range(0, 9)) + [M // 8 - 1, M // 8, M // 8 + 1, M // 4, M // 2 + 3, M - 1, 12345 % M]:
            ch, cl, sh, sl = (np.zeros(1) for _ in range(4))
            lib().or_dd_cossin(m, M, P(ch, _dp), P(cl, _dp), P(sh, _dp), P(sl, _dp))
            ang = 2 * mp.pi * m / M
            assert abs(mp.mpf(float(ch[0])) + mp.mpf(float(cl[0])) - mp.cos(ang)) < mp.mpf(2) ** -100
            assert abs(mp.mpf(float(sh[0])) + mp.mpf(float(sl[0])) - mp.sin(ang)) < mp.mpf(2) ** -100


def test_encode_exact_vs_definition(tiny):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    n = tiny.n
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, n // 2)
    scale = 2.0 ** 40
    m, ties = tiny.encode(z, scale)
    assert ties == 0
    t = [pow(5, j, 2 * n) for j in range(n // 2)]
    for k in range(n):
        s = mp.mpf(0)
        for j in range(n // 2):
            s += mp.mpf(float(z[j])) * mp.cos(mp.pi * ((t[j] * k) % (2 * n)) / n)
        v = s * 2 / n * mp.mpf(scale)
        r = int(mp.floor(v + mp.mpf(0.5))) if v >= 0 else -int(mp.floor(-v + mp.mpf(0.5)))
        assert int(m[k]) == r


def test_encode_decode_and_rotation_direction():
    o = O.Oracle(10, [50], [50], 3.2)
    n = o.n
    rng = np.random.default_rng(12)
    z = rng.uniform(-1, 1, n // 2)
    m, _ = o.encode(z, 2.0 ** 40)
    back = o.decode([int(x) for x in m], 2.0 ** 40)
    assert np.max(np.abs(back - z)) < 1e-9
    # sigma_{5^r} on the coefficients rotates the slots LEFT by r
    for r in (1, 3, n // 2 - 1):
        g = pow(5, r, 2 * n)
        rot = [0] * n
        for k in range(n):
            e = k * g % (2 * n)
            if e < n:
                rot[e] = int(m[k])
            else:
                rot[e - n] = -int(m[k])
        zr = o.decode(rot, 2.0 ** 40)
        assert np.max(np.abs(zr - np.roll(z, -r))) < 1e-9


# ----------------------------------------------------------------- encryption
def _small_poly(fn, *args, n):
    out = np.zeros(n, dtype=np.int8)
    fn(*args, n, P(out, _i8p))
    return [int(x) for x in out]


def test_encryption_noise_identity():
    o = O.Oracle(5, [40, 35], [41], 3.2)
    n = o.n
    seed, ct_id = 77, 4
    keys = o.keygen(seed, [], relin=False)
    rng = np.random.default_rng(5)
    m = rng.integers(-(1 << 20), 1 << 20, n).astype(np.int64)
    ct = o.encrypt_m(keys.pk, m, seed, ct_id, 1.0)
    res = o.decrypt_residues(keys, ct)
    got = [centre(x, Q) for x, Q in [(v, crt(res, o.q)[1]) for v in crt(res, o.q)[0]]]
    s = _small_poly(lib().or_sample_ternary, seed, O.P_SK, 0, n=n)
    e = _small_poly(lambda *a: lib().or_sample_gauss(o.h, *a), seed, O.P_PK_E, 0, n=n)
    v = _small_poly(lib().or_sample_ternary, seed, O.P_ENC_V, ct_id, n=n)
    e0 = _small_poly(lambda *a: lib().or_sample_gauss(o.h, *a), seed, O.P_ENC_E0, ct_id, n=n)
    e1 = _small_poly(lambda *a: lib().or_sample_gauss(o.h, *a), seed, O.P_ENC_E1, ct_id, n=n)
    assert s == [int(x) for x in keys.s]
    ve = negacyclic_schoolbook(v, e, 0)
    e1s = negacyclic_schoolbook(e1, s, 0)
    want = [int(m[k]) + ve[k] + e0[k] + e1s[k] for k in range(n)]
    assert got == want


# ----------------------------------------------------------------- automorphism
def test_automorphism_identities(tiny):
    n = tiny.n
    rng = np.random.default_rng(6)
    pr = np.array([0], dtype=np.uint32)
    q = tiny.primes[0]

    def auto(a, g):
        out = np.zeros_like(a)
        lib().or_automorphism_coeff(tiny.h, 1, P(pr, _u32p), g, P(a), P(out))
        return out

    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    for g, h in ((5, 25), (2 * n - 1, 5), (pow(5, 7, 2 * n), 3)):
        ab = np.array(negacyclic_schoolbook(a, b, q), dtype=np.uint64)
        lhs = auto(ab, g)
        rhs = np.array(negacyclic_schoolbook(auto(a, g), auto(b, g), q), dtype=np.uint64)
        assert np.array_equal(lhs, rhs)
        assert np.array_equal(auto(auto(a, h), g), auto(a, g * h % (2 * n)))
        A = tiny.ntt_fwd(a[None], [0])
        out = np.zeros_like(A)
        lib().or_automorphism_ntt(tiny.h, 1, g, P(A), P(out))
        assert np.array_equal(out, tiny.ntt_fwd(auto(a, g)[None], [0]))


# ----------------------------------------------------------------- basis conversion, rescale, key switch
@pytest.fixture(scope="module")
def hybrid():
    # K = alpha = 2 special primes, 5 ciphertext primes -> digits {0,1},{2,3},{4}
    return O.Oracle(6, [45, 30, 30, 30, 30], [45, 45], 3.2)


def _rand_level_poly(o, level, rng):
    return np.stack([rng.integers(0, q, o.n, dtype=np.uint64) for q in o.q[:level + 1]])


def test_modup_closed_form(hybrid):
    o = hybrid
    rng = np.random.default_rng(8)
    for level in (4, 3, 0):
        a = _rand_level_poly(o, level, rng)
        d = o.ntt_fwd(a, list(range(level + 1)))
        ext = o.modup(level, d)
        W = level + 1 + o.n_p
        prime_of = list(range(level + 1)) + [o.n_q + k for k in range(o.n_p)]
        for j in range(o.dnum(level)):
            lo, hi = 2 * j, min(2 * j + 2, level + 1)
            qs = o.q[lo:hi]
            A, Qj = crt(a[lo:hi], qs)
            coeff = o.ntt_inv(ext[j], prime_of)
            for t in range(W):
                pt = o.primes[prime_of[t]]
                for k in range(o.n):
                    diff = (int(coeff[t][k]) - A[k]) % pt
                    # Conv(a) = a + u Q_j with 0 <= u < alpha
                    assert any(diff == (u * Qj) % pt for u in range(hi - lo)), (level, j, t, k)


def test_moddown_closed_form(hybrid):
    o = hybrid
    rng = np.random.default_rng(9)
    level = 3
    prime_of = list(range(level + 1)) + [o.n_q + k for k in range(o.n_p)]
    x = np.stack([rng.integers(0, o.primes[p], o.n, dtype=np.uint64) for p in prime_of])
    X, QP = crt(x, [o.primes[p] for p in prime_of])
    out = o.moddown(level, o.ntt_fwd(x, prime_of))
    out = o.ntt_inv(out, list(range(level + 1)))
    Pp = o.p[0] * o.p[1]
    for i in range(level + 1):
        q = o.q[i]
        for k in range(o.n):
            fl = X[k] // Pp
            # (x - Conv_P(x_P)) / P = floor(x / P) - u, 0 <= u < K
            assert any(int(out[i][k]) == (fl - u) % q for u in range(o.n_p))


def test_rescale_closed_form(hybrid):
    o = hybrid
    rng = np.random.default_rng(10)
    level = 4
    a = _rand_level_poly(o, level, rng)
    X, Q = crt(a, o.q[:level + 1])
    ct = O.Ct(o.ntt_fwd(a, list(range(level + 1)))[None], level, 1.0)
    r = o.ntt_inv(o.rescale(ct).data[0], list(range(level)))
    ql = o.q[level]
    for k in range(o.n):
        rem = X[k] % ql
        if rem > (ql - 1) // 2:
            rem -= ql
        want = (X[k] - rem) // ql           # round(X / q_l), half-way cases away from +inf
        for i in range(level):
            assert int(r[i][k]) == want % o.q[i]


def test_keyswitch_error_bound(hybrid):
    o = hybrid
    n = o.n
    seed = 123
    g = pow(5, 3, 2 * n)
    keys = o.keygen(seed, [g])
    rng = np.random.default_rng(13)
    s = [int(v) for v in keys.s]
    sg = [0] * n
    for k in range(n):
        e = k * g % (2 * n)
        if e < n:
            sg[e] = s[k]
        else:
            sg[e - n] = -s[k]
    s2 = negacyclic_schoolbook(s, s, 0)
    for level in (4, 2):
        qs = o.q[:level + 1]
        a = _rand_level_poly(o, level, rng)
        d = o.ntt_fwd(a, list(range(level + 1)))
        for swk, target in ((keys.relin, s2), (keys.rot[g], sg)):
            u0, u1 = o.keyswitch(level, d, swk, 1)
            u0 = o.ntt_inv(u0, list(range(level + 1)))
            u1 = o.ntt_inv(u1, list(range(level + 1)))
            U0, Q = crt(u0, qs)
            U1, _ = crt(u1, qs)
            D, _ = crt(a, qs)
            u1s = negacyclic_schoolbook(U1, s, 0)
            dt = negacyclic_schoolbook(D, target, 0)
            err = [abs(centre((U0[k] + u1s[k] - dt[k]) % Q, Q)) for k in range(n)]
            Pp = o.p[0] * o.p[1]
            max_digit = max(o.q[2 * j] * (o.q[2 * j + 1] if 2 * j + 1 <= level else 1)
                            for j in range(o.dnum(level)))
            bound = o.dnum(level) * 2 * max_digit * n * 19 // Pp + o.n_p * (n + 1) + 1
            assert max(err) <= bound, (level, max(err), bound)
            assert max(err) > 0


# ----------------------------------------------------------------- composed operations
@pytest.fixture(scope="module")
def mid():
    o = O.Oracle(10, [50, 40, 40, 40], [50], 3.2)
    return o


def test_rotation_and_hoisting_decrypt(mid):
    o = mid
    rng = np.random.default_rng(14)
    z = rng.uniform(-1, 1, o.n // 2)
    steps = [1, 2, 7, o.n // 2 - 3]
    keys = o.keygen(55, [O.galois_for_step(s, o.n) for s in steps])
    ct = o.encrypt(keys.pk, z, 55, 0, 2.0 ** 40)
    outs = o.rotate_hoisted(ct, steps, keys)
    for st, r in zip(steps, outs):
        assert np.max(np.abs(o.decrypt(keys, r) - np.roll(z, -st))) < 1e-6
    # rho^a o rho^b = rho^(a+b) on decrypted slots
    r12 = o.rotate(o.rotate(ct, 1, keys), 2, keys)
    assert np.max(np.abs(o.decrypt(keys, r12) - np.roll(z, -3))) < 1e-6


def test_multiplication_decrypts_to_product(mid):
    o = mid
    rng = np.random.default_rng(15)
    a = rng.uniform(-1, 1, o.n // 2)
    b = rng.uniform(-1, 1, o.n // 2)
    keys = o.keygen(56, [])
    ca = o.encrypt(keys.pk, a, 56, 0, 2.0 ** 40)
    cb = o.encrypt(keys.pk, b, 56, 1, 2.0 ** 40)
    prod = o.mul_relin_rescale(ca, cb, keys)
    assert prod.level == o.L - 1
    assert prod.scale == 2.0 ** 80 / o.q[o.L]
    assert np.max(np.abs(o.decrypt(keys, prod) - a * b)) < 1e-6


def test_bsgs_plan_rule():
    assert O.bsgs_split(128) == (16, 8)
    assert O.bsgs_split(512) == (32, 16)
    assert O.bsgs_split(2) == (2, 1)
    assert O.bsgs_split(16) == (4, 4)
    assert O.bsgs_split(32) == (8, 4)
    assert O.bsgs_split(1) == (1, 1)


def test_bsgs_matches_fp64_and_full_step(mid):
    o = mid
    rng = np.random.default_rng(16)
    d_in, d_out = 64, 16
    k = (o.n // 2) // d_in
    W = rng.normal(0, 0.2, (d_out, d_in))
    x = rng.uniform(-1, 1, d_in)
    z, kk = O.pack_clips(x[None], o.n // 2)
    assert kk == k
    steps = O.rotation_steps([("fc", W)], d_in, k) + [i * k for i in range(1, d_out)]
    keys = o.keygen(57, [O.galois_for_step(s, o.n) for s in sorted(set(steps))])
    ct = o.encrypt(keys.pk, z, 57, 0, 2.0 ** 40)
    out = o.fc(ct, W, k, keys)
    dec = o.decrypt(keys, out)
    y = W @ x
    M = o.n // 2 // k
    got = dec.reshape(M, k)[:, 0]
    assert np.max(np.abs(got - np.tile(y, M // d_out))) < 1e-6
    # full-step: sum_i diag_i * rho^i(x), then rotate-and-sum, all rotations unhoisted
    ql = float(o.q[ct.level])
    acc = None
    for i in range(d_out):
        xi = ct if i == 0 else o.rotate(ct, i * k, keys)
        pt = o.encode_pt(o.expand(o.diag_vector(W, i, M), k), ql, ct.level)
        pr = o.mulplain(xi, pt, ql)
        acc = pr if acc is None else o.add(acc, pr)
    acc = o.rescale(acc)
    s = d_out
    while s < d_in:
        acc = o.add(acc, o.rotate(acc, s * k, keys))
        s *= 2
    full = o.decrypt(keys, acc).reshape(M, k)[:, 0]
    assert np.max(np.abs(full - got)) < 1e-6


def test_toy_network_within_bound():
    from paper_2104_09164_gb300.workloads import make_workload
    w = make_workload("toy")
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
    z, k = O.pack_clips(w.clips, w.slots)
    steps = O.rotation_steps(w.layers, w.clip_dim, k)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
    ct = o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale)
    out = o.evaluate(w.layers, ct, k, keys)
    dec = o.decrypt(keys, out)
    logits = np.array([dec[p * k] for p in O.output_positions(w.layers)])
    assert np.max(np.abs(logits - w.fp64_forward(w.clips)[0])) <= 2.0 ** -15


def test_rotsum_radix_folds_the_same_sum():
    """the hoisted rotate-and-sum rounds of any radix decrypt to sum_j rho^(j*step*k)(z)"""
    from oracle import oracle as O
    o = O.Oracle(12, [50, 40, 40], [50], 3.2)
    S = o.n // 2
    k = 4
    steps = set()
    for radix in (2, 4, 16):
        steps.update(s * k for s in O.rotsum_steps(8, 16, radix))
    keys = o.keygen(7, [O.galois_for_step(s, o.n) for s in steps])
    z = np.random.default_rng(3).uniform(-1, 1, S)
    ct = o.encrypt(keys.pk, z, 11, 0, 2.0 ** 40)
    want = sum(np.roll(z, -j * 8 * k) for j in range(16))
    for radix in (2, 4, 16):
        got = o.decrypt(keys, o.rotsum(ct, 8, 16, k, keys, radix))
        assert np.max(np.abs(got - want)) < 2.0 ** -20, radix
    assert O.rotsum_steps(8, 16, 4) == [8, 16, 24, 32, 64, 96]
    assert O.rotsum_steps(1, 64, 16) == list(range(1, 16)) + [16, 32, 48]


def test_hoisted_moddown_fc_matches_plain_product():
    """the FC with baby steps kept over Q_l u P and one ModDown per giant-step sum decrypts
    to W x (and agrees with the per-rotation ModDown form), for several baby-step counts;
    the P-lift of the identity and the extended products are exact identities"""
    from oracle import oracle as O
    o = O.Oracle(12, [50, 40, 40], [50], 3.2)
    S = o.n // 2
    rng = np.random.default_rng(8)
    k = 16
    M = S // k
    W = rng.normal(0, 0.1, size=(16, M))
    steps = set()
    for n1 in (2, 4, 16):
        steps.update(O.rotation_steps([("fc", W)], M, k, 2, n1))
    keys = o.keygen(9, [O.galois_for_step(s, o.n) for s in steps])
    x = rng.uniform(-1, 1, M)
    ct = o.encrypt(keys.pk, np.repeat(x, k), 12, 0, 2.0 ** 40)
    want = np.repeat(W @ x, 1)
    for n1 in (2, 4, 16):
        r_dh = o.fc(ct, W, k, keys, radix=2, n1=n1, dh=True)
        r_std = o.fc(ct, W, k, keys, radix=2, n1=n1, dh=False)
        got_dh = o.decrypt(keys, r_dh)[::k][:16]
        got_std = o.decrypt(keys, r_std)[::k][:16]
        assert np.max(np.abs(got_dh - want)) < 2.0 ** -20, n1
        assert np.max(np.abs(got_dh - got_std)) < 2.0 ** -20, n1
        assert r_dh.level == r_std.level and r_dh.scale == r_std.scale
    # ModDown(P x lifted) = x exactly
    lifted = o.scale_p_ext(ct)
    back = np.stack([o.moddown(ct.level, lifted[p]) for p in range(2)])
    assert np.array_equal(back, ct.data)


def test_hoisted_sums_fc_and_rotsum():
    """hoisted sums (one ModDown per giant-step sum and per rotate-and-sum round, the
    rotations kept over Q_l u P): with one rotation per round and at most two giant steps it
    is bit-identical to the per-rotation ModDown form (ModDown(P a + b) = a + ModDown(b)
    exactly); with more rotations per sum it differs only by ModDown rounding and still
    decrypts to W x, with and without hoisted ModDown of the babies"""
    from oracle import oracle as O
    o = O.Oracle(12, [50, 40, 40], [50], 3.2)
    S = o.n // 2
    rng = np.random.default_rng(18)
    k = 16
    M = S // k
    W = rng.normal(0, 0.1, size=(16, M))
    steps = set()
    for n1, radix in ((8, 2), (2, 8), (4, 8)):
        steps.update(O.rotation_steps([("fc", W)], M, k, radix, n1))
    keys = o.keygen(19, [O.galois_for_step(s, o.n) for s in steps])
    x = rng.uniform(-1, 1, M)
    ct = o.encrypt(keys.pk, np.repeat(x, k), 13, 0, 2.0 ** 40)
    want = W @ x
    # n1 = 8 of D = 16: two giant steps; radix 2: one rotation per round
    a = o.fc(ct, W, k, keys, radix=2, n1=8, hs=True)
    b = o.fc(ct, W, k, keys, radix=2, n1=8, hs=False)
    assert np.array_equal(a.data, b.data) and a.scale == b.scale
    for n1, radix, dh in ((2, 8, False), (4, 8, True), (2, 8, True)):
        r_hs = o.fc(ct, W, k, keys, radix=radix, n1=n1, dh=dh, hs=True)
        r = o.fc(ct, W, k, keys, radix=radix, n1=n1, dh=dh, hs=False)
        assert r_hs.level == r.level and r_hs.scale == r.scale
        assert not np.array_equal(r_hs.data, r.data), (n1, radix, dh)
        got = o.decrypt(keys, r_hs)[::k][:16]
        assert np.max(np.abs(got - want)) < 2.0 ** -20, (n1, radix, dh)
        assert np.max(np.abs(got - o.decrypt(keys, r)[::k][:16])) < 2.0 ** -20


def test_fc_bias_is_added_after_the_rotate_and_sum():
    """an FC layer with bias decrypts to W x + b in every replicated position (the bias is
    not multiplied by the rotate-and-sum's copy count); the residues differ from the bias-free
    layer by exactly the encoded bias plaintext"""
    from oracle import oracle as O
    o = O.Oracle(12, [50, 40, 40], [50], 3.2)
    S = o.n // 2
    rng = np.random.default_rng(28)
    k = 16
    M = S // k
    W = rng.normal(0, 0.1, size=(16, M))
    b = rng.normal(0, 0.3, 16)
    keys = o.keygen(29, [O.galois_for_step(s, o.n) for s in O.rotation_steps([("fc", W)], M, k)])
    x = rng.uniform(-1, 1, M)
    ct = o.encrypt(keys.pk, np.repeat(x, k), 14, 0, 2.0 ** 40)
    r_b = o.fc(ct, W, k, keys, bias=b)
    r = o.fc(ct, W, k, keys)
    got = o.decrypt(keys, r_b)
    want = np.repeat((W @ x + b)[np.arange(M) % 16], k)
    assert np.max(np.abs(got - want)) < 2.0 ** -20
    pt = o.encode_pt(o.expand(b[np.arange(M) % 16], k), r.scale, r.level)
    assert np.array_equal(r_b.data, o.add_plain(r, pt).data) and r_b.scale == r.scale
