"""The allocation-free rescale against the regular one.

hear_rescale_noalloc serves callers that cannot call cudaMalloc (a device-memory quota
already held by another allocator, a real-time loop that must not take the allocator's
locks or latency, a host that owns only host memory and a stream): it works in a fixed
device array inside the library.  Its output must equal hear_rescale's bit for bit, on
consecutive calls that reuse that array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def test_rescale_noalloc_equals_rescale(H):
    log_n, q_bits, p_bits = 14, [60] + [40] * 7, [60]
    ctx = H.hear_context_create(log_n, q_bits, p_bits, 40.0, 3.2, 0)
    sk, pk, evk = H.hear_keygen(ctx, 7, [])
    rng = np.random.default_rng(5)
    try:
        # two calls in a row with different inputs and levels: the shared array keeps the
        # previous call's contents, which must not leak into the next result
        cases = []
        for i, drop in enumerate((0, 3)):
            z = rng.uniform(-1, 1, (1 << log_n) // 2)
            ct = H.hear_encrypt(ctx, pk, z, 2.0 ** 40, 11, i)
            for _ in range(drop):
                nxt = H.hear_rescale(ct)
                H.hear_ciphertext_destroy(ct)
                ct = nxt
            cases.append(ct)
        for ct in cases:
            level, n_poly, _ = H.hear_ciphertext_info(ct)
            ref = H.hear_rescale(ct)
            want = H.hear_ciphertext_export(ref)
            got = H.hear_rescale_noalloc(ctx, H.hear_ciphertext_export(ct), level, n_poly)
            assert got.shape == want.shape
            assert np.array_equal(got, want)
            H.hear_ciphertext_destroy(ref)
        # a buffer whose size does not match n_poly * (level + 1) * N is refused before any
        # copy (the library reads and writes only what the sizes it is given allow)
        level, n_poly, _ = H.hear_ciphertext_info(cases[0])
        words = H.hear_ciphertext_export(cases[0]).reshape(-1)
        with pytest.raises(H.HearError) as e:
            H.hear_rescale_noalloc(ctx, words[: words.size // 2], level, n_poly, n=1 << log_n)
        assert e.value.code == H.HEAR_E_FORMAT
        with pytest.raises(H.HearError) as e:
            H.hear_rescale_noalloc(ctx, np.concatenate([words, words]), level, n_poly, n=1 << log_n)
        assert e.value.code == H.HEAR_E_FORMAT
        # a residue that is not reduced mod its limb's prime is refused too
        primes = H.hear_context_primes(ctx)
        bad = words.copy()
        bad[3 << log_n] = np.uint64(primes[3])
        with pytest.raises(H.HearError) as e:
            H.hear_rescale_noalloc(ctx, bad, level, n_poly)
        assert e.value.code == H.HEAR_E_FORMAT
        # and the array still serves a correct call after the refusals
        ref = H.hear_rescale(cases[0])
        assert np.array_equal(H.hear_rescale_noalloc(ctx, words, level, n_poly), H.hear_ciphertext_export(ref))
        H.hear_ciphertext_destroy(ref)
        # a level-0 ciphertext has no prime left to divide by
        with pytest.raises(H.HearError) as e:
            H.hear_rescale_noalloc(ctx, np.zeros(2 << log_n, dtype=np.uint64), 0, 2)
        assert e.value.code == -4
        # sizes beyond the fixed array are refused with a clear error, not truncated
        big_ctx = H.hear_context_create(16, [50] * 12, [50], 40.0, 3.2, 0)
        try:
            big = np.zeros(3 * 12 * (1 << 16), dtype=np.uint64)
            with pytest.raises(H.HearError) as e:
                H.hear_rescale_noalloc(big_ctx, big, 11, 3)
            assert e.value.code == -9 and "exceeds" in str(e.value)
        finally:
            H.hear_context_destroy(big_ctx)
    finally:
        for ct in cases:
            H.hear_ciphertext_destroy(ct)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
        H.hear_context_destroy(ctx)
