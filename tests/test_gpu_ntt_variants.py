"""The three NTT launch forms (two-pass wide, two-pass narrow, one-launch cluster) give the
same transform: ring products against the oracle's NTT product for every prime, inverse o
forward = identity on small and large launches, and a whole encrypted network bit-exact
against the oracle under each forced form and after the tuner has picked its table."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

SETS = [(12, [50, 40, 40], [50]), (14, [60] + [40] * 7, [60]), (15, [60] + [40] * 14, [60, 60])]


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


@pytest.mark.parametrize("log_n,qb,pb", SETS)
def test_variants_compute_the_same_transform(H, log_n, qb, pb):
    ctx = H.hear_context_create(log_n, qb, pb, 40.0, 3.2, 0)
    o = O.Oracle(log_n, qb, pb, 3.2)
    n = 1 << log_n
    rng = np.random.default_rng(log_n)
    try:
        for pi in (0, 1, len(qb) - 1, len(qb)):
            q = o.primes[pi]
            a = rng.integers(0, q, n, dtype=np.uint64)
            b = rng.integers(0, q, n, dtype=np.uint64)
            A, B = o.ntt_fwd(a[None], [pi]), o.ntt_fwd(b[None], [pi])
            C = np.array([int(x) * int(y) % q for x, y in zip(A[0], B[0])], dtype=np.uint64)
            want = o.ntt_inv(C[None], [pi])[0]
            for v in (H.HEAR_NTT_WIDE, H.HEAR_NTT_NARROW, H.HEAR_NTT_FUSED, H.HEAR_NTT_TINY):
                H.hear_ntt_set_variant(ctx, v)
                assert np.array_equal(H.hear_dbg_poly_mul(ctx, pi, a, b), want), (pi, v)
        for n_limbs in (1, 7, 300):
            limbs = np.stack([rng.integers(0, o.primes[i % len(o.primes)], n, dtype=np.uint64)
                              for i in range(n_limbs)])
            for v in (H.HEAR_NTT_WIDE, H.HEAR_NTT_NARROW, H.HEAR_NTT_FUSED, H.HEAR_NTT_TINY):
                H.hear_ntt_set_variant(ctx, v)
                assert np.array_equal(H.hear_dbg_ntt_roundtrip(ctx, limbs), limbs), (n_limbs, v)
        H.hear_ntt_set_variant(ctx, -1)
        choice, ms = H.hear_ntt_tune(ctx, 64, 2)
        assert set(np.unique(choice)) <= {0, 1, 3}          # the one-launch form is timed, not chosen
        assert np.all(ms[:, :7, :] > 0)
    finally:
        H.hear_context_destroy(ctx)


@pytest.mark.parametrize("variant", ["wide", "narrow", "fused", "tiny", "tuned"])
def test_small_network_bit_exact_under_each_variant(H, variant):
    w = make_workload("small")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        if variant == "tuned":
            H.hear_ntt_tune(ctx, 128, 2)
        else:
            H.hear_ntt_set_variant(ctx, {"wide": 0, "narrow": 1, "fused": 2, "tiny": 3}[variant])
        model = H.hear_model_create(ctx, w.layers, w.clip_dim)
        steps = H.hear_model_rotations(model)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
        out = H.hear_evaluate(model, evk, [ct])[0]
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
        k = w.slots // w.clip_dim
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(0), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale), kk, keys)
        assert np.array_equal(H.hear_ciphertext_export(out), o.to_coeff(r))
        for h in (ct, out):
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
