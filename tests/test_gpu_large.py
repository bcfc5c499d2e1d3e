"""Full-size parity of the large network (N = 2^15, 15 ciphertext primes, 2 special primes,
256 clips packed 8 per ciphertext) in the launch configuration bench.py times: all 32
ciphertexts evaluated in one batch through the C ABI.  The oracle recomputes sampled
outputs (the first and the last ciphertext) limb by limb; every clip's logits are checked
against the FP64 network."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

LOGIT_TOL = 2.0 ** -15


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def test_large_network_batch_bit_exact_samples(H):
    w = make_workload("large")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    model = H.hear_model_create(ctx, w.layers, w.clip_dim)
    steps = H.hear_model_rotations(model)
    k = w.slots // w.clip_dim
    assert steps == O.rotation_steps(w.layers, w.clip_dim, k)
    sk, pk, evk = H.hear_keygen(ctx, 301, steps)
    cts = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(w.n_ct)]
    outs = H.hear_evaluate(model, evk, cts)
    pos = H.hear_model_output_positions(model)
    ref = w.fp64_forward(w.clips)
    worst = 0.0
    for i, o in enumerate(outs):
        dec = H.hear_decrypt(ctx, sk, o)
        for c, clip in enumerate(range(i * w.clips_per_ct, (i + 1) * w.clips_per_ct)):
            logits = np.array([dec[p * k + c] for p in pos])
            worst = max(worst, float(np.max(np.abs(logits - ref[clip]))))
    assert worst <= LOGIT_TOL, worst

    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
    for i in (0, w.n_ct - 1):
        z, kk = O.pack_clips(w.ct_clips(i), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, i, 2.0 ** w.log2_scale), kk, keys)
        got = H.hear_ciphertext_export(outs[i])
        assert H.hear_ciphertext_info(outs[i])[:2] == (r.level, 2)
        assert H.hear_ciphertext_info(outs[i])[2] == r.scale
        assert np.array_equal(got, o.to_coeff(r)), i
    for h in cts + outs:
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)
    H.hear_eval_keys_destroy(evk)
    H.hear_public_key_destroy(pk)
    H.hear_secret_key_destroy(sk)
    H.hear_context_destroy(ctx)


def test_small_network_batch_of_128_clips_sampled(H):
    """the batched small-network launch bench.py times (128 clips, 32 ciphertexts in one
    graph replay): sampled ciphertexts bit-exact, every clip's logits within 2^-15"""
    w = make_workload("small", 128)
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    model = H.hear_model_create(ctx, w.layers, w.clip_dim)
    steps = H.hear_model_rotations(model)
    k = w.slots // w.clip_dim
    sk, pk, evk = H.hear_keygen(ctx, 301, steps)
    cts = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(w.n_ct)]
    outs = H.hear_evaluate(model, evk, cts)
    pos = H.hear_model_output_positions(model)
    ref = w.fp64_forward(w.clips)
    worst = 0.0
    for i, o in enumerate(outs):
        dec = H.hear_decrypt(ctx, sk, o)
        for c, clip in enumerate(range(i * w.clips_per_ct, (i + 1) * w.clips_per_ct)):
            logits = np.array([dec[p * k + c] for p in pos])
            worst = max(worst, float(np.max(np.abs(logits - ref[clip]))))
    assert worst <= LOGIT_TOL, worst
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
    for i in (0, w.n_ct - 1):
        z, kk = O.pack_clips(w.ct_clips(i), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, i, 2.0 ** w.log2_scale), kk, keys)
        assert np.array_equal(H.hear_ciphertext_export(outs[i]), o.to_coeff(r)), i
    for h in cts + outs:
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)
    H.hear_eval_keys_destroy(evk)
    H.hear_public_key_destroy(pk)
    H.hear_secret_key_destroy(sk)
    H.hear_context_destroy(ctx)
