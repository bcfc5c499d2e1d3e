"""FC layers with bias: the small network FC 2048->128 (+b1) -> x^2 -> FC 128->2 (+b2), in the
default FC form and in the tuned form (32 baby steps, hoisted ModDown and sums), on two
ciphertexts: bit-exact against the oracle, logits within 2^-15 of the FP64 network with the
biases (so the biases are added once, not once per rotate-and-sum copy)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


@pytest.mark.parametrize("n1,dh,hs", [(None, False, False), (32, True, True)])
def test_fc_bias_bit_exact(H, n1, dh, hs):
    w = make_workload("small", 8)
    rng = np.random.default_rng(41)
    (_, W1), sq, (_, W2) = w.layers
    layers = [("fc", W1, rng.normal(0, 0.05, W1.shape[0])), sq, ("fc", W2, rng.normal(0, 0.05, W2.shape[0]))]
    w.layers = layers
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        model = H.hear_model_create(ctx, layers, w.clip_dim, fc_n1=n1, hoist_moddown=dh, hoist_sums=hs)
        k = w.slots // w.clip_dim
        steps = H.hear_model_rotations(model)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        cts = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(w.n_ct)]
        outs = H.hear_evaluate(model, evk, cts)
        pos = H.hear_model_output_positions(model)
        ref = w.fp64_forward(w.clips)
        for i, o in enumerate(outs):
            dec = H.hear_decrypt(ctx, sk, o)
            for c, clip in enumerate(range(i * w.clips_per_ct, (i + 1) * w.clips_per_ct)):
                logits = np.array([dec[p * k + c] for p in pos])
                assert np.max(np.abs(logits - ref[clip])) <= 2.0 ** -15
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(1), w.slots)
        r = o.evaluate(layers, o.encrypt(keys.pk, z, 401, 1, 2.0 ** w.log2_scale), kk, keys, n1=n1, dh=dh, hs=hs)
        assert H.hear_ciphertext_info(outs[1])[2] == r.scale
        assert np.array_equal(H.hear_ciphertext_export(outs[1]), o.to_coeff(r))
        # the same network without biases gives other ciphertexts
        plain = H.hear_model_create(ctx, [("fc", W1), sq, ("fc", W2)], w.clip_dim, fc_n1=n1, hoist_moddown=dh,
                                    hoist_sums=hs)
        nb = H.hear_evaluate(plain, evk, cts[:1])[0]
        assert not np.array_equal(H.hear_ciphertext_export(nb), H.hear_ciphertext_export(outs[0]))
        H.hear_ciphertext_destroy(nb)
        H.hear_model_destroy(plain)
        with pytest.raises(ValueError):
            H.hear_model_create(ctx, [("fc", W1, np.zeros(3))], w.clip_dim)
        for h in cts + outs:
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
