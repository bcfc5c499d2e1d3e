"""Hoisted sums (hear_model_opts.hoist_sums): the giant-step rotations of every FC layer
and every rotate-and-sum round are summed over Q_l u P and ModDowned once.  Bit-exact
against the oracle evaluating the same form (toy network with its collapsed
FC -> x^2 -> FC, small and large networks, with and without hoisted ModDown of the babies),
logits within 2^-15 of FP64."""
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


@pytest.mark.parametrize("name,n1,dh,n_clips", [("toy", None, False, None), ("small", None, False, 8),
                                                ("small", 32, True, 8), ("large", 64, True, 16)])
def test_hoisted_sums_bit_exact(H, name, n1, dh, n_clips):
    w = make_workload(name, n_clips)
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        model = H.hear_model_create(ctx, w.layers, w.clip_dim, fc_n1=n1, hoist_moddown=dh, hoist_sums=True)
        k = w.slots // w.clip_dim
        steps = H.hear_model_rotations(model)
        assert steps == O.rotation_steps(w.layers, w.clip_dim, k, O.ROTSUM_RADIX, n1)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        cts = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(w.n_ct)]
        outs = H.hear_evaluate(model, evk, cts)
        pos = H.hear_model_output_positions(model)
        ref = w.fp64_forward(w.clips)
        for i, o in enumerate(outs):
            dec = H.hear_decrypt(ctx, sk, o)
            for c, clip in enumerate(range(i * w.clips_per_ct, min((i + 1) * w.clips_per_ct, w.n_clips))):
                logits = np.array([dec[p * k + c] for p in pos])
                assert np.max(np.abs(logits - ref[clip])) <= 2.0 ** -15
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        i = w.n_ct - 1
        z, kk = O.pack_clips(w.ct_clips(i), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, i, 2.0 ** w.log2_scale), kk, keys, n1=n1, dh=dh, hs=True)
        assert H.hear_ciphertext_info(outs[i])[2] == r.scale
        assert np.array_equal(H.hear_ciphertext_export(outs[i]), o.to_coeff(r))
        for h in cts + outs:
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
