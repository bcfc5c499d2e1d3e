"""Minimal-start-level evaluation: ciphertexts dropped (no division) to the level the
network's depth needs and a model whose plaintexts carry only the limbs of each level of
use.  Bit-exact against the oracle evaluating the same dropped ciphertext; logits within
2^-15 of FP64."""
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


def test_drop_level_keeps_the_lower_residues(H):
    w = make_workload("small")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        sk, pk, evk = H.hear_keygen(ctx, 301, [])
        ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
        d = H.hear_ciphertext_drop_level(ct, 3)
        assert H.hear_ciphertext_info(d) == (3, 2, H.hear_ciphertext_info(ct)[2])
        full = H.hear_ciphertext_export(ct).reshape(2, len(w.q_bits), -1)
        assert np.array_equal(H.hear_ciphertext_export(d).reshape(2, 4, -1), full[:, :4])
        with pytest.raises(H.HearError):
            H.hear_ciphertext_drop_level(d, 5)
        for h in (ct, d):
            H.hear_ciphertext_destroy(h)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)


@pytest.mark.parametrize("name,level,n_ct", [("small", 3, 1), ("large", 5, 2)])
def test_network_from_minimal_level_bit_exact(H, name, level, n_ct):
    w = make_workload(name, n_clips=None if name == "small" else 16)
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        model = H.hear_model_create(ctx, w.layers, w.clip_dim, level)
        assert H.hear_model_levels(model) == (level, 0)
        steps = H.hear_model_rotations(model)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        top = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(n_ct)]
        cts = [H.hear_ciphertext_drop_level(c, level) for c in top]
        outs = H.hear_evaluate(model, evk, cts)
        pos = H.hear_model_output_positions(model)
        k = w.slots // w.clip_dim
        ref = w.fp64_forward(w.clips)
        for i, o in enumerate(outs):
            dec = H.hear_decrypt(ctx, sk, o)
            for c, clip in enumerate(range(i * w.clips_per_ct, min((i + 1) * w.clips_per_ct, w.n_clips))):
                logits = np.array([dec[p * k + c] for p in pos])
                assert np.max(np.abs(logits - ref[clip])) <= LOGIT_TOL
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(n_ct - 1), w.slots)
        x = o.encrypt(keys.pk, z, 401, n_ct - 1, 2.0 ** w.log2_scale)
        while x.level > level:
            x = o.drop_level(x)
        r = o.evaluate(w.layers, x, kk, keys)
        assert H.hear_ciphertext_info(outs[-1])[2] == r.scale
        assert np.array_equal(H.hear_ciphertext_export(outs[-1]), o.to_coeff(r))
        for h in top + cts + outs:
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
