"""Rotate-and-sum in hoisted rounds of r - 1 rotations (hear_model_opts.rotsum_radix):
bit-exact against the oracle folding the same rounds, for the small network (FC 2048->128:
16 copies; FC 128->2: 64 copies) and the collapsed toy network, at radix 4 and 16."""
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


@pytest.mark.parametrize("name,radix", [("small", 4), ("small", 16), ("toy", 8)])
def test_rotsum_radix_bit_exact(H, name, radix):
    w = make_workload(name)
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        model = H.hear_model_create(ctx, w.layers, w.clip_dim, rotsum_radix=radix)
        k = w.slots // w.clip_dim
        steps = H.hear_model_rotations(model)
        assert steps == O.rotation_steps(w.layers, w.clip_dim, k, radix)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
        out = H.hear_evaluate(model, evk, [ct])[0]
        pos = H.hear_model_output_positions(model)
        dec = H.hear_decrypt(ctx, sk, out)
        logits = np.array([dec[p * k] for p in pos])
        assert np.max(np.abs(logits - w.fp64_forward(w.clips)[0])) <= 2.0 ** -15
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(0), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale), kk, keys, radix=radix)
        assert np.array_equal(H.hear_ciphertext_export(out), o.to_coeff(r))
        for h in (ct, out):
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
