"""FC evaluation-form tuner (autotune.tune_fc): it times every candidate form through the C
ABI, the candidates include the default form, and the chosen form's network is bit-exact
against the oracle evaluating the same form."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.autotune import fc_candidates, tune_fc
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def test_tuned_fc_form_bit_exact(H):
    import torch
    w = make_workload("small")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        st = torch.cuda.Stream()
        (n1, dh, hs), report = tune_fc(H, ctx, w.layers, w.clip_dim, w.n_ct, w.slots, steps=2, stream=st)
        assert [(r["fc_n1"], r["hoist_moddown"], r["hoist_sums"]) for r in report] == fc_candidates(w.layers)
        assert (16, False, False) in fc_candidates(w.layers)   # the default split is a candidate
        assert all(r["ms"] > 0 for r in report)
        assert min(r["ms"] for r in report) == [r["ms"] for r in report
                                                if (r["fc_n1"], r["hoist_moddown"], r["hoist_sums"]) == (n1, dh, hs)][0]
        model = H.hear_model_create(ctx, w.layers, w.clip_dim, fc_n1=n1, hoist_moddown=dh, hoist_sums=hs)
        steps = H.hear_model_rotations(model)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
        out = H.hear_evaluate(model, evk, [ct])[0]
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        z, kk = O.pack_clips(w.ct_clips(0), w.slots)
        r = o.evaluate(w.layers, o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale), kk, keys, n1=n1, dh=dh, hs=hs)
        assert np.array_equal(H.hear_ciphertext_export(out), o.to_coeff(r))
        for h in (ct, out):
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)
