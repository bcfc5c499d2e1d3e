"""Launch forms of the key-switch inner product and the BSGS inner sums (the autotuner's
candidates): the small network evaluated under every forced form, one ciphertext and a
batch of six (ciphertext chunks of 4 with a ragged last chunk), in the default FC form and
in the hoisted-ModDown form with 32 baby steps, gives the same ciphertexts bit for bit as
the default form, which equals the oracle; the tuner fills a valid table and its choice
evaluates identically too."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

FORMS = [(None, False), (32, True)]


@pytest.fixture(scope="module")
def env():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear as H
    w = make_workload("small", 24)
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    models = [H.hear_model_create(ctx, w.layers, w.clip_dim, fc_n1=n1, hoist_moddown=dh) for n1, dh in FORMS]
    steps = sorted(set(s for m in models for s in H.hear_model_rotations(m)))
    sk, pk, evk = H.hear_keygen(ctx, 301, steps)
    cts = [H.hear_encrypt_clips(ctx, pk, w.ct_clips(i), 401, i) for i in range(6)]
    yield H, w, ctx, models, steps, evk, cts
    for c in cts:
        H.hear_ciphertext_destroy(c)
    for m in models:
        H.hear_model_destroy(m)
    H.hear_eval_keys_destroy(evk)
    H.hear_public_key_destroy(pk)
    H.hear_secret_key_destroy(sk)
    H.hear_context_destroy(ctx)


def _eval(H, model, evk, cts):
    outs = H.hear_evaluate(model, evk, cts)
    words = [H.hear_ciphertext_export(o) for o in outs]
    for o in outs:
        H.hear_ciphertext_destroy(o)
    return words


def test_every_form_is_bit_exact(env):
    H, w, ctx, models, steps, evk, cts = env
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
    z, k = O.pack_clips(w.ct_clips(0), w.slots)
    fresh = o.encrypt(keys.pk, z, 401, 0, 2.0 ** w.log2_scale)
    for fi, (model, (n1, dh)) in enumerate(zip(models, FORMS)):
        H.hear_ks_set_variant(ctx, 0)
        ref1 = _eval(H, model, evk, cts[:1])
        ref6 = _eval(H, model, evk, cts)
        want = o.to_coeff(o.evaluate(w.layers, fresh, k, keys, n1=n1, dh=dh))
        assert np.array_equal(ref1[0], want), fi
        assert np.array_equal(ref6[0], want), fi
        for v in (1, 2, 3, 4):
            H.hear_ks_set_variant(ctx, v)
            assert all(np.array_equal(a, b) for a, b in zip(_eval(H, model, evk, cts[:1]), ref1)), (fi, v)
            assert all(np.array_equal(a, b) for a, b in zip(_eval(H, model, evk, cts), ref6)), (fi, v)
    H.hear_ks_set_variant(ctx, -1)
    assert H.hear_async_status(ctx) == 0          # no bounded wait of the bulk-copy forms ran out


def test_tuner_table_is_valid_and_exact(env):
    H, w, ctx, models, steps, evk, cts = env
    H.hear_ks_set_variant(ctx, 0)
    ref = _eval(H, models[1], evk, cts)
    H.hear_ks_set_variant(ctx, -1)
    choice, ms = H.hear_ks_tune(ctx, 8, 2)
    assert choice.shape == (3, 8)
    assert np.all(choice[0] < 4) and np.all(choice[1] < 5) and np.all(choice[2] < 5)
    assert np.all(ms[0, :4, :4] > 0) and np.all(ms[1, 1:5, :5] > 0) and np.all(ms[2, :4, :5] > 0)
    table = H.hear_ks_get_table(ctx)
    assert len(table) == 24
    assert all(np.array_equal(a, b) for a, b in zip(_eval(H, models[1], evk, cts), ref))
    H.hear_ks_set_table(ctx, "0" * 24)
    assert H.hear_ks_get_table(ctx) == "0" * 24
    with pytest.raises(H.HearError):
        H.hear_ks_set_table(ctx, "5" * 24)          # table 0 has 4 forms, tables 1 and 2 have 5


def test_bounded_wait_runs_out_and_is_reported(env):
    """a wait on an mbarrier that nothing completes returns after its limit (no hang, no
    fault), is counted, reported once by hear_async_status and cleared; the context stays
    usable and evaluates bit-identically afterwards"""
    H, w, ctx, models, steps, evk, cts = env
    assert H.hear_async_status(ctx) == 0
    assert H.hear_dbg_wait_probe(ctx, 20000) is True
    assert H.hear_dbg_wait_probe(ctx, 0) is True
    assert H.hear_async_status(ctx) == 2
    assert H.hear_async_status(ctx) == 0
    H.hear_ks_set_variant(ctx, 0)
    ref = _eval(H, models[0], evk, cts[:1])
    H.hear_ks_set_variant(ctx, 4)
    assert np.array_equal(_eval(H, models[0], evk, cts[:1])[0], ref[0])
    H.hear_ks_set_variant(ctx, -1)
    assert H.hear_async_status(ctx) == 0
