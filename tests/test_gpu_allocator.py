"""A caller-supplied device allocator (hear_set_allocator): the context's allocations go
through it (here PyTorch's caching allocator), the results stay bit-identical to the
stream-ordered pool's, an allocation the caller refuses makes the call fail with
HEAR_E_NOMEM without poisoning the context, and everything allocated through the hook is
returned through it."""
import numpy as np
import pytest

from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def _run(H, ctx, w, keep=None):
    model = H.hear_model_create(ctx, w.layers, w.clip_dim)
    sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_model_rotations(model))
    ct = H.hear_encrypt_clips(ctx, pk, w.ct_clips(0), 401, 0)
    out = H.hear_evaluate(model, evk, [ct])[0]
    words = H.hear_ciphertext_export(out)
    handles = (model, sk, pk, evk, ct, out)
    if keep is not None:
        keep.extend(handles)
        return words
    H.hear_ciphertext_destroy(out)
    H.hear_ciphertext_destroy(ct)
    H.hear_model_destroy(model)
    H.hear_eval_keys_destroy(evk)
    H.hear_public_key_destroy(pk)
    H.hear_secret_key_destroy(sk)
    return words


def test_caller_allocator(H):
    import torch
    w = make_workload("small")
    ctx0 = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    try:
        ref = _run(H, ctx0, w)
    finally:
        H.hear_context_destroy(ctx0)

    calls = {"alloc": 0, "free": 0, "fail_at": None}
    live = {}

    def alloc(n, stream):
        calls["alloc"] += 1
        if calls["fail_at"] == calls["alloc"]:
            return 0
        p = torch.cuda.caching_allocator_alloc(n, device=0, stream=stream)
        live[p] = n
        return p

    def free(p, stream):
        calls["free"] += 1
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    keep = []
    try:
        H.hear_set_allocator(ctx, alloc, free)
        got = _run(H, ctx, w, keep)
        assert calls["alloc"] > 0 and live
        assert np.array_equal(got, ref)
        model, sk, pk, evk, ct, out = keep
        # the next allocation is refused: the call fails cleanly, the context stays usable
        calls["fail_at"] = calls["alloc"] + 1
        with pytest.raises(H.HearError) as e:
            H.hear_evaluate(model, evk, [ct])
        assert e.value.code == H.HEAR_E_NOMEM
        calls["fail_at"] = None
        again = H.hear_evaluate(model, evk, [ct])[0]
        assert np.array_equal(H.hear_ciphertext_export(again), ref)
        keep.append(again)
        with pytest.raises(H.HearError):
            H.hear_set_allocator(ctx, alloc, None)         # one function without the other
        # back to the pool: the handles made through the hook still release their memory
        # through it when they are destroyed below (the callbacks must stay alive)
        H.hear_set_allocator(ctx, None, None)
        import gc
        gc.collect()
        n_alloc = calls["alloc"]
        tmp = H.hear_evaluate(model, evk, [ct])[0]
        assert calls["alloc"] == n_alloc                   # no longer through the hook
        H.hear_ciphertext_destroy(tmp)
    finally:
        model, sk, pk, evk = keep[0], keep[1], keep[2], keep[3]
        for h in keep[4:]:
            H.hear_ciphertext_destroy(h)
        H.hear_model_destroy(model)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
        H.hear_context_destroy(ctx)
    torch.cuda.synchronize()
    assert not live and calls["free"] == calls["alloc"] - 1   # the refused one was never made
