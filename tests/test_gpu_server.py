"""Continuous-batching server: requests of different sizes submitted together from two
threads are admitted, mixed into batches and overlapped on the device; every result must
be bit-identical to the same request evaluated alone, and the admission must respect the
HBM budget."""
import threading
import time

import numpy as np
import pytest

from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear as H
    w = make_workload("toy")
    ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
    model = H.hear_model_create(ctx, w.layers, w.clip_dim)
    sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_model_rotations(model))
    rng = np.random.default_rng(77)
    reqs = []
    for i, n_ct in enumerate([1, 3, 2, 1, 1, 2, 3, 1, 2, 1]):
        words = []
        for j in range(n_ct):
            x = rng.uniform(-1, 1, (1, w.clip_dim))
            ct = H.hear_encrypt_clips(ctx, pk, x, 500 + i, j)
            words.append(H.hear_ciphertext_export(ct).reshape(-1))
            H.hear_ciphertext_destroy(ct)
        reqs.append((n_ct, np.concatenate(words)))
    yield H, w, ctx, model, evk, reqs
    H.hear_model_destroy(model)
    for h, f in ((evk, H.hear_eval_keys_destroy), (pk, H.hear_public_key_destroy), (sk, H.hear_secret_key_destroy)):
        f(h)
    H.hear_context_destroy(ctx)


def _wait(H, srv, ids, out_words, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids) and time.time() - t0 < timeout:
        for rid, n_ct in ids:
            if rid not in res:
                r = H.hear_server_poll(srv, rid, n_ct * out_words)
                if r is not None:
                    res[rid] = r
        time.sleep(0.001)
    assert len(res) == len(ids), "requests did not complete"
    return res


def test_results_in_the_mix_equal_results_alone(setup):
    H, w, ctx, model, evk, reqs = setup
    scale = 2.0 ** w.log2_scale
    alone = [H.hear_evaluate_host(model, evk, words, n_ct, scale)[0] for n_ct, words in reqs]
    out_words = alone[0].size // reqs[0][0]
    srv = H.hear_server_create(model, evk, max_batch=4, n_slots=2, hbm_budget_bytes=8 << 30)
    try:
        ids = [None] * len(reqs)

        def submit(idx):
            for i in idx:
                ids[i] = (H.hear_server_submit(srv, reqs[i][1], reqs[i][0], reqs[i][0], scale), reqs[i][0])
        th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        res = _wait(H, srv, ids, out_words)
        for i, (rid, _) in enumerate(ids):
            assert np.array_equal(res[rid], alone[i]), i
        st = H.hear_server_stats(srv)
        assert st["requests_done"] == len(reqs)
        assert st["ciphertexts_done"] == sum(n for n, _ in reqs)
        assert 1 <= st["batches"] < len(reqs)          # requests were mixed into batches
        assert 0 < st["p50_ms"] <= st["p99_ms"]
        with pytest.raises(H.HearError):
            H.hear_server_poll(srv, ids[0][0], out_words)   # ids are released once read
    finally:
        H.hear_server_destroy(srv)


def test_admission_respects_the_hbm_budget(setup):
    H, w, ctx, model, evk, reqs = setup
    scale = 2.0 ** w.log2_scale
    probe = H.hear_server_create(model, evk, max_batch=4, n_slots=2, hbm_budget_bytes=1 << 40)
    per_ct = H.hear_server_stats(probe)["bytes_per_ciphertext"]
    H.hear_server_destroy(probe)
    assert per_ct > 0
    srv = H.hear_server_create(model, evk, max_batch=4, n_slots=2, hbm_budget_bytes=2 * per_ct)
    try:
        singles = [r for r in reqs if r[0] == 1]
        ids = [(H.hear_server_submit(srv, words, 1, 1, scale), 1) for _, words in singles]
        out_words = H.hear_evaluate_host(model, evk, singles[0][1], 1, scale)[0].size
        _wait(H, srv, ids, out_words)
        st = H.hear_server_stats(srv)
        assert st["requests_done"] == len(singles)
        assert st["max_in_flight_ciphertexts"] <= 2
        three = [r for r in reqs if r[0] == 3][0]
        with pytest.raises(H.HearError) as e:
            H.hear_server_submit(srv, three[1], 3, 3, scale)
        assert e.value.code == -2
    finally:
        H.hear_server_destroy(srv)


def test_two_networks_served_together_equal_alone():
    """small (N = 2^14) and large (N = 2^15) requests interleaved from one submitter into two
    servers running at once on one GPU: every result equals its request evaluated alone"""
    from paper_2104_09164_gb300 import hear as H
    rng = np.random.default_rng(91)
    nets = []
    for name, n_clips in (("small", None), ("large", 8)):
        w = make_workload(name, n_clips)
        ctx = H.hear_context_create(w.log_n, w.q_bits, w.p_bits, w.log2_scale, w.sigma, 0)
        model = H.hear_model_create(ctx, w.layers, w.clip_dim)
        sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_model_rotations(model))
        k = w.slots // w.clip_dim
        reqs = []
        for i, n_ct in enumerate([1, 2, 1, 3] if name == "small" else [1, 1, 2]):
            words = []
            for j in range(n_ct):
                x = rng.uniform(-1, 1, (k, w.clip_dim))
                ct = H.hear_encrypt_clips(ctx, pk, x, 700 + i, j)
                words.append(H.hear_ciphertext_export(ct).reshape(-1))
                H.hear_ciphertext_destroy(ct)
            reqs.append((n_ct, np.concatenate(words)))
        scale = 2.0 ** w.log2_scale
        alone = [H.hear_evaluate_host(model, evk, words, n_ct, scale)[0] for n_ct, words in reqs]
        srv = H.hear_server_create(model, evk, max_batch=4, n_slots=2, hbm_budget_bytes=32 << 30)
        nets.append(dict(H=H, ctx=ctx, model=model, keys=(sk, pk, evk), reqs=reqs, alone=alone, srv=srv,
                         scale=scale, out_words=alone[0].size // reqs[0][0]))
    try:
        order = [(0, i) for i in range(len(nets[0]["reqs"]))] + [(1, i) for i in range(len(nets[1]["reqs"]))]
        rng.shuffle(order)
        ids = {}
        for ni, i in order:
            n = nets[ni]
            n_ct, words = n["reqs"][i]
            ids[(ni, i)] = H.hear_server_submit(n["srv"], words, n_ct, n_ct, n["scale"])
        for ni, n in enumerate(nets):
            mine = [(ids[(ni, i)], n["reqs"][i][0]) for i in range(len(n["reqs"]))]
            res = _wait(H, n["srv"], mine, n["out_words"])
            for i, (rid, _) in enumerate(mine):
                assert np.array_equal(res[rid], n["alone"][i]), (ni, i)
    finally:
        for n in nets:
            H.hear_server_destroy(n["srv"])
            H.hear_model_destroy(n["model"])
            sk, pk, evk = n["keys"]
            H.hear_eval_keys_destroy(evk)
            H.hear_public_key_destroy(pk)
            H.hear_secret_key_destroy(sk)
            H.hear_context_destroy(n["ctx"])


def test_busy_timeout_and_pause(setup):
    """bounded waits and refusals, made deterministic with the pause switch: while paused
    nothing is admitted, so a wait runs out (HEAR_E_TIMEOUT, the request stays queued), a
    submit beyond the staging buffers or the queue limit is refused (HEAR_E_BUSY, nothing
    queued); after resuming every queued request completes bit-identical to alone"""
    H, w, ctx, model, evk, reqs = setup
    scale = 2.0 ** w.log2_scale
    two = [r for r in reqs if r[0] == 2]
    one = [r for r in reqs if r[0] == 1]
    alone2 = H.hear_evaluate_host(model, evk, two[0][1], 2, scale)[0]
    alone1 = H.hear_evaluate_host(model, evk, one[0][1], 1, scale)[0]
    out1 = alone1.size
    srv = H.hear_server_create(model, evk, max_batch=4, n_slots=1, hbm_budget_bytes=8 << 30, staging_cts=4,
                               max_pending=3)
    try:
        H.hear_server_pause(srv, True)
        a = H.hear_server_submit(srv, two[0][1], 2, 2, scale)
        b = H.hear_server_submit(srv, one[0][1], 1, 1, scale)
        t0 = time.time()
        with pytest.raises(H.HearError) as e:
            H.hear_server_wait(srv, a, 2 * out1, timeout_ms=50)
        assert e.value.code == H.HEAR_E_TIMEOUT
        assert time.time() - t0 >= 0.045
        # 3 of 4 staging buffers are taken: a 2-ciphertext request does not fit
        with pytest.raises(H.HearError) as e:
            H.hear_server_submit(srv, two[0][1], 2, 2, scale)
        assert e.value.code == H.HEAR_E_BUSY
        c = H.hear_server_submit(srv, one[0][1], 1, 1, scale)
        # the queue holds max_pending = 3 requests now
        with pytest.raises(H.HearError) as e:
            H.hear_server_submit(srv, one[0][1], 1, 1, scale)
        assert e.value.code == H.HEAR_E_BUSY
        st = H.hear_server_stats(srv)
        assert st["pending"] == 3 and st["busy_refusals"] == 2 and st["requests_done"] == 0
        H.hear_server_pause(srv, False)
        assert np.array_equal(H.hear_server_wait(srv, a, 2 * out1, timeout_ms=60000), alone2)
        assert np.array_equal(H.hear_server_wait(srv, b, out1, timeout_ms=60000), alone1)
        assert np.array_equal(H.hear_server_wait(srv, c, out1, timeout_ms=60000), alone1)
        # buffers came back: the refused request is accepted now
        d = H.hear_server_submit(srv, two[0][1], 2, 2, scale)
        assert np.array_equal(H.hear_server_wait(srv, d, 2 * out1, timeout_ms=60000), alone2)
        with pytest.raises(H.HearError):
            H.hear_server_wait(srv, d, 2 * out1, timeout_ms=10)     # the id was released
        # an unreduced residue is refused without queueing anything
        bad = one[0][1].copy()
        bad[5] = np.uint64(H.hear_context_primes(ctx)[0])
        with pytest.raises(H.HearError) as e:
            H.hear_server_submit(srv, bad, 1, 1, scale)
        assert e.value.code == H.HEAR_E_FORMAT
        assert H.hear_server_stats(srv)["pending"] == 0
    finally:
        H.hear_server_destroy(srv)
