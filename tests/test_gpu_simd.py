"""Slot-batched evaluation (one clip per slot, one ciphertext per feature) through the C ABI:
ciphertexts bit-exact against the oracle (toy networks whole; the small network's FC
2048->128 at full size on sampled outputs), decrypted logits within 2^-15 of FP64 for every
clip of full batches (small: 8192 clips, large: 16384 clips), the host end-to-end entry
point, and the error paths."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

LOGIT_TOL = 2.0 ** -15
SEED_KEYS, SEED_ENC = 301, 401


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def _ctx(H, log_n, q_bits, p_bits):
    return H.hear_context_create(log_n, q_bits, p_bits, 40.0, 3.2, 0)


def _oracle_encrypt(o, pk, X, seed, scale):
    """the oracle's encrypt_simd, ciphertexts encrypted in parallel (same streams)"""
    X = np.asarray(X, dtype=np.float64)

    def one(i):
        z = np.zeros(o.n // 2)
        z[:X.shape[0]] = X[:, i]
        return o.encrypt(pk, z, seed, i, scale)
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        return list(ex.map(one, range(X.shape[1])))


def _fp64(layers, X):
    h = np.asarray(X, dtype=np.float64)
    for layer in layers:
        if layer[0] == "fc":
            h = h @ layer[1].T
        elif layer[0] == "square":
            h = h * h
        else:
            y = h @ layer[1].T
            h = (y * y) @ layer[2].T
    return h


def _run(H, ctx, layers, X, level=0):
    m = H.hear_simd_model_create(ctx, layers, level)
    sk, pk, evk = H.hear_keygen(ctx, SEED_KEYS, [])
    b = H.hear_simd_encrypt(ctx, pk, X, SEED_ENC, level)
    out = H.hear_simd_evaluate(m, evk, b)
    return m, (sk, pk, evk), b, out


def _free(H, m, keys, *batches):
    for b in batches:
        H.hear_simd_batch_destroy(b)
    H.hear_simd_model_destroy(m)
    H.hear_eval_keys_destroy(keys[2])
    H.hear_public_key_destroy(keys[1])
    H.hear_secret_key_destroy(keys[0])


@pytest.mark.parametrize("level", [0, 1])
def test_simd_encrypt_matches_oracle(H, level):
    w = make_workload("toy", n_clips=300)
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        sk, pk, evk = H.hear_keygen(ctx, SEED_KEYS, [])
        X = w.clips[:, :12]
        b = H.hear_simd_encrypt(ctx, pk, X, SEED_ENC, level)
        n_ct, lv, sc = H.hear_simd_batch_info(b)
        top = len(w.q_bits) - 1
        assert (n_ct, lv, sc) == (12, level or top, 2.0 ** 40)
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=1)
        keys = o.keygen(SEED_KEYS, [])
        ref = _oracle_encrypt(o, keys.pk, X, SEED_ENC, 2.0 ** 40)
        got = H.hear_simd_batch_export(b)
        for i, c in enumerate(ref):
            while c.level > lv:
                c = o.drop_level(c)
            assert np.array_equal(got[i], o.to_coeff(c))
        H.hear_simd_batch_destroy(b)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_context_destroy(ctx)


def test_toy_network_bit_exact_and_logits(H):
    """FC 64->16 -> x^2 -> FC 16->2 (collapsed) with a clip in every one of the 2048 slots"""
    w = make_workload("toy", n_clips=2048)
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        m, keys, b, out = _run(H, ctx, w.layers, w.clips)
        assert H.hear_simd_model_info(m) == (64, 2, 2, 0)
        n_ct, lv, sc = H.hear_simd_batch_info(out)
        assert (n_ct, lv) == (2, 0)
        logits = H.hear_simd_decrypt(ctx, keys[0], out, w.n_clips)
        assert np.max(np.abs(logits - w.fp64_forward(w.clips))) <= LOGIT_TOL
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        ok = o.keygen(SEED_KEYS, [])
        r = o.evaluate_simd(w.layers, _oracle_encrypt(o, ok.pk, w.clips, SEED_ENC, 2.0 ** 40), ok)
        got = H.hear_simd_batch_export(out)
        assert sc == r[0].scale
        for j in range(2):
            assert np.array_equal(got[j], o.to_coeff(r[j]))
        _free(H, m, keys, b, out)
    finally:
        H.hear_context_destroy(ctx)


def test_fc_square_fc_bit_exact(H):
    """separate FC 64->20 (ragged rows) -> x^2 -> FC 20->3 on a three-level chain with a
    50-bit first prime (the 31-bit-piece form of the matrix product), 1000 clips"""
    log_n, q_bits, p_bits = 12, [50, 40, 40, 40], [50]
    rng = np.random.default_rng(77)
    X = rng.uniform(-1, 1, size=(1000, 64))
    layers = [("fc", rng.normal(0, 0.15, size=(20, 64))), ("square",), ("fc", rng.normal(0, 0.3, size=(3, 20)))]
    ctx = _ctx(H, log_n, q_bits, p_bits)
    try:
        m, keys, b, out = _run(H, ctx, layers, X)
        assert H.hear_simd_model_info(m) == (64, 3, 3, 0)
        logits = H.hear_simd_decrypt(ctx, keys[0], out, 1000)
        assert np.max(np.abs(logits - _fp64(layers, X))) <= LOGIT_TOL
        o = O.Oracle(log_n, q_bits, p_bits, 3.2, threads=os.cpu_count() or 0)
        ok = o.keygen(SEED_KEYS, [])
        r = o.evaluate_simd(layers, _oracle_encrypt(o, ok.pk, X, SEED_ENC, 2.0 ** 40), ok)
        got = H.hear_simd_batch_export(out)
        for j in range(3):
            assert np.array_equal(got[j], o.to_coeff(r[j]))
        # the same from host buffers (copies both ways inside the call)
        words = H.hear_simd_batch_export(b)
        flat, lv, sc = H.hear_simd_evaluate_host(m, keys[2], words, 2.0 ** 40)
        assert lv == 0 and sc == H.hear_simd_batch_info(out)[2]
        assert np.array_equal(flat.reshape(got.shape), got)
        _free(H, m, keys, b, out)
    finally:
        H.hear_context_destroy(ctx)


def test_small_fc_full_size_sampled(H):
    """FC 2048->128 of the small network at N = 2^14 on 8192 clips (the benchmarked launch):
    two sampled output ciphertexts bit-exact against the oracle"""
    w = make_workload("small", n_clips=8192)
    W1 = w.layers[0][1]
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        m, keys, b, out = _run(H, ctx, [("fc", W1)], w.clips)
        got = H.hear_simd_batch_export(out)
        assert got.shape[0] == 128
        o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=1)
        ok = o.keygen(SEED_KEYS, [])
        cts = _oracle_encrypt(o, ok.pk, w.clips, SEED_ENC, 2.0 ** 40)
        o2 = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=os.cpu_count() or 0)
        for j in (0, 101):
            r = o2.fc_simd(cts, W1[j:j + 1])[0]
            assert np.array_equal(got[j], o2.to_coeff(r))
        _free(H, m, keys, b, out)
    finally:
        H.hear_context_destroy(ctx)


@pytest.mark.parametrize("name,n_clips", [("small", 8192), ("large", 16384)])
def test_full_batch_logits(H, name, n_clips):
    w = make_workload(name, n_clips=n_clips)
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        m, keys, b, out = _run(H, ctx, w.layers, w.clips)
        d_in, d_out, lin, lout = H.hear_simd_model_info(m)
        assert (d_in, d_out, lin) == (2048, 2, len(w.q_bits) - 1)
        assert H.hear_simd_batch_info(out)[:2] == (2, lout)
        logits = H.hear_simd_decrypt(ctx, keys[0], out, n_clips)
        assert np.max(np.abs(logits - w.fp64_forward(w.clips))) <= LOGIT_TOL
        _free(H, m, keys, b, out)
    finally:
        H.hear_context_destroy(ctx)


def test_simd_error_paths(H):
    w = make_workload("toy", n_clips=10)
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        m, keys, b, out = _run(H, ctx, w.layers, w.clips)
        short = H.hear_simd_encrypt(ctx, keys[1], w.clips[:, :32], SEED_ENC)
        with pytest.raises(H.HearError):
            H.hear_simd_evaluate(m, keys[2], short)          # 32 ciphertexts, the model wants 64
        low = H.hear_simd_encrypt(ctx, keys[1], w.clips, SEED_ENC, 1)
        with pytest.raises(H.HearError):
            H.hear_simd_evaluate(m, keys[2], low)            # below the model's input level
        with pytest.raises(H.HearError):
            H.hear_simd_model_create(ctx, [("square",)])     # no linear first layer
        with pytest.raises(H.HearError):
            H.hear_simd_model_create(ctx, w.layers + [("square",)])   # out of levels
        with pytest.raises(H.HearError):
            H.hear_simd_encrypt(ctx, keys[1], np.zeros((2049, 4)), SEED_ENC)   # more clips than slots
        with pytest.raises(H.HearError):
            H.hear_simd_model_create(ctx, [("fc", np.full((2, 64), 2.0 ** 60))])   # scalar out of range
        _free(H, m, keys, b, out, short, low)
    finally:
        H.hear_context_destroy(ctx)


def test_imad_peak_probe(H):
    """the multiply-add throughput probe returns a rate between 1 and 200 T lane-ops/s, and
    the 32-bit form is not slower than the widening one"""
    w = make_workload("toy")
    ctx = _ctx(H, w.log_n, w.q_bits, w.p_bits)
    try:
        wide = H.hear_dbg_imad_peak(ctx, 0, 1024)
        lo = H.hear_dbg_imad_peak(ctx, 1, 1024)
        assert 1e12 < wide < 2e14 and 1e12 < lo < 2e14
        assert lo > 0.8 * wide
        with pytest.raises(H.HearError):
            H.hear_dbg_imad_peak(ctx, 2, 16)
    finally:
        H.hear_context_destroy(ctx)
