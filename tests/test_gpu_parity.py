"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Ciphertexts, keys and encodings must agree bit for bit (compared in the coefficient
domain, so each side's NTT ordering stays internal); decrypted values must agree with
the FP64 plaintext computation within the stated bound.
"""
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


class Pair:
    """the same parameter set on both sides, keys from the same seed"""

    def __init__(self, H, log_n, q_bits, p_bits, steps, seed=301, relin=True):
        self.H = H
        self.o = O.Oracle(log_n, q_bits, p_bits, 3.2)
        self.ctx = H.hear_context_create(log_n, q_bits, p_bits, 40.0, 3.2, 0)
        self.n = 1 << log_n
        self.steps = sorted(set(int(s) for s in steps))
        self.sk, self.pk, self.evk = H.hear_keygen(self.ctx, seed, self.steps)
        gal = sorted(set(O.galois_for_step(s, self.n) for s in self.steps) - {1})
        self.keys = self.o.keygen(seed, gal, relin=relin)

    def close(self):
        H = self.H
        H.hear_eval_keys_destroy(self.evk)
        H.hear_public_key_destroy(self.pk)
        H.hear_secret_key_destroy(self.sk)
        H.hear_context_destroy(self.ctx)

    def export(self, ct):
        return self.H.hear_ciphertext_export(ct)

    def same(self, gpu_ct, oracle_ct):
        g = self.export(gpu_ct)
        o = self.o.to_coeff(oracle_ct)
        lv, npl, sc = self.H.hear_ciphertext_info(gpu_ct)
        assert (lv, npl) == (oracle_ct.level, oracle_ct.n_poly)
        assert sc == oracle_ct.scale
        return g.shape == o.shape and np.array_equal(g, o)


@pytest.fixture(scope="module")
def toy(H):
    w = make_workload("toy")
    z, k = O.pack_clips(w.clips, w.slots)
    steps = O.rotation_steps(w.layers, w.clip_dim, k) + [1, 2, 5, -3, 100]
    p = Pair(H, w.log_n, w.q_bits, w.p_bits, steps)
    p.w, p.z, p.k = w, z, k
    yield p
    p.close()


@pytest.fixture(scope="module")
def hybrid(H):
    # two special primes: digits of alpha = 2 limbs (five limbs -> digits {0,1},{2,3},{4})
    p = Pair(H, 12, [50, 40, 40, 40, 40], [50, 50], [1, 3, 64, -7])
    yield p
    p.close()


# ------------------------------------------------------------------ set-up and NTT
def test_primes_and_cdt_match(toy, hybrid):
    for p in (toy, hybrid):
        assert p.H.hear_context_primes(p.ctx) == p.o.primes
        import ctypes
        t = np.zeros(64, dtype=np.uint64)
        cnt = np.zeros(1, dtype=np.uint32)
        O.lib().or_cdt_table(p.o.h, O.P(t), 64, O.P(cnt, O._u32p))
        assert p.H.hear_context_cdt(p.ctx) == [int(x) for x in t[:int(cnt[0])]]


def test_ntt_product_matches_oracle(toy, hybrid):
    rng = np.random.default_rng(1)
    for p in (toy, hybrid):
        for pi, q in enumerate(p.o.primes):
            a = rng.integers(0, q, p.n, dtype=np.uint64)
            b = rng.integers(0, q, p.n, dtype=np.uint64)
            A = p.o.ntt_fwd(a[None], [pi])
            B = p.o.ntt_fwd(b[None], [pi])
            C = np.array([int(x) * int(y) % q for x, y in zip(A[0], B[0])], dtype=np.uint64)
            want = p.o.ntt_inv(C[None], [pi])[0]
            assert np.array_equal(p.H.hear_dbg_poly_mul(p.ctx, pi, a, b), want), pi
        limbs = np.stack([rng.integers(0, p.o.primes[i % len(p.o.primes)], p.n, dtype=np.uint64)
                          for i in range(7)])
        assert np.array_equal(p.H.hear_dbg_ntt_roundtrip(p.ctx, limbs), limbs)


# ------------------------------------------------------------------ keys, encoding, encryption
def test_keys_match_oracle(toy, hybrid):
    for p in (toy, hybrid):
        H, o = p.H, p.o
        assert np.array_equal(H.hear_secret_key_export(p.sk), p.keys.s)
        pk = H.hear_public_key_export(p.pk).reshape(2, o.n_q, p.n)
        assert np.array_equal(pk, o.to_coeff(O.Ct(p.keys.pk, o.L, 1)))
        nqp = o.n_q + o.n_p
        allp = list(range(nqp))

        def coeff_key(key):
            return np.stack([np.stack([o.ntt_inv(key[j, b], allp) for b in range(2)])
                             for j in range(key.shape[0])])
        relin = H.hear_eval_key_export(p.evk, 1).reshape(-1, 2, nqp, p.n)
        assert np.array_equal(relin, coeff_key(p.keys.relin))
        g = O.galois_for_step(p.steps[0], p.n)
        rot = H.hear_eval_key_export(p.evk, g).reshape(-1, 2, nqp, p.n)
        assert np.array_equal(rot, coeff_key(p.keys.rot[g]))


def test_encode_matches_oracle(toy):
    rng = np.random.default_rng(2)
    for scale in (2.0 ** 40, float(toy.o.q[2]), 12345.678):
        z = rng.uniform(-1, 1, toy.n // 2)
        m_o, ties = toy.o.encode(z, scale)
        assert ties == 0
        assert np.array_equal(toy.H.hear_encode(toy.ctx, z, scale), m_o)


@pytest.mark.parametrize("ct_id", [0, 7])
def test_encrypt_and_decrypt(toy, ct_id):
    H = toy.H
    ct = H.hear_encrypt(toy.ctx, toy.pk, toy.z, 2.0 ** 40, 401, ct_id)
    ref = toy.o.encrypt(toy.keys.pk, toy.z, 401, ct_id, 2.0 ** 40)
    assert toy.same(ct, ref)
    dec = H.hear_decrypt(toy.ctx, toy.sk, ct)
    assert np.max(np.abs(dec - toy.z)) < 1e-6
    assert np.max(np.abs(dec - toy.o.decrypt(toy.keys, ref))) < 1e-9
    H.hear_ciphertext_destroy(ct)


def test_encrypt_clips_packing(toy):
    H = toy.H
    ct = H.hear_encrypt_clips(toy.ctx, toy.pk, toy.w.clips, 401, 0)
    ref = toy.o.encrypt(toy.keys.pk, toy.z, 401, 0, 2.0 ** 40)
    assert toy.same(ct, ref)
    H.hear_ciphertext_destroy(ct)


# ------------------------------------------------------------------ primitives
def _fresh(p, seed=401, ct_id=0):
    rng = np.random.default_rng(100 + ct_id)
    z = rng.uniform(-1, 1, p.n // 2)
    g = p.H.hear_encrypt(p.ctx, p.pk, z, 2.0 ** 40, seed, ct_id)
    o = p.o.encrypt(p.keys.pk, z, seed, ct_id, 2.0 ** 40)
    assert p.same(g, o)
    return z, g, o


@pytest.mark.parametrize("which", ["toy", "hybrid"])
def test_rotations_bit_exact(which, request):
    p = request.getfixturevalue(which)
    H = p.H
    z, g, o = _fresh(p, ct_id=3)
    steps = [s for s in p.steps if s in (1, 3, 5, -3, -7, 64, 100)]
    outs = H.hear_rotate_hoisted(p.evk, g, steps)
    refs = p.o.rotate_hoisted(o, steps, p.keys)
    for st, a, b in zip(steps, outs, refs):
        assert p.same(a, b), st
        assert np.max(np.abs(H.hear_decrypt(p.ctx, p.sk, a) - np.roll(z, -st))) < 1e-5
        H.hear_ciphertext_destroy(a)
    single = H.hear_rotate(p.evk, g, steps[0])
    assert p.same(single, refs[0])
    H.hear_ciphertext_destroy(single)
    H.hear_ciphertext_destroy(g)


@pytest.mark.parametrize("which", ["toy", "hybrid"])
def test_rescale_mul_mulplain_add_bit_exact(which, request):
    p = request.getfixturevalue(which)
    H, o = p.H, p.o
    za, ga, oa = _fresh(p, ct_id=1)
    zb, gb, ob = _fresh(p, ct_id=2)
    # ciphertext product with relinearisation, then rescale
    gm = H.hear_multiply_relin(p.evk, ga, gb)
    om = o.relinearize(o.tensor(oa, ob), p.keys)
    assert p.same(gm, om)
    gr = H.hear_rescale(gm)
    orr = o.rescale(om)
    assert p.same(gr, orr)
    assert np.max(np.abs(H.hear_decrypt(p.ctx, p.sk, gr) - za * zb)) < 1e-5
    # MultPlain at scale q_L, add, rescale
    w = np.random.default_rng(9).uniform(-2, 2, p.n // 2)
    ql = float(o.q[o.L])
    gp = H.hear_mulplain(ga, w, ql)
    op = o.mulplain(oa, o.encode_pt(w, ql, o.L), ql)
    assert p.same(gp, op)
    gs = H.hear_add(gp, gp)
    os_ = o.add(op, op)
    assert p.same(gs, os_)
    for h in (ga, gb, gm, gr, gp, gs):
        H.hear_ciphertext_destroy(h)


def test_import_export_roundtrip(toy):
    H = toy.H
    z, g, o = _fresh(toy, ct_id=4)
    words = H.hear_ciphertext_export(g)
    g2 = H.hear_ciphertext_import(toy.ctx, words, toy.o.L, 2, 2.0 ** 40)
    assert toy.same(g2, o)
    bad = words.copy()
    bad[0, 0, 0] = toy.o.q[0]
    with pytest.raises(H.HearError):
        H.hear_ciphertext_import(toy.ctx, bad, toy.o.L, 2, 2.0 ** 40)
    H.hear_ciphertext_destroy(g)
    H.hear_ciphertext_destroy(g2)


def test_missing_key_and_level_errors(toy):
    H = toy.H
    z, g, o = _fresh(toy, ct_id=5)
    with pytest.raises(H.HearError) as e:
        H.hear_rotate(toy.evk, g, 11)
    assert e.value.code == -6
    lvl0 = g
    for _ in range(toy.o.L):
        nxt = H.hear_rescale(lvl0)
        if lvl0 != g:
            H.hear_ciphertext_destroy(lvl0)
        lvl0 = nxt
    with pytest.raises(H.HearError) as e:
        H.hear_rescale(lvl0)
    assert e.value.code == -4
    H.hear_ciphertext_destroy(lvl0)
    H.hear_ciphertext_destroy(g)


# ------------------------------------------------------------------ network
def test_toy_network_bit_exact(toy):
    H, o, w = toy.H, toy.o, toy.w
    model = H.hear_model_create(toy.ctx, w.layers, w.clip_dim)
    assert H.hear_model_rotations(model) == O.rotation_steps(w.layers, w.clip_dim, toy.k)
    ct = H.hear_encrypt_clips(toy.ctx, toy.pk, w.clips, 401, 0)
    out = H.hear_evaluate(model, toy.evk, [ct])[0]
    ref = o.evaluate(w.layers, o.encrypt(toy.keys.pk, toy.z, 401, 0, 2.0 ** 40), toy.k, toy.keys)
    assert toy.same(out, ref)
    dec = H.hear_decrypt(toy.ctx, toy.sk, out)
    pos = H.hear_model_output_positions(model)
    assert pos == O.output_positions(w.layers)
    logits = np.array([dec[p * toy.k] for p in pos])
    assert np.max(np.abs(logits - w.fp64_forward(w.clips)[0])) <= LOGIT_TOL
    for h in (ct, out):
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)


def test_toy_ragged_batch_equals_singles(toy):
    """ciphertexts evaluated together in a batch of 3 equal the ones evaluated alone"""
    H, w = toy.H, toy.w
    model = H.hear_model_create(toy.ctx, w.layers, w.clip_dim)
    cts = [H.hear_encrypt_clips(toy.ctx, toy.pk, w.clips * (0.5 + 0.2 * i), 401, i) for i in range(3)]
    batch = H.hear_evaluate(model, toy.evk, cts)
    for i, c in enumerate(cts):
        alone = H.hear_evaluate(model, toy.evk, [c])[0]
        assert np.array_equal(H.hear_ciphertext_export(alone), H.hear_ciphertext_export(batch[i]))
        H.hear_ciphertext_destroy(alone)
    for h in cts + batch:
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)


@pytest.fixture(scope="module")
def small(H):
    w = make_workload("small")
    z, k = O.pack_clips(w.ct_clips(0), w.slots)
    steps = O.rotation_steps(w.layers, w.clip_dim, k)
    p = Pair(H, w.log_n, w.q_bits, w.p_bits, steps)
    p.w, p.z, p.k = w, z, k
    yield p
    p.close()


def test_small_network_per_layer_bit_exact(small):
    """N = 2^14, FC 2048->128 -> x^2 -> FC 128->2: every layer's output equals the oracle's."""
    H, o, w = small.H, small.o, small.w
    model = H.hear_model_create(small.ctx, w.layers, w.clip_dim)
    g = H.hear_encrypt_clips(small.ctx, small.pk, w.ct_clips(0), 401, 0)
    r = o.encrypt(small.keys.pk, small.z, 401, 0, 2.0 ** 40)
    assert small.same(g, r)
    for li, layer in enumerate(w.layers):
        g2 = H.hear_evaluate_layer(model, li, small.evk, [g])[0]
        r = o.evaluate([layer], r, small.k, small.keys)
        assert small.same(g2, r), li
        H.hear_ciphertext_destroy(g)
        g = g2
    dec = H.hear_decrypt(small.ctx, small.sk, g)
    logits = np.array([dec[p * small.k] for p in H.hear_model_output_positions(model)])
    assert np.max(np.abs(logits - w.fp64_forward(w.ct_clips(0))[0])) <= LOGIT_TOL
    # whole network in one call and through host buffers give the same ciphertext
    c0 = H.hear_encrypt_clips(small.ctx, small.pk, w.ct_clips(0), 401, 0)
    whole = H.hear_evaluate(model, small.evk, [c0])[0]
    assert np.array_equal(H.hear_ciphertext_export(whole), H.hear_ciphertext_export(g))
    words, lv, sc = H.hear_evaluate_host(model, small.evk, H.hear_ciphertext_export(c0), 1, 2.0 ** 40)
    assert lv == r.level and sc == r.scale
    assert np.array_equal(words.reshape(2, lv + 1, -1), o.to_coeff(r))
    # the host path again (its captured graph replayed) on two other ciphertexts in one call:
    # each equals the NTT-domain path's result
    c1 = H.hear_encrypt_clips(small.ctx, small.pk, w.ct_clips(0), 402, 1)
    c2 = H.hear_encrypt_clips(small.ctx, small.pk, w.ct_clips(0), 403, 2)
    for _ in range(2):
        words2, _, _ = H.hear_evaluate_host(model, small.evk, np.concatenate(
            [H.hear_ciphertext_export(c).reshape(-1) for c in (c1, c2)]), 2, 2.0 ** 40)
        dev = H.hear_evaluate(model, small.evk, [c1, c2])
        assert np.array_equal(words2.reshape(2, -1), np.stack([H.hear_ciphertext_export(d).reshape(-1) for d in dev]))
        for d in dev:
            H.hear_ciphertext_destroy(d)
    for h in (g, c0, c1, c2, whole):
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)


def test_graph_replay_equals_direct_launches(toy):
    """Whole evaluations replay a captured CUDA graph; with the stage profiler on the same
    kernels are launched one by one.  Both must give the same ciphertext, and the profiler
    must account for the launches."""
    H, w = toy.H, toy.w
    model = H.hear_model_create(toy.ctx, w.layers, w.clip_dim)
    ct = H.hear_encrypt_clips(toy.ctx, toy.pk, w.clips, 401, 9)
    g1 = H.hear_evaluate(model, toy.evk, [ct])[0]        # builds and replays the graph
    g2 = H.hear_evaluate(model, toy.evk, [ct])[0]        # replays it again
    H.hear_profile_begin(toy.ctx)
    n0 = H.hear_launch_count()
    d = H.hear_evaluate(model, toy.evk, [ct])[0]         # direct launches
    n1 = H.hear_launch_count()
    stages = H.hear_profile_end(toy.ctx)
    ref = H.hear_ciphertext_export(d)
    assert np.array_equal(H.hear_ciphertext_export(g1), ref)
    assert np.array_equal(H.hear_ciphertext_export(g2), ref)
    assert sum(v[0] for v in stages.values()) == n1 - n0 > 0
    assert all(v[1] >= 0 for v in stages.values()) and "ntt_fwd" in stages
    for h in (ct, g1, g2, d):
        H.hear_ciphertext_destroy(h)
    H.hear_model_destroy(model)
