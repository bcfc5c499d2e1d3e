"""Pins of the oracle's slot-batched evaluation (one clip per slot, one ciphertext per
feature) against things other than itself: the general slot encoder, closed-form matrix
products and the FP64 network, and the independence of the slots.  CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_09164_gb300.workloads import make_workload

THREADS = os.cpu_count() or 0


@pytest.fixture(scope="module")
def toy():
    w = make_workload("toy", n_clips=300)
    o = O.Oracle(w.log_n, w.q_bits, w.p_bits, w.sigma, threads=THREADS)
    keys = o.keygen(11, [])
    return w, o, keys


def test_constant_slot_vector_encodes_to_the_scalar(toy):
    """the general encoder (double-double inverse canonical embedding) maps the constant
    vector w to the constant polynomial whose coefficient is the scalar's integer"""
    w, o, _ = toy
    slots = o.n // 2
    rng = np.random.default_rng(5)
    vals = list(rng.normal(0.0, 0.3, size=12)) + [0.0, -0.0, 1.0, -1.0, 3.0 / o.q[2], -2.0 / o.q[1]]
    for level in (1, 2):
        res = o.scalar_residues(np.array(vals), level)
        for v, r in zip(vals, res):
            m, ties = o.encode(np.full(slots, v), float(o.q[level]))
            assert ties == 0
            assert np.all(m[1:] == 0)
            f = Fraction(float(v)) * o.q[level]
            assert abs(Fraction(int(m[0])) - f) <= Fraction(1, 2)
            assert [int(m[0]) % q for q in o.q[:level + 1]] == [int(x) for x in r]
    # w = +-0.5 times an odd q_l is an exact half-integer: ties round away from zero
    for level in (1, 2):
        ql = o.q[level]
        r = o.scalar_residues(np.array([0.5, -0.5, 1.5]), level)
        assert [int(x) for x in r[0]] == [((ql + 1) // 2) % q for q in o.q[:level + 1]]
        assert [int(x) for x in r[1]] == [(-((ql + 1) // 2)) % q for q in o.q[:level + 1]]
        assert [int(x) for x in r[2]] == [((3 * ql + 1) // 2) % q for q in o.q[:level + 1]]


def test_mul_scalar_is_mulplain_with_the_encoded_constant(toy):
    w, o, keys = toy
    slots = o.n // 2
    rng = np.random.default_rng(6)
    ct = o.encrypt(keys.pk, rng.uniform(-1, 1, slots), 21, 0, 2.0 ** 40)
    for v in (0.37, -0.81, 0.0):
        pt = o.encode_pt(np.full(slots, v), float(o.q[ct.level]), ct.level)
        a = o.mul_scalar(ct, o.scalar_residues(v, ct.level), float(o.q[ct.level]))
        b = o.mulplain(ct, pt, float(o.q[ct.level]))
        assert np.array_equal(a.data, b.data) and a.scale == b.scale


def test_fc_simd_decrypts_to_the_matrix_product(toy):
    w, o, keys = toy
    n_clips = 37
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, size=(n_clips, 8))
    W = rng.normal(0.0, 0.3, size=(5, 8))
    cts = o.encrypt_simd(keys.pk, X, 22, 2.0 ** 40)
    assert len(cts) == 8
    y = o.fc_simd(cts, W)
    assert len(y) == 5 and all(c.level == o.L - 1 for c in y)
    dec = np.stack([o.decrypt(keys, c) for c in y], axis=1)          # [slots][5]
    assert np.max(np.abs(dec[:n_clips] - X @ W.T)) < 2.0 ** -20
    assert np.max(np.abs(dec[n_clips:])) < 2.0 ** -20                # empty slots stay empty
    # a transposed or mis-indexed weight matrix would not pass
    assert np.max(np.abs(dec[:n_clips, :5] - X[:, :5] @ W[:, :5].T)) > 2.0 ** -10


def test_network_simd_matches_fp64(toy):
    """toy network FC 64->16 -> x^2 -> FC 16->2 (collapsed), 300 clips in the slots"""
    w, o, keys = toy
    cts = o.encrypt_simd(keys.pk, w.clips, 23, 2.0 ** 40)
    out = o.evaluate_simd(w.layers, cts, keys)
    assert len(out) == 2 and out[0].level == o.L - 2
    logits = o.decrypt_simd(keys, out, w.n_clips)
    ref = w.fp64_forward(w.clips)
    assert np.max(np.abs(logits - ref)) <= 2.0 ** -15


def test_simd_slots_are_independent(toy):
    """changing one clip changes only its own slot of every output"""
    w, o, keys = toy
    X = np.array(w.clips[:20])
    W = np.random.default_rng(8).normal(0.0, 0.2, size=(3, 64))
    a = o.decrypt_simd(keys, o.fc_simd(o.encrypt_simd(keys.pk, X, 24, 2.0 ** 40), W), 20)
    X2 = X.copy()
    X2[4] = -X2[4]
    b = o.decrypt_simd(keys, o.fc_simd(o.encrypt_simd(keys.pk, X2, 24, 2.0 ** 40), W), 20)
    keep = np.arange(20) != 4
    assert np.max(np.abs(a[keep] - b[keep])) < 2.0 ** -25
    assert np.max(np.abs(b[4] - X2[4] @ W.T)) < 2.0 ** -20


def test_fc_square_fc_simd_matches_fp64():
    """separate FC -> x^2 -> FC layers (three levels: q = 50 + 3x40 bits), 50 clips, ragged
    dimensions; every clip's logits within 2^-15 of FP64, the unused slots stay empty"""
    o = O.Oracle(12, [50, 40, 40, 40], [50], 3.2, threads=THREADS)
    keys = o.keygen(12, [])
    rng = np.random.default_rng(13)
    X = rng.uniform(-1, 1, size=(50, 16))
    W1, W2 = rng.normal(0, 0.2, size=(6, 16)), rng.normal(0, 0.4, size=(3, 6))
    layers = [("fc", W1), ("square",), ("fc", W2)]
    out = o.evaluate_simd(layers, o.encrypt_simd(keys.pk, X, 25, 2.0 ** 40), keys)
    assert len(out) == 3 and out[0].level == 0
    ref = ((X @ W1.T) ** 2) @ W2.T
    assert np.max(np.abs(o.decrypt_simd(keys, out, 50) - ref)) <= 2.0 ** -15
    assert np.max(np.abs(o.decrypt(keys, out[0])[50:])) <= 2.0 ** -15
