"""GPU parity of the skeleton CNN (hear_cnn_*) against the oracle's CNN plan.

* toy 1D / 2D CNNs (N = 2^12, 12 levels): the whole network on two samples in one batch,
  every convolution / FC strategy, bit-exact output ciphertexts, logits within 2^-15;
* the paper-shaped 1D-CNN-64 (N = 2^15, 2 x 32 x 15 inputs) at full size: two samples
  batched, the oracle recomputes the second; logits of both within 2^-15;
* single punctured convolutional layers of the Table 1 microbenchmark (N = 2^14), ordinary
  and fast: sampled output ciphertexts (first and last) bit-exact, every output within
  2^-15 of the plain convolution.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import cnn as OC
from oracle import oracle as O
from paper_2104_09164_gb300.workloads import (CONV_BENCH_PARAMS, _conv_same, cnn_forward, cnn_spec,
                                              conv_bench_layer, make_cnn)

pytestmark = pytest.mark.gpu

LOGIT_TOL = 2.0 ** -15


@pytest.fixture(scope="module")
def H():
    from paper_2104_09164_gb300.build import build
    build()
    from paper_2104_09164_gb300 import hear
    return hear


def _check_ops(H, m, ops):
    info = H.hear_cnn_ops(m)
    kinds = {"diag": 1, "pack": 2, "rotsum": 3, "quad": 4, "bias": 5}
    assert [i["kind"] for i in info] == [kinds[op[0]] for op in ops]
    for i, op in zip(info, ops):
        if op[0] == "diag":
            assert i["n_out"] == op[1]


def _network(H, name, strategies, n_samples, oracle_samples):
    net = make_cnn(name, n_samples=n_samples)
    spec = cnn_spec(net)               # as trained: the library collapses it
    ospec = OC.collapse(spec)          # the oracle collapses it on its own
    S = net.slots
    ops, out = OC.build_plan(ospec, S, strategies)
    ctx = H.hear_context_create(net.log_n, net.q_bits, net.p_bits, net.log2_scale, net.sigma, 0)
    m = H.hear_cnn_create(ctx, spec, strategies)
    try:
        _check_ops(H, m, ops)
        steps = H.hear_cnn_rotations(m)
        assert steps == OC.plan_rotations(ops, S)
        assert H.hear_cnn_output_slots(m) == out
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        cts = [H.hear_cnn_encrypt(ctx, pk, m, clip, 401, s)[0] for s, clip in enumerate(net.clips)]
        outs = H.hear_cnn_evaluate(m, evk, 0, len(ops), cts, n_samples)
        for s, clip in enumerate(net.clips):
            dec = H.hear_decrypt(ctx, sk, outs[s])
            assert np.max(np.abs(np.asarray(dec)[out] - cnn_forward(net, clip))) <= LOGIT_TOL
        o = O.Oracle(net.log_n, net.q_bits, net.p_bits, net.sigma, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        pool = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)
        for s in oracle_samples:
            ct = o.encrypt(keys.pk, OC.pack_input(ospec, net.clips[s], S), 401, s, 2.0 ** net.log2_scale)
            r = OC.evaluate(o, ops, [ct], keys, pool)[0]
            lv, npoly, sc = H.hear_ciphertext_info(outs[s])
            assert (lv, npoly) == (r.level, 2) and sc == r.scale
            assert np.array_equal(H.hear_ciphertext_export(outs[s]), o.to_coeff(r)), s
        for h in cts + outs:
            H.hear_ciphertext_destroy(h)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_cnn_destroy(m)
        H.hear_context_destroy(ctx)


@pytest.mark.parametrize("name", ["cnn_toy", "cnn2d_toy"])
@pytest.mark.parametrize("strategy", [None, "full", "baby", "giant", ("hybrid", 2)])
def test_toy_cnn_bit_exact(H, name, strategy):
    _network(H, name, None if strategy is None else [strategy] * 4, 2, [0, 1])


def test_cnn1d64_full_size(H):
    _network(H, "cnn1d64", None, 2, [1])


@pytest.mark.parametrize("idx", [1, 4])
@pytest.mark.parametrize("fast", [False, True])
def test_table1_layer_sampled(H, idx, fast):
    spec, xs = conv_bench_layer(idx, fast)
    log_n, qb, pb = CONV_BENCH_PARAMS
    S = xs.shape[2]
    ops, _ = OC.build_plan(spec, S)
    ctx = H.hear_context_create(log_n, qb, pb, 40.0, 3.2, 0)
    m = H.hear_cnn_create(ctx, spec)
    try:
        _check_ops(H, m, ops)
        steps = H.hear_cnn_rotations(m)
        assert steps == OC.plan_rotations(ops, S)
        sk, pk, evk = H.hear_keygen(ctx, 301, steps)
        cts = [H.hear_encrypt(ctx, pk, xs[0][i], 2.0 ** 40, 401, i) for i in range(xs.shape[1])]
        outs = H.hear_cnn_evaluate(m, evk, 0, len(ops), cts, 1)
        # every output against the plain convolution of the punctured maps
        lay = OC.input_layout(spec, S)
        dims = spec["conv_dims"]
        inmap = OC.channel_maps(lay, xs[0])
        ref = _conv_same(inmap if dims == 2 else inmap[:, 0, :], spec["layers"][0][1], dims)
        olay = OC.Layout(S, lay.dist, lay.h, lay.w, lay.pitch, lay.stride, len(outs),
                         lambda i, mm, p, cb=lay.cbar: cb * i + mm, lay.cbar)
        got = OC.channel_maps(olay, [np.asarray(H.hear_decrypt(ctx, sk, h)) for h in outs])
        assert np.max(np.abs((got if dims == 2 else got[:, 0, :]) - ref)) <= LOGIT_TOL
        # sampled outputs bit-exact against the oracle
        o = O.Oracle(log_n, qb, pb, 3.2, threads=os.cpu_count() or 0)
        keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in steps])
        pool = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)
        x = [o.encrypt(keys.pk, xs[0][i], 401, i, 2.0 ** 40) for i in range(xs.shape[1])]
        n_out = len(outs)
        for op in ops:
            if op[0] == "pack":
                x = OC.pack(o, x, op[1], op[2], op[3], keys)
            elif op[0] == "diag":
                full = OC.diag_layer(o, x, op[1], op[2], keys, pool, only_j=0)
                last = OC.diag_layer(o, x, op[1], op[2], keys, pool, only_j=n_out - 1)
                x = {0: full[0], n_out - 1: last[n_out - 1]}
            elif op[0] == "rotsum":
                x = {j: OC.rotsum(o, c, op[1], keys) for j, c in x.items()}
        for j, r in x.items():
            assert H.hear_ciphertext_info(outs[j])[2] == r.scale
            assert np.array_equal(H.hear_ciphertext_export(outs[j]), o.to_coeff(r)), j
        for h in cts + outs:
            H.hear_ciphertext_destroy(h)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
    finally:
        H.hear_cnn_destroy(m)
        H.hear_context_destroy(ctx)


def test_autotuned_strategies_bit_exact(H):
    """the tuner's per-layer choice evaluates bit-exactly like the oracle with that choice"""
    from paper_2104_09164_gb300.autotune import tune_cnn
    net = make_cnn("cnn_toy", n_samples=2)
    spec = cnn_spec(net)
    ctx = H.hear_context_create(net.log_n, net.q_bits, net.p_bits, net.log2_scale, net.sigma, 0)
    try:
        strategies, report = tune_cnn(H, ctx, spec, net.slots, len(net.q_bits) - 1, iters=2)
    finally:
        H.hear_context_destroy(ctx)
    assert len(report) == 3 and all(r["best"] in r["ms"] for r in report)
    _network(H, "cnn_toy", strategies, 2, [0])


def test_cnn_rejects_bad_inputs(H):
    """errors come back as status codes: a fast convolution on a dense input, channel counts
    that do not fill the blocks, missing rotation keys, inputs at the wrong level"""
    net = make_cnn("cnn_toy", n_samples=1)
    spec = cnn_spec(net)
    ctx = H.hear_context_create(net.log_n, net.q_bits, net.p_bits, net.log2_scale, net.sigma, 0)
    try:
        bad = dict(spec, layers=[("conv", spec["layers"][0][1], True)] + spec["layers"][1:])
        with pytest.raises(H.HearError) as e:
            H.hear_cnn_create(ctx, bad)
        assert e.value.code == -1
        W = spec["layers"][0][1]
        with pytest.raises(H.HearError):
            H.hear_cnn_create(ctx, dict(spec, layers=[("conv", W[:6], False)]))
        m = H.hear_cnn_create(ctx, spec)
        sk, pk, evk = H.hear_keygen(ctx, 301, H.hear_cnn_rotations(m)[:3])
        ct = H.hear_cnn_encrypt(ctx, pk, m, net.clips[0], 401, 0)
        with pytest.raises(H.HearError) as e:
            H.hear_cnn_evaluate(m, evk, 0, len(H.hear_cnn_ops(m)), ct, 1)
        assert e.value.code == -6
        low = H.hear_ciphertext_drop_level(ct[0], 3)
        with pytest.raises(H.HearError) as e:
            H.hear_cnn_evaluate(m, evk, 0, 1, [low], 1)
        assert e.value.code == -4
        for h in ct + [low]:
            H.hear_ciphertext_destroy(h)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
        H.hear_cnn_destroy(m)
    finally:
        H.hear_context_destroy(ctx)
