"""CPU pins of the oracle's CNN part (oracle/cnn.py) and of the network collapse (the
oracle's own, and the library's host-only one, which must agree to the bit).

The plan builder (slot layouts, convolution plaintexts of Eq. conv, the fast
convolution's packing and phase sums, pooling, global pooling, the FC on pooled features)
is pinned by running its plan on plain slot vectors against a plain FP64 convolutional
network written directly from the network description; the encrypted primitives it adds
(plaintext addition, level drop, the Horner-form quadratic, the generic diagonal
operation, packing) are pinned against exact residue identities and against the plain
simulation."""
import os

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import cnn as OC
from oracle import oracle as O
from paper_2104_09164_gb300.workloads import (TABLE1_LAYERS, _conv_same, cnn_forward, cnn_spec,
                                              conv_bench_layer, make_cnn)

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def toy():
    o = O.Oracle(12, [60] + [40] * 4, [60, 60], 3.2)
    S = o.n // 2
    rng = np.random.default_rng(5)
    steps = [1, 3, 64, 100, S - 1, S - 64, 512]
    keys = o.keygen(17, [O.galois_for_step(s, o.n) for s in steps])
    return o, keys, rng


def test_add_plain_is_exact(toy):
    o, keys, rng = toy
    S = o.n // 2
    ct = o.encrypt(keys.pk, rng.uniform(-1, 1, S), 3, 0, 2.0 ** 40)
    m, _ = o.encode(rng.uniform(-1, 1, S), 2.0 ** 40)
    pt = np.empty((ct.level + 1, o.n), dtype=np.uint64)
    for t in range(ct.level + 1):
        q = o.q[t]
        pt[t] = [int(v) % q for v in m]
    pt = o.ntt_fwd(pt, list(range(ct.level + 1)))
    r0 = o.decrypt_residues(keys, ct)
    r1 = o.decrypt_residues(keys, o.add_plain(ct, pt))
    for t in range(ct.level + 1):
        q = o.q[t]
        assert np.array_equal((r1[t].astype(object) - r0[t].astype(object)) % q,
                              np.array([int(v) % q for v in m], dtype=object))


def test_drop_level_keeps_the_residues(toy):
    o, keys, rng = toy
    S = o.n // 2
    ct = o.encrypt(keys.pk, rng.uniform(-1, 1, S), 3, 1, 2.0 ** 40)
    d = o.drop_level(ct)
    assert d.level == ct.level - 1 and d.scale == ct.scale
    assert np.array_equal(o.decrypt_residues(keys, d), o.decrypt_residues(keys, ct)[:ct.level])


def test_quad_matches_fp64(toy):
    o, keys, rng = toy
    S = o.n // 2
    x = rng.uniform(-1, 1, S)
    A, B, C = rng.uniform(-1, 1, S), rng.uniform(-1, 1, S), rng.uniform(-1, 1, S)
    ct = o.encrypt(keys.pk, x, 3, 2, 2.0 ** 40)
    r = OC.quad(o, ct, A, B, C, keys)
    assert r.level == ct.level - 2
    got = o.decrypt(keys, r)
    assert np.max(np.abs(got - (A * x * x + B * x + C))) < 2.0 ** -20


def test_diag_layer_matches_plain_rotations(toy):
    """random terms on two inputs / two outputs, every split kind (b only, g only, both)"""
    o, keys, rng = toy
    S = o.n // 2
    xs = [rng.uniform(-1, 1, S) for _ in range(2)]
    cts = [o.encrypt(keys.pk, x, 3, 10 + i, 2.0 ** 40) for i, x in enumerate(xs)]
    splits = [(0, 0), (1, 0), (3, 0), (0, 64), (1, 64), (S - 1, 512), (100, 0), (0, S - 64)]
    terms = {}
    for i in range(2):
        for j in range(2):
            for b, g in splits:
                terms[(i, j, b, g)] = rng.uniform(-1, 1, S)
    outs = OC.diag_layer(o, cts, 2, terms, keys, ThreadPoolExecutor(4))
    ref = OC.simulate([("diag", 2, terms)], xs)
    for j in range(2):
        assert outs[j].level == cts[0].level - 1
        assert np.max(np.abs(o.decrypt(keys, outs[j]) - ref[j])) < 2.0 ** -20


@pytest.mark.parametrize("name", ["cnn_toy", "cnn2d_toy", "cnn1d64", "cnn2d64"])
@pytest.mark.parametrize("strategy", [None, "full", "baby", "giant", ("hybrid", 2)])
def test_plan_on_plain_slots_equals_fp64_network(name, strategy):
    net = make_cnn(name, n_samples=1)
    spec = OC.collapse(cnn_spec(net))
    S = net.slots
    ops, out = OC.build_plan(spec, S, None if strategy is None else [strategy] * 4)
    got = OC.simulate(ops, [OC.pack_input(spec, net.clips[0], S)])[0][out]
    ref = cnn_forward(net, net.clips[0])
    assert np.max(np.abs(got - ref)) < 1e-12


def test_library_collapse_equals_the_oracle_collapse():
    """the library's collapse (hear_cnn_collapse, host only) and the oracle's, from the
    same trained network, give the same doubles bit for bit (the encoded plaintexts depend
    on every bit), and a deliberately different order of the same formula does not"""
    pytest.importorskip("ctypes")
    from paper_2104_09164_gb300 import hear as H
    def flat(collapsed):
        out = []
        for layer in collapsed["layers"]:
            if layer[0] in ("conv", "fc"):
                out.append(np.asarray(layer[1], dtype=np.float64).ravel())
            elif layer[0] == "quad":
                out += [np.asarray(v, dtype=np.float64).ravel() for v in layer[1:4]]
        return np.concatenate(out)

    for name in ("cnn_toy", "cnn2d_toy", "cnn1d64", "cnn2d64"):
        spec = cnn_spec(make_cnn(name, n_samples=1))
        got = H.hear_cnn_collapse(spec)
        want = flat(OC.collapse(spec))
        assert got.shape == want.shape
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        # an already-collapsed network passes through the library's collapse unchanged
        coll = OC.collapse(spec)
        assert np.array_equal(H.hear_cnn_collapse(coll).view(np.uint64), want.view(np.uint64))
    # B = 2 a s t + b s formed as 2 a (s t) + b s instead differs in some bits: the order matters
    cv = make_cnn("cnn2d64", n_samples=1).convs[1]
    s = cv["gamma"] / np.sqrt(cv["var"] + 1e-5)
    t = s * (cv["bias"] - cv["mean"]) + cv["beta"]
    a, b, _ = cv["act"]
    assert not np.array_equal(2.0 * a * s * t + b * s, 2.0 * a * (s * t) + b * s)


def test_collapse_keeps_the_network():
    """collapsed form evaluated plainly (no slots) = the uncollapsed network"""
    for name in ("cnn_toy", "cnn2d64"):
        net = make_cnn(name, n_samples=2)
        spec = OC.collapse(cnn_spec(net))
        dims = spec["conv_dims"]
        for clip in net.clips:
            h = clip.reshape(2, -1) if dims == 1 else clip
            for layer in spec["layers"]:
                if layer[0] == "conv":
                    h = _conv_same(h, layer[1], dims)
                elif layer[0] == "quad":
                    sh = (-1,) + (1,) * (h.ndim - 1)
                    a, b, c = (np.asarray(v).reshape(sh) for v in layer[1:4])
                    h = a * h * h + b * h + c
                elif layer[0] == "pool":
                    if dims == 1:
                        L = h.shape[1] // 2
                        h = h[:, 0:2 * L:2] + h[:, 1:2 * L:2]
                    else:
                        H, W = h.shape[1] // 2, h.shape[2] // 2
                        h = (h[:, 0:2 * H:2, 0:2 * W:2] + h[:, 1:2 * H:2, 0:2 * W:2] +
                             h[:, 0:2 * H:2, 1:2 * W:2] + h[:, 1:2 * H:2, 1:2 * W:2])
                elif layer[0] == "gap":
                    h = h.reshape(h.shape[0], -1).sum(axis=1)
                elif layer[0] == "fc":
                    h = layer[1] @ h + layer[2]
            assert np.max(np.abs(h - cnn_forward(net, clip))) < 1e-12


def _table1():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_conv_shapes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            net, layer, mp, filt, n_in, n_out, n_p = line.split()
            rows.append((net, layer, mp, int(filt), int(n_in), int(n_out), int(n_p)))
    return rows


def test_table1_ciphertext_counts_and_load_numbers():
    """N = 2^14: n_in, n_out and the load number n_P of every Table 1 layer"""
    gold = _table1()
    assert len(gold) == len(TABLE1_LAYERS)
    for idx, row in enumerate(gold):
        spec, xs = conv_bench_layer(idx, True)
        net, layer, dims, (h, w), pitch, stride, c_in, c_out = TABLE1_LAYERS[idx]
        assert (net, layer) == row[:2] and c_out == row[3]
        assert row[2] == (str(w) if dims == 1 else "%dx%d" % (h, w))
        ops, _ = OC.build_plan(spec, xs.shape[2])
        pack = [op for op in ops if op[0] == "pack"][0]
        diag = [op for op in ops if op[0] == "diag"][0]
        assert xs.shape[1] == row[4] and diag[1] == row[5] and pack[2] == row[6]


@pytest.mark.parametrize("idx", range(len(TABLE1_LAYERS)))
def test_punctured_conv_layer_equals_fp64(idx):
    """ordinary and fast convolution of a punctured input (junk between the valid
    positions) = plain same-padded convolution of the maps; the fast form takes n_P
    products and n_P - 1 rotations per packed ciphertext before, log2(n_P) rotations after"""
    for fast in (False, True):
        spec, xs = conv_bench_layer(idx, fast)
        S = xs.shape[2]
        lay = OC.input_layout(spec, S)
        ops, _ = OC.build_plan(spec, S)
        y = OC.simulate(ops, list(xs[0]))
        dims = spec["conv_dims"]
        inmap = OC.channel_maps(lay, xs[0])
        ref = _conv_same(inmap if dims == 2 else inmap[:, 0, :], spec["layers"][0][1], dims)
        olay = OC.Layout(S, lay.dist, lay.h, lay.w, lay.pitch, lay.stride, len(y),
                         lambda i, m, p, cb=lay.cbar: cb * i + m, lay.cbar)
        got = OC.channel_maps(olay, y)
        assert np.max(np.abs((got if dims == 2 else got[:, 0, :]) - ref)) < 1e-12
        if fast:
            pack = [op for op in ops if op[0] == "pack"][0]
            n_p, offs = pack[2], pack[3]
            assert len([o for o in offs if o]) == n_p - 1
            post = ops[-1]
            assert post[0] == "rotsum" and len(post[1]) == int(np.log2(n_p))


def test_encrypted_toy_cnn_matches_fp64():
    net = make_cnn("cnn_toy", n_samples=1)
    spec = OC.collapse(cnn_spec(net))
    S = net.slots
    ops, out = OC.build_plan(spec, S)
    assert OC.plan_depth(ops) == len(net.q_bits) - 1
    o = O.Oracle(net.log_n, net.q_bits, net.p_bits, net.sigma)
    keys = o.keygen(301, [O.galois_for_step(s, o.n) for s in OC.plan_rotations(ops, S)])
    ct = o.encrypt(keys.pk, OC.pack_input(spec, net.clips[0], S), 401, 0, 2.0 ** 40)
    r = OC.evaluate(o, ops, [ct], keys)
    assert len(r) == 1 and r[0].level == 0
    dec = o.decrypt(keys, r[0])
    assert np.max(np.abs(dec[out] - cnn_forward(net, net.clips[0]))) < 2.0 ** -15
    assert np.max(np.abs(dec - OC.simulate(ops, [OC.pack_input(spec, net.clips[0], S)])[0])) < 2.0 ** -15


def test_autotune_layer_geometry_matches_the_network_plan():
    """the single-layer specs the tuner times have the layouts and level drops the layers
    have inside the network (compared with the oracle's network plan)"""
    from paper_2104_09164_gb300.autotune import candidates, conv_layer_specs
    for name in ("cnn_toy", "cnn2d64"):
        net = make_cnn(name, n_samples=1)
        spec = OC.collapse(cnn_spec(net))
        S = net.slots
        ops, _ = OC.build_plan(spec, S)
        depth_before = []
        used = 0
        for op in ops:
            if op[0] in ("pack", "diag"):
                depth_before.append(used)
            used += {"diag": 1, "pack": 1, "quad": 2}.get(op[0], 0)
        diags = [op for op in ops if op[0] == "diag"][:-1]      # the convolutions (last = FC)
        singles = conv_layer_specs(spec)
        assert len(singles) == len(diags)
        k = 0
        for (si, used_before, single), diag in zip(singles, diags):
            sops, _ = OC.build_plan(single, S)
            sdiag = [op for op in sops if op[0] == "diag"][0]
            assert sdiag[1] == diag[1]
            assert sorted(sdiag[2].keys()) == sorted(diag[2].keys())
            for key in diag[2]:
                assert np.allclose(sdiag[2][key], diag[2][key])
            assert used_before == depth_before[k]
            k += 2 if single["layers"][0][2] else 1
    assert candidates(32) == ["full", "baby", "giant", ("hybrid", 2), ("hybrid", 4), ("hybrid", 8),
                              ("hybrid", 16)]


def test_fc_form_candidates():
    """the FC-form candidates bracket the default baby-step count of the widest FC layer"""
    from paper_2104_09164_gb300.autotune import fc_candidates
    from paper_2104_09164_gb300.workloads import make_workload
    assert fc_candidates(make_workload("small").layers) == [(n, d, h) for n in (8, 16, 32) for d in (False, True)
                                                            for h in (False, True)]
    assert fc_candidates(make_workload("large").layers) == [(n, d, h) for n in (16, 32, 64) for d in (False, True)
                                                            for h in (False, True)]
