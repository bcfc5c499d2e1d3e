"""Strategy autotuning: the per-layer rotation split of the encrypted skeleton CNN and the FC
evaluation form of the FC / x^2 networks.

Every convolution of Eq. (conv) can split its rotations r_k + dist*l into a hoisted baby
step and a giant step applied to the summed products in several ways -- the full-step,
giant-step and baby-step strategies of the paper (Methods, "Algorithmic and cryptographic
optimizations") and the hybrid splits between them -- and which is fastest depends on the
numbers of input and output ciphertexts.  ``tune_cnn`` times each candidate on the GPU for
each convolutional layer at the geometry and level the layer has inside the network, on
random inputs with throw-away keys, and returns the fastest per layer.  Every candidate
computes the same convolution (bit-exact against the oracle with that strategy).

Host logic only: all timing goes through the C ABI (``hear.py``).
"""
import time

import numpy as np


def conv_layer_specs(spec):
    """[(index among the conv / FC layers, level drop before it, single-layer spec)] for every
    convolution of a network (as trained or collapsed): the map geometry, channel count and
    puncture at the layer's input; the level drop counts the levels the network consumes
    before the layer (timing only: the weights' pooling factors do not matter here)."""
    dims = spec["conv_dims"]
    c, h, w = spec["c_in"], spec["h"], spec["w"]
    pitch = spec.get("pitch") or w
    stride = spec.get("stride", 1)
    used = 0
    out = []
    si = 0
    for layer in spec["layers"]:
        kind = layer[0]
        if kind == "conv":
            single = {"conv_dims": dims, "c_in": c, "h": h, "w": w,
                      "pitch": w if dims == 1 else pitch, "stride": stride,
                      "layers": [("conv", layer[1], layer[2])]}
            out.append((si, used, single))
            si += 1
            used += 2 if layer[2] else 1
            c = layer[1].shape[0]
        elif kind in ("quad", "bn_quad"):
            used += 2
        elif kind in ("pool", "avgpool"):
            stride *= 2
            w //= 2
            if dims == 2:
                h //= 2
        elif kind == "fc":
            si += 1
            used += 1
    return out


def candidates(lr):
    """strategies for a convolution whose block shifts span lr ciphertext blocks"""
    c = ["full", "baby", "giant"]
    n1 = 2
    while n1 < lr:
        c.append(("hybrid", n1))
        n1 *= 2
    return c


def _block_shifts(H, ctx, single, level):
    """block shifts of the layer = number of giant steps of its baby-step split"""
    m = H.hear_cnn_create(ctx, dict(single, level=level), ["baby"])
    try:
        diag = [o for o in H.hear_cnn_ops(m) if o["kind"] == H.HEAR_CNN_OP_DIAG][0]
        return diag["n_giants"]
    finally:
        H.hear_cnn_destroy(m)


def time_layer(H, ctx, single, level, strategy, slots, n_samples=1, iters=3, stream=None, seed=7):
    """median device ms of the whole single-layer plan (pack / conv / phase sums) on random
    input ciphertexts at `level`, throw-away keys"""
    import torch
    m = H.hear_cnn_create(ctx, dict(single, level=level), [strategy])
    try:
        ops = H.hear_cnn_ops(m)
        sk, pk, evk = H.hear_keygen(ctx, 9001, H.hear_cnn_rotations(m))
        n_in = ops[0]["n_in"]
        rng = np.random.default_rng(seed)
        st = stream if stream is not None else torch.cuda.current_stream()
        cts = []
        for k in range(n_samples * n_in):
            top = H.hear_encrypt(ctx, pk, rng.uniform(-1.0, 1.0, slots), 2.0 ** 40, 9002, k, st)
            cts.append(H.hear_ciphertext_drop_level(top, ops[0]["level_in"], st))
            H.hear_ciphertext_destroy(top)
        for o in H.hear_cnn_evaluate(m, evk, 0, len(ops), cts, n_samples, st):
            H.hear_ciphertext_destroy(o)
        times = []
        for _ in range(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            outs = H.hear_cnn_evaluate(m, evk, 0, len(ops), cts, n_samples, st)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            for o in outs:
                H.hear_ciphertext_destroy(o)
        for h in cts:
            H.hear_ciphertext_destroy(h)
        H.hear_eval_keys_destroy(evk)
        H.hear_public_key_destroy(pk)
        H.hear_secret_key_destroy(sk)
        times.sort()
        return times[len(times) // 2]
    finally:
        H.hear_cnn_destroy(m)


def tune_cnn(H, ctx, spec, slots, top_level, n_samples=1, iters=3, stream=None):
    """-> (strategies for hear_cnn_create, report) with the fastest candidate per conv layer
    (FC layers keep the default); `top_level` = the level of the network's input"""
    n_tunable = sum(1 for layer in spec["layers"] if layer[0] in ("conv", "fc"))
    strategies = [None] * n_tunable
    report = []
    for si, used, single in conv_layer_specs(spec):
        level = top_level - used
        lr = _block_shifts(H, ctx, single, level)
        t0 = time.perf_counter()
        timed = [(time_layer(H, ctx, single, level, cand, slots, n_samples, iters, stream), cand)
                 for cand in candidates(lr)]
        timed.sort(key=lambda t: t[0])
        strategies[si] = timed[0][1]
        report.append({"layer": si, "level": level, "block_shifts": lr,
                       "ms": {_name(c): t for t, c in timed}, "best": _name(timed[0][1]),
                       "tune_s": time.perf_counter() - t0})
    return strategies, report


def _name(s):
    return s if isinstance(s, str) else "%s(%d)" % s


# ---------------------------------------------------------------- FC evaluation form
def fc_candidates(layers):
    """(fc_n1, hoist_moddown, hoist_sums) forms to try for a network of FC / x^2 layers:
    baby-step counts d/2, d and 2d around d = the smallest power of two with d^2 >= D of the
    widest FC (D = its output dimension; each layer clamps n1 to its own D), each with and
    without hoisted ModDown of the babies and with and without hoisted sums"""
    D = max(layer[1].shape[0] for layer in layers if layer[0] == "fc")
    d = 1
    while d * d < D:
        d *= 2
    n1s = sorted({max(2, d // 2), d, min(2 * d, D)})
    return [(n1, dh, hs) for n1 in n1s for dh in (False, True) for hs in (False, True)]


def tune_fc(H, ctx, layers, clip_dim, n_ct, slots, level=None, steps=3, warmup=1, stream=None, seed=7):
    """-> ((fc_n1, hoist_moddown, hoist_sums), report): the fastest FC evaluation form (Methods,
    "Algorithmic and cryptographic optimizations": the baby-step / giant-step split and where
    the ModDown of the hoisted rotations happens) for whole-network evaluations of n_ct
    ciphertexts, timed through the C ABI (CUDA-graph replay, CUDA events on `stream`) on random
    inputs with throw-away keys (one key set per baby-step count: the forms of one count
    need the same rotations).  Every form computes the same network; the oracle evaluates
    each one bit-exactly."""
    import torch
    st = stream if stream is not None else torch.cuda.Stream()
    rng = np.random.default_rng(seed)
    report = []
    by_n1 = {}
    for n1, dh, hs in fc_candidates(layers):
        by_n1.setdefault(n1, []).append((dh, hs))
    for n1, forms in by_n1.items():
        t0 = time.perf_counter()
        models = [H.hear_model_create(ctx, layers, clip_dim, level, fc_n1=n1, hoist_moddown=dh, hoist_sums=hs)
                  for dh, hs in forms]
        try:
            sk, pk, evk = H.hear_keygen(ctx, 9001, H.hear_model_rotations(models[0]))
            cts = []
            for i in range(n_ct):
                c = H.hear_encrypt(ctx, pk, rng.uniform(-1.0, 1.0, slots), 2.0 ** 40, 9002, i, st)
                if level is not None:
                    low = H.hear_ciphertext_drop_level(c, level, st)
                    H.hear_ciphertext_destroy(c)
                    c = low
                cts.append(c)
            setup_s = time.perf_counter() - t0
            for m, (dh, hs) in zip(models, forms):
                t1 = time.perf_counter()
                for _ in range(warmup):
                    for o in H.hear_evaluate(m, evk, cts, st):
                        H.hear_ciphertext_destroy(o)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(steps):
                    for o in H.hear_evaluate(m, evk, cts, st):
                        H.hear_ciphertext_destroy(o)
                e1.record(st)
                torch.cuda.synchronize()
                report.append({"fc_n1": n1, "hoist_moddown": dh, "hoist_sums": hs, "ms": e0.elapsed_time(e1) / steps,
                               "tune_s": time.perf_counter() - t1 + setup_s / len(forms)})
            for c in cts:
                H.hear_ciphertext_destroy(c)
            H.hear_eval_keys_destroy(evk)
            H.hear_public_key_destroy(pk)
            H.hear_secret_key_destroy(sk)
        finally:
            for m in models:
                H.hear_model_destroy(m)
    best = min(report, key=lambda r: r["ms"])
    return (best["fc_n1"], best["hoist_moddown"], best["hoist_sums"]), report
