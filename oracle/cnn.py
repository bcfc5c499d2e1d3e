"""CNN part of the CPU oracle: multi-channel homomorphic convolution (ordinary and fast,
merge-and-conquer), average and global average pooling, the FC layer on pooled features
and the general quadratic activation A*x^2 + B*x + C per feature map.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module.  It shares no code with the CUDA
library; it composes the primitives of ``oracle.Oracle``.

Slot layout (Methods, "Notation", "Multi-channel homomorphic convolutions", "Data
encryption"): the N/2 slots of a ciphertext are cut into cbar = N/2 / dist blocks of dist
slots; block m holds one channel as a row-major map (row pitch P slots).  A map punctured
by pooling keeps position (y, x) at offset stride*(y*P + x) of its block.  The input
ciphertext holds copies of the c_in input planes: block m carries plane m mod c_in.  With
c >= cbar channels, ciphertext i block m carries channel cbar*i + m.

A network as trained (convolutions, bias + batch normalisation + quadratic activation,
average pooling, global average pooling, FC) is first collapsed by ``collapse`` (Methods,
"Non-convolutional layers"); the collapsed network becomes a *plan*,
a list of slot-level operations on the ciphertexts of one sample:

  ("diag", n_out, terms)   terms {(i, j, b, g): z}: output j receives z (.) rho^(b+g)(x_i).
        Evaluated as out_j = rescale(sum_g rho^g(sum_(i,b) Enc(rho^-g(z)) (.) rho^b(x_i))):
        babies rho^b(x_i) hoisted per input ciphertext, plaintexts pre-rotated by rho^-g
        and encoded at scale q_level (level-aware encoding), giants rotated without
        hoisting, one rescale (lazy rescaling) -- Methods, "Algorithmic and cryptographic
        optimizations", the full-step / giant-step / baby-step strategies are the splits
        a = b + g with g = 0, b = dist*l, b = r_k respectively.
  ("pack", mask, n_P, offs) fast convolution step (i): out_t = sum_p rho^(-offs[p])(
        rescale(x_(t*n_P+p) (.) Enc(mask)))  (Methods, "Fast homomorphic convolutions").
  ("rotsum", steps)        x <- x + rho^s(x) for s in steps, every ciphertext (pooling,
        global pooling, fast convolution step (iii)).
  ("quad", A, B, C)        per ciphertext i: A_i x^2 + B_i x + C_i.
  ("bias", z)              x <- x + Enc(z) at the ciphertext's own scale.

Convolution terms follow Eq. (conv): for output block j, input ciphertext i, block shift
l and filter tap (u, v) the rotation is r_(u,v) + dist*l with r_(u,v) = stride*(du*P + dv)
(Eq. heconvsimple applied to a punctured map), and the plaintext holds
F[o][c][u][v] at every output position whose input position (y+du, x+dv) lies inside the
map (zero padding is carried by the plaintexts, not by the data).

``simulate`` runs a plan on plain slot vectors (np.roll for rotations); ``evaluate`` runs
it on ciphertexts.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .oracle import Ct


# ------------------------------------------------------------------ layer collapsing
def collapse(spec):
    """Layer collapsing (Methods, "Non-convolutional layers"): everything between two linear
    layers that acts per feature map is folded into one polynomial per map, and the scale
    of the average pooling is folded into the next linear layer.

    * bias + BN + activation: batch normalisation of y + bias is the affine map
      z = s*y + t with s = gamma / sqrt(var + eps) and t = s*(bias - mean) + beta; the
      activation p(z) = a z^2 + b z + c then equals A y^2 + B y + C with
      A = a s^2, B = 2 a s t + b s, C = a t^2 + b t + c (expand p(s y + t)).
    * average pooling = (1/m) x the plain window sum of m = 2 (1D) or 4 (2D) slots; the
      plain sum is what the ciphertexts compute (rotate-and-sum), and 1/m multiplies the
      next convolution's weights.  Global average pooling = 1/(h w) x the sum over the map,
      and 1/(h w) divides the FC weights (h, w = the map after the last pooling).

    IEEE double, operations in the order written above from left to right (A = (a s) s,
    B = ((2 a) s) t + b s, C = ((a t) t + b t) + c; conv weights w f, FC weights (w f)/(h w)
    with f the pooling factor still pending), which is the library's order too: the
    encoded plaintexts depend on every bit of these doubles.  Layers already in collapsed
    form ("quad", "pool", "gap") are kept as they are."""
    dims = spec["conv_dims"]
    h, w = spec["h"], spec["w"]
    out = dict(spec)
    out["layers"] = []
    factor = 1.0          # pending 1/m of average poolings
    divisor = 1.0         # pending h*w of a global average pooling
    for layer in spec["layers"]:
        kind = layer[0]
        if kind == "conv":
            W = np.asarray(layer[1], dtype=np.float64)
            out["layers"].append(("conv", W * factor if factor != 1.0 else W, layer[2]))
            factor = 1.0
        elif kind == "bn_quad":
            bias, gamma, beta, mean, var, eps, act = layer[1:8]
            gamma = np.asarray(gamma, dtype=np.float64)
            bias = np.zeros_like(gamma) if bias is None else np.asarray(bias, dtype=np.float64)
            s = gamma / np.sqrt(np.asarray(var, dtype=np.float64) + eps)
            t = s * (bias - np.asarray(mean, dtype=np.float64)) + np.asarray(beta, dtype=np.float64)
            a, b, c = (float(v) for v in act)
            out["layers"].append(("quad", a * s * s, 2.0 * a * s * t + b * s, a * t * t + b * t + c))
        elif kind in ("avgpool", "pool"):
            if kind == "avgpool":
                factor *= 0.5 if dims == 1 else 0.25
            w //= 2
            if dims == 2:
                h //= 2
            out["layers"].append(("pool",))
        elif kind in ("gavgpool", "gap"):
            if kind == "gavgpool":
                divisor = float(h * w)
            out["layers"].append(("gap",))
        elif kind == "fc":
            W = np.asarray(layer[1], dtype=np.float64)
            if factor != 1.0 or divisor != 1.0:
                W = (W * factor) / divisor
            out["layers"].append(("fc", W) + tuple(layer[2:]))
            factor = divisor = 1.0
        else:
            out["layers"].append(layer)
    return out


# ------------------------------------------------------------------ layout
class Layout:
    def __init__(self, S, dist, h, w, pitch, stride, n_ct, chan, lr, offs=(0,)):
        self.S, self.dist = S, dist
        self.cbar = S // dist
        self.h, self.w, self.pitch, self.stride = h, w, pitch, stride
        self.n_ct = n_ct
        self.chan = chan            # (i, m, p) -> channel held at ct i, block m, phase p
        self.lr = lr                # block shifts l in [0, lr) that reach every channel
        self.offs = list(offs)      # phase offsets of a packed ciphertext
        self.clean = True           # non-valid slots hold zeros

    def positions(self):
        y, x = np.meshgrid(np.arange(self.h), np.arange(self.w), indexing="ij")
        y, x = y.ravel(), x.ravel()
        return y, x, self.stride * (y * self.pitch + x)

    def valid_mask(self):
        z = np.zeros(self.S)
        _, _, off = self.positions()
        for m in range(self.cbar):
            z[m * self.dist + off] = 1.0
        return z


def input_layout(spec, S):
    """dist = the smallest power of two covering the map at its puncture stride
    (stride * h * pitch slots); fewer channels than blocks are held as copies"""
    h, w, c_in = spec["h"], spec["w"], spec["c_in"]
    pitch = spec.get("pitch") or w
    stride = spec.get("stride", 1)
    dist = 1
    while dist < stride * h * pitch:
        dist *= 2
    cbar = S // dist
    if c_in < cbar:
        assert cbar % c_in == 0
        return Layout(S, dist, h, w, pitch, stride, 1, lambda i, m, p: m % c_in, c_in)
    assert c_in % cbar == 0
    return Layout(S, dist, h, w, pitch, stride, c_in // cbar, lambda i, m, p: cbar * i + m, cbar)


def pack_input(spec, x, S):
    """slot vector of the input ciphertext of a dense (stride 1) input tensor with at most
    cbar channels: block m = plane (m mod c_in), row-major"""
    lay = input_layout(spec, S)
    assert lay.stride == 1 and lay.n_ct == 1
    planes = np.asarray(x, dtype=np.float64).reshape(spec["c_in"], spec["h"], spec["w"])
    z = np.zeros(S)
    for m in range(lay.cbar):
        for y in range(spec["h"]):
            z[m * lay.dist + y * lay.pitch:m * lay.dist + y * lay.pitch + spec["w"]] = planes[m % spec["c_in"], y]
    return z


def channel_maps(lay, xs):
    """feature maps [c][h][w] read from the valid positions of slot vectors xs (one per
    ciphertext) in layout lay"""
    y, x, off = lay.positions()
    n_ch = lay.n_ct * lay.cbar
    out = np.zeros((n_ch, lay.h, lay.w))
    for i in range(lay.n_ct):
        for m in range(lay.cbar):
            out[lay.chan(i, m, 0), y, x] = np.asarray(xs[i])[m * lay.dist + off]
    return out


# ------------------------------------------------------------------ plan
def split_amount(strategy, r, l, dist):
    """(b, g) with b + g = r + dist*l for a strategy ("full" | "baby" | "giant" |
    ("hybrid", n1))"""
    if strategy == "full":
        return r + dist * l, 0
    if strategy == "baby":
        return r, dist * l
    if strategy == "giant":
        return dist * l, r
    kind, n1 = strategy
    assert kind == "hybrid" and n1 >= 1
    return r + dist * (l % n1), dist * n1 * (l // n1)


def conv_terms(lay, W, strategy, only_j=None):
    c_out, c_in, fh, fw = W.shape
    cbar, S, dist = lay.cbar, lay.S, lay.dist
    assert c_out % cbar == 0
    n_out = c_out // cbar
    js = range(n_out) if only_j is None else [only_j]
    y, x, off0 = lay.positions()
    terms = {}
    for u in range(fh):
        du = u - fh // 2
        for v in range(fw):
            dv = v - fw // 2
            ok = (y + du >= 0) & (y + du < lay.h) & (x + dv >= 0) & (x + dv < lay.w)
            pos = off0[ok]
            r = lay.stride * (du * lay.pitch + dv)
            for l in range(lay.lr):
                b, g = split_amount(strategy, r, l, dist)
                for i in range(lay.n_ct):
                    for j in js:
                        z = np.zeros(S)
                        for m in range(cbar):
                            o = cbar * j + m
                            for p, off in enumerate(lay.offs):
                                c = lay.chan(i, (m + l) % cbar, p)
                                z[m * dist + pos + off] = W[o, c, u, v]
                        key = (i, j, b % S, g % S)
                        terms[key] = terms[key] + z if key in terms else z
    return n_out, terms


def fc_terms(lay, W, strategy):
    """FC on globally pooled features: ct i block m start holds channel chan(i, m, 0);
    logit o lands at slot o*dist (Methods, "Non-convolutional layers": the weight matrix
    is cut into c_out x cbar blocks, one per input ciphertext)"""
    n_cls = W.shape[0]
    cbar, S, dist = lay.cbar, lay.S, lay.dist
    assert n_cls <= cbar
    terms = {}
    for d in range(cbar):
        b, g = split_amount(strategy, 0, d, dist)
        for i in range(lay.n_ct):
            z = np.zeros(S)
            for o in range(n_cls):
                z[o * dist] = W[o, lay.chan(i, (o + d) % cbar, 0)]
            key = (i, 0, b % S, g % S)
            terms[key] = terms[key] + z if key in terms else z
    return 1, terms


def build_plan(spec, S, strategies=None):
    """spec: collapsed network; strategies: one entry per conv / fc layer in order
    (default ("hybrid", 4) capped at the number of block shifts)"""
    lay = input_layout(spec, S)
    dims = spec["conv_dims"]
    ops = []
    si = 0

    def strat(lr):
        nonlocal si
        s = None if strategies is None else strategies[si]
        si += 1
        if s is None:
            s = ("hybrid", min(4, lr))
        return s

    for layer in spec["layers"]:
        kind = layer[0]
        if kind == "conv":
            W, fast = layer[1], layer[2]
            c_out = W.shape[0]
            if fast:
                s = lay.stride
                assert s > 1
                # load number: as many punctured ciphertexts as there are phases, at most
                # the number of input ciphertexts (phases in x first, then y)
                n_p = s if dims == 1 else s * s
                while lay.n_ct % n_p:
                    n_p //= 2
                nx = min(s, n_p)
                ny = n_p // nx
                offs = [py * lay.pitch + px for py in range(ny) for px in range(nx)]
                ops.append(("pack", lay.valid_mask(), n_p, offs))
                old = lay
                lay = Layout(S, old.dist, old.h, old.w, old.pitch, s, old.n_ct // n_p,
                             lambda t, m, p, old=old, n_p=n_p: old.chan(t * n_p + p, m, 0),
                             old.cbar, offs)
            n_out, terms = conv_terms(lay, W, strat(lay.lr))
            ops.append(("diag", n_out, terms))
            if fast:
                # step (iii): rotate-and-sum over the phases, log2(n_P) rotations
                steps = []
                t = 1
                while t < nx:
                    steps.append(t)
                    t *= 2
                t = 1
                while t < ny:
                    steps.append(t * lay.pitch)
                    t *= 2
                ops.append(("rotsum", steps))
            cbar = lay.cbar
            lay = Layout(S, lay.dist, lay.h, lay.w, lay.pitch, lay.stride, n_out,
                         lambda i, m, p, cbar=cbar: cbar * i + m, cbar)
            lay.clean = not fast
        elif kind == "quad":
            A, B, C = (np.asarray(v, dtype=np.float64) for v in layer[1:4])
            _, _, off = lay.positions()
            vecs = []
            for coef in (A, B, C):
                per_ct = []
                for i in range(lay.n_ct):
                    z = np.zeros(S)
                    for m in range(lay.cbar):
                        z[m * lay.dist + off] = coef[lay.chan(i, m, 0)]
                    per_ct.append(z)
                vecs.append(per_ct)
            ops.append(("quad",) + tuple(vecs))
            lay.clean = True
        elif kind == "pool":
            steps = [lay.stride] if dims == 1 else [lay.stride, lay.stride * lay.pitch]
            ops.append(("rotsum", steps))
            lay.stride *= 2
            if dims == 1:
                lay.w //= 2
            else:
                lay.h //= 2
                lay.w //= 2
            lay.clean = False
        elif kind == "gap":
            assert lay.clean, "global pooling needs zeros outside the map"
            steps = []
            t = lay.stride
            while t < lay.dist:
                steps.append(t)
                t *= 2
            ops.append(("rotsum", steps))
        elif kind == "fc":
            W, bias = layer[1], layer[2]
            n_out, terms = fc_terms(lay, W, strat(lay.cbar))
            ops.append(("diag", n_out, terms))
            if bias is not None:
                z = np.zeros(S)
                for o in range(W.shape[0]):
                    z[o * lay.dist] = bias[o]
                ops.append(("bias", z))
            out_slots = [o * lay.dist for o in range(W.shape[0])]
            return ops, out_slots
        else:
            raise ValueError(kind)
    return ops, None


def plan_rotations(ops, S):
    """left-rotation amounts (in [1, S)) every key switch of the plan uses"""
    steps = set()
    for op in ops:
        if op[0] == "diag":
            for (i, j, b, g) in op[2]:
                if b:
                    steps.add(b)
                if g:
                    steps.add(g)
        elif op[0] == "pack":
            for off in op[3]:
                if off:
                    steps.add((-off) % S)
        elif op[0] == "rotsum":
            steps.update(s % S for s in op[1])
    return sorted(steps)


def plan_depth(ops):
    return sum({"diag": 1, "pack": 1, "quad": 2}.get(op[0], 0) for op in ops)


# ------------------------------------------------------------------ plain simulation
def rho(v, a):
    """left rotation by a slots"""
    return np.roll(v, -a)


def simulate(ops, xs):
    """the plan on plain slot vectors (xs: list of length-S arrays)"""
    xs = [np.asarray(x, dtype=np.float64) for x in xs]
    for op in ops:
        if op[0] == "diag":
            n_out, terms = op[1], op[2]
            out = [np.zeros_like(xs[0]) for _ in range(n_out)]
            for (i, j, b, g), z in terms.items():
                out[j] += z * rho(xs[i], b + g)
            xs = out
        elif op[0] == "pack":
            mask, n_p, offs = op[1], op[2], op[3]
            xs = [sum(rho(mask * xs[t * n_p + p], -offs[p]) for p in range(n_p))
                  for t in range(len(xs) // n_p)]
        elif op[0] == "rotsum":
            for s in op[1]:
                xs = [x + rho(x, s) for x in xs]
        elif op[0] == "quad":
            A, B, C = op[1], op[2], op[3]
            xs = [A[i] * x * x + B[i] * x + C[i] for i, x in enumerate(xs)]
        elif op[0] == "bias":
            xs = [x + op[1] for x in xs]
        else:
            raise ValueError(op[0])
    return xs


# ------------------------------------------------------------------ encrypted evaluation
def _encode_many(o, items, pool):
    """items: list of (slot vector, scale, level) -> plaintexts"""
    return list(pool.map(lambda it: o.encode_pt(*it), items))


def diag_layer(o, cts, n_out, terms, keys, pool, only_j=None):
    level = cts[0].level
    ql = float(o.q[level])
    S = o.n // 2
    babies = {}
    for i in sorted({k[0] for k in terms}):
        bs = sorted({k[2] for k in terms if k[0] == i and (only_j is None or k[1] == only_j)})
        rots = [b for b in bs if b != 0]
        d = dict(zip(rots, o.rotate_hoisted(cts[i], rots, keys))) if rots else {}
        if 0 in bs:
            d[0] = cts[i]
        babies[i] = d
    outs = []
    for j in range(n_out):
        if only_j is not None and j != only_j:
            outs.append(None)
            continue
        keys_j = sorted(k for k in terms if k[1] == j)
        pts = dict(zip(keys_j, _encode_many(
            o, [(np.roll(terms[k], k[3]), ql, level) for k in keys_j], pool)))
        acc = None
        for g in sorted({k[3] for k in keys_j}):
            inner = None
            for k in keys_j:
                if k[3] != g:
                    continue
                prod = o.mulplain(babies[k[0]][k[2]], pts[k], ql)
                inner = prod if inner is None else o.add(inner, prod)
            if g != 0:
                inner = o.rotate(inner, g, keys)
            acc = inner if acc is None else o.add(acc, inner)
        outs.append(o.rescale(acc))
    return outs


def pack(o, cts, mask, n_p, offs, keys):
    level = cts[0].level
    ql = float(o.q[level])
    S = o.n // 2
    ptm = o.encode_pt(mask, ql, level)
    out = []
    for t in range(len(cts) // n_p):
        acc = None
        for p in range(n_p):
            y = o.rescale(o.mulplain(cts[t * n_p + p], ptm, ql))
            if offs[p]:
                y = o.rotate(y, (-offs[p]) % S, keys)
            acc = y if acc is None else o.add(acc, y)
        out.append(acc)
    return out


def rotsum(o, ct, steps, keys):
    S = o.n // 2
    for s in steps:
        ct = o.add(ct, o.rotate(ct, s % S, keys))
    return ct


def quad(o, ct, A, B, C, keys):
    """A x^2 + B x + C in Horner form x*(A x + B) + C: u = rescale(x (.) Enc_(q_l)(A)) + B,
    then rescale(relin(drop(x) * u)) + C -- two levels; every plaintext is encoded at the
    scale of the ciphertext it meets, so the slot values carry no scale error"""
    level = ct.level
    ql = float(o.q[level])
    u = o.rescale(o.mulplain(ct, o.encode_pt(A, ql, level), ql))
    u = o.add_plain(u, o.encode_pt(B, u.scale, u.level))
    v = o.mul_relin_rescale(o.drop_level(ct), u, keys)
    return o.add_plain(v, o.encode_pt(C, v.scale, v.level))


def evaluate(o, ops, cts, keys, pool=None):
    if pool is None:
        pool = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)
    for op in ops:
        if op[0] == "diag":
            cts = diag_layer(o, cts, op[1], op[2], keys, pool)
        elif op[0] == "pack":
            cts = pack(o, cts, op[1], op[2], op[3], keys)
        elif op[0] == "rotsum":
            cts = [rotsum(o, c, op[1], keys) for c in cts]
        elif op[0] == "quad":
            cts = [quad(o, c, op[1][i], op[2][i], op[3][i], keys) for i, c in enumerate(cts)]
        elif op[0] == "bias":
            cts = [o.add_plain(c, o.encode_pt(op[1], c.scale, c.level)) for c in cts]
        else:
            raise ValueError(op[0])
    return cts
