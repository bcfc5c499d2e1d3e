"""Seeded synthetic workloads: CKKS parameter sets, clip features and network weights.

This module holds no homomorphic arithmetic.  It only draws the FP64 inputs that both
the CUDA library and the CPU oracle consume, so both sides see identical data.

The paper evaluates skeleton CNNs on a private test set (608 clips of 2x32x15
min-max-normalised joint coordinates, Methods "Data preprocessing"); that data and the
trained weights are not available, so these synthetic inputs stand in for them:

* ``toy``   -- N = 2^12, q = 50 + 40 + 40 bits, one 50-bit special prime; 64-dim (one by default)
  input uniform in [-1, 1]; FC 64->16 -> x^2 -> FC 16->2 with N(0, 0.1^2) weights.
* ``small`` -- N = 2^14, q = 60 + 7x40 bits, one 60-bit special prime; one clip of
  16 frames x 128 features ~ N(0,1) clipped to [-1, 1]; FC 2048->128 -> x^2 -> FC 128->2.
* ``large`` -- N = 2^15, q = 60 + 14x40 bits, two 60-bit special primes; 256 clips packed
  8 per ciphertext; FC 2048->512 -> x^2 -> FC 512->128 -> x^2 -> FC 128->2.

Weights of ``small`` / ``large``: Xavier-normal (std sqrt(2/(fan_in+fan_out))) times
c_l = 1/max(1, max|pre-activation of layer l|) over the generated clips, layer by layer,
so that every activation stays inside [-1, 1].
"""
from dataclasses import dataclass, field
from typing import List, Tuple
import numpy as np

SEED_WEIGHTS = 101
SEED_INPUTS = 201
SEED_KEYS = 301
SEED_ENC = 401


@dataclass
class Workload:
    name: str
    log_n: int
    q_bits: List[int]
    p_bits: List[int]
    log2_scale: float
    sigma: float
    clip_dim: int            # features per clip (one input vector)
    n_clips: int             # clips in the whole workload
    clips_per_ct: int        # clips packed (interleaved) into one ciphertext
    layers: list = field(default_factory=list)   # ("fc", W) | ("square",) | ("fc_sq_fc", W1, W2)
    clips: np.ndarray = None  # [n_clips, clip_dim] float64

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2

    @property
    def n_ct(self):
        return (self.n_clips + self.clips_per_ct - 1) // self.clips_per_ct

    def ct_clips(self, i: int) -> np.ndarray:
        """clips carried by ciphertext i"""
        return self.clips[i * self.clips_per_ct:(i + 1) * self.clips_per_ct]

    def fp64_forward(self, x: np.ndarray) -> np.ndarray:
        """Plain FP64 evaluation of the network on rows of x (reference for decrypted logits)."""
        h = np.asarray(x, dtype=np.float64)
        for layer in self.layers:
            if layer[0] == "fc":
                h = h @ layer[1].T
                if len(layer) > 2 and layer[2] is not None:
                    h = h + layer[2]
            elif layer[0] == "square":
                h = h * h
            elif layer[0] == "fc_sq_fc":
                y = h @ layer[1].T
                h = (y * y) @ layer[2].T
            else:
                raise ValueError(layer[0])
        return h


def _xavier_scaled(rng, dims, x):
    """Xavier-normal weights scaled layer by layer to keep activations in [-1, 1]."""
    layers = []
    h = x
    for li, (d_out, d_in) in enumerate(dims):
        std = np.sqrt(2.0 / (d_in + d_out))
        W = rng.normal(0.0, std, size=(d_out, d_in))
        pre = h @ W.T
        c = 1.0 / max(1.0, float(np.max(np.abs(pre))))
        W = W * c
        layers.append(("fc", W))
        h = pre * c
        if li < len(dims) - 1:
            layers.append(("square",))
            h = h * h
    return layers


def make_workload(name: str, n_clips: int = None) -> Workload:
    if name == "toy":
        w = Workload("toy", 12, [50, 40, 40], [50], 40.0, 3.2, clip_dim=64,
                     n_clips=1, clips_per_ct=1)
        rw = np.random.default_rng(SEED_WEIGHTS)
        W1 = rw.normal(0.0, 0.1, size=(16, 64))
        W2 = rw.normal(0.0, 0.1, size=(2, 16))
        # FC -> x^2 -> FC needs three rescales but the chain holds two scaling primes:
        # the activation and the second FC are collapsed into one quadratic form.
        w.layers = [("fc_sq_fc", W1, W2)]
        ri = np.random.default_rng(SEED_INPUTS)
        w.n_clips = 1 if n_clips is None else n_clips
        w.clips = ri.uniform(-1.0, 1.0, size=(w.n_clips, 64))
        return w
    if name == "small":
        w = Workload("small", 14, [60] + [40] * 7, [60], 40.0, 3.2, clip_dim=2048,
                     n_clips=1 if n_clips is None else n_clips, clips_per_ct=4)
        dims = [(128, 2048), (2, 128)]
    elif name == "large":
        w = Workload("large", 15, [60] + [40] * 14, [60, 60], 40.0, 3.2, clip_dim=2048,
                     n_clips=256 if n_clips is None else n_clips, clips_per_ct=8)
        dims = [(512, 2048), (128, 512), (2, 128)]
    else:
        raise ValueError(name)
    ri = np.random.default_rng(SEED_INPUTS)
    w.clips = np.clip(ri.normal(0.0, 1.0, size=(w.n_clips, w.clip_dim)), -1.0, 1.0)
    rw = np.random.default_rng(SEED_WEIGHTS)
    w.layers = _xavier_scaled(rw, dims, w.clips)
    return w


def layer_descs(w: Workload) -> List[Tuple]:
    return list(w.layers)


# ---------------------------------------------------------------------------------------
# Skeleton CNNs (Methods, "Network architecture for action recognition"; Fig. 3)
#
# Three convolutional layers (3 filter taps in 1D, 3x3 in 2D, stride 1, same padding),
# each followed by a bias, batch normalisation, a trained quadratic activation
# a*y^2 + b*y + c and average pooling (window 2 / 2x2, stride 2; global average pooling
# after the third), then an FC layer to the classes.  f filters in the first layer,
# doubled at every halving of the map.  Inputs are 2 x 32 x 15 tensors (x / y coordinate
# planes, 32 frames x 15 joints, min-max normalised per coordinate, Methods "Data
# preprocessing"); the 1D networks slide their kernels along the row-major flattening
# (length 480) of each plane.
#
# Synthetic stand-ins (the trained weights and the clips are not available):
# * clips: a 15-joint standing skeleton (fixed template), random body scale / position,
#   per-joint sinusoidal motion of random amplitude, frequency and phase over 32 frames,
#   half of the clips with a fall (the body centre drops and rotates over the last
#   frames), Gaussian jitter; then min-max normalisation per coordinate plane;
# * conv / FC weights Xavier-normal, biases N(0, 0.05^2), BN gamma U(0.8, 1.2), beta
#   N(0, 0.05^2), running mean N(0, 0.05^2), running variance U(0.5, 1.5), eps 1e-5;
#   quadratic coefficients per layer (a, b, c) = (0.25, 0.5, 0.125) + N(0, 0.02^2) each
#   (a ReLU-like quadratic); each conv layer's weights are rescaled so that its BN output
#   stays inside [-1, 1] over the generated clips.
# ---------------------------------------------------------------------------------------

SEED_CNN_WEIGHTS = 111
SEED_CNN_INPUTS = 211
BN_EPS = 1e-5


@dataclass
class CnnNet:
    name: str
    log_n: int
    q_bits: List[int]
    p_bits: List[int]
    log2_scale: float
    sigma: float
    conv_dims: int                 # 1 or 2
    filters: List[int]             # output channels of conv1..conv3
    n_classes: int
    fast: List[bool]               # fast (merge-and-conquer) convolution per conv layer
    convs: list = field(default_factory=list)   # dicts: W, bias, gamma, beta, mean, var, act
    fc_w: np.ndarray = None        # [n_classes][filters[-1]]
    fc_b: np.ndarray = None
    clips: np.ndarray = None       # [n_samples][2][32][15]

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2


def skeleton_clips(rng, n: int) -> np.ndarray:
    """n synthetic 2 x 32 x 15 skeleton clips (see the module comment)."""
    template = np.array([  # (x, y) of 15 joints of a standing body, head up
        [0.0, 1.70], [0.0, 1.55], [-0.20, 1.45], [0.20, 1.45], [-0.25, 1.15], [0.25, 1.15],
        [-0.28, 0.90], [0.28, 0.90], [-0.12, 0.95], [0.12, 0.95], [-0.13, 0.50],
        [0.13, 0.50], [-0.14, 0.05], [0.14, 0.05], [0.0, 1.25]])
    t = np.arange(32)[:, None]
    out = np.empty((n, 2, 32, 15))
    for s in range(n):
        scale = rng.uniform(0.7, 1.3)
        pos = rng.uniform(-1.0, 1.0, size=2)
        amp = rng.uniform(0.0, 0.12, size=(2, 15))
        freq = rng.uniform(0.05, 0.4, size=(2, 15))
        ph = rng.uniform(0.0, 2 * np.pi, size=(2, 15))
        xy = np.empty((2, 32, 15))
        for d in range(2):
            xy[d] = scale * template[:, d][None, :] + pos[d] + amp[d] * np.sin(2 * np.pi * freq[d] * t + ph[d])
        if s % 2 == 1:   # fall: from frame f0 the body rotates towards the floor
            f0 = rng.integers(8, 24)
            k = np.clip((t - f0) / 8.0, 0.0, 1.0)           # [32, 1] progress
            ang = k * (np.pi / 2) * rng.choice([-1.0, 1.0])
            base = scale * template[:, 1][None, :] * np.ones((32, 1))
            xy[0] = xy[0] + base * np.sin(ang)
            xy[1] = xy[1] - base * (1.0 - np.cos(ang))
        xy = xy + rng.normal(0.0, 0.01, size=xy.shape)
        for d in range(2):
            lo, hi = xy[d].min(), xy[d].max()
            xy[d] = (xy[d] - lo) / (hi - lo)
        out[s] = xy
    return out


def _conv_same(x, W, dims):
    """plain same-padded, stride-1 cross-correlation: x [c_in][H][W] (1D: [c_in][L])"""
    if dims == 1:
        c_in, L = x.shape
        f = W.shape[-1]
        xp = np.pad(x, ((0, 0), (f // 2, f // 2)))
        y = np.zeros((W.shape[0], L))
        for k in range(f):
            y += W[:, :, 0, k] @ xp[:, k:k + L]
        return y
    c_in, H, Wd = x.shape
    fh, fw = W.shape[2], W.shape[3]
    xp = np.pad(x, ((0, 0), (fh // 2, fh // 2), (fw // 2, fw // 2)))
    y = np.zeros((W.shape[0], H, Wd))
    for u in range(fh):
        for v in range(fw):
            y += np.einsum("oc,chw->ohw", W[:, :, u, v], xp[:, u:u + H, v:v + Wd])
    return y


def _pool_avg(x, dims):
    if dims == 1:
        L = x.shape[1] // 2
        return 0.5 * (x[:, 0:2 * L:2] + x[:, 1:2 * L:2])
    H, Wd = x.shape[1] // 2, x.shape[2] // 2
    return 0.25 * (x[:, 0:2 * H:2, 0:2 * Wd:2] + x[:, 1:2 * H:2, 0:2 * Wd:2] +
                   x[:, 0:2 * H:2, 1:2 * Wd:2] + x[:, 1:2 * H:2, 1:2 * Wd:2])


def cnn_input_map(clip, dims):
    """network input: [2][480] (1D) or [2][32][15] (2D)"""
    return clip.reshape(2, -1) if dims == 1 else clip


def cnn_forward(net: CnnNet, clip, upto=None):
    """Plain FP64 forward of the uncollapsed network (conv + bias -> BN -> a y^2 + b y + c
    -> average pooling; global average pooling; FC + bias).  ``upto`` = number of conv
    blocks to run (returns the feature map after that block's pooling)."""
    h = cnn_input_map(np.asarray(clip, dtype=np.float64), net.conv_dims)
    n_blocks = len(net.convs) if upto is None else upto
    for li in range(n_blocks):
        cv = net.convs[li]
        y = _conv_same(h, cv["W"], net.conv_dims)
        y = y + cv["bias"].reshape((-1,) + (1,) * (y.ndim - 1))
        sh = (-1,) + (1,) * (y.ndim - 1)
        y = cv["gamma"].reshape(sh) * (y - cv["mean"].reshape(sh)) / np.sqrt(cv["var"].reshape(sh) + BN_EPS) \
            + cv["beta"].reshape(sh)
        a, b, c = cv["act"]
        y = a * y * y + b * y + c
        if li < len(net.convs) - 1:
            h = _pool_avg(y, net.conv_dims)
        else:
            h = y
    if upto is not None:
        return h
    g = h.reshape(h.shape[0], -1).mean(axis=1)
    return net.fc_w @ g + net.fc_b


def cnn_spec(net: CnnNet) -> dict:
    """The network as trained, in the layer vocabulary of hear_cnn_create: per block the
    convolution, its bias with batch normalisation and the quadratic activation
    ("bn_quad"), then average pooling (global after the last block), and the FC.  No
    arithmetic: the collapse is done by the library (and, separately, by the oracle)."""
    dims = net.conv_dims
    h, w = (1, 480) if dims == 1 else (32, 15)
    spec = {"conv_dims": dims, "c_in": 2, "h": h, "w": w, "layers": []}
    for li, cv in enumerate(net.convs):
        spec["layers"].append(("conv", cv["W"], bool(net.fast[li])))
        spec["layers"].append(("bn_quad", cv["bias"], cv["gamma"], cv["beta"], cv["mean"], cv["var"], BN_EPS,
                               tuple(cv["act"])))
        spec["layers"].append(("avgpool",) if li < len(net.convs) - 1 else ("gavgpool",))
    spec["layers"].append(("fc", net.fc_w, np.asarray(net.fc_b, dtype=np.float64)))
    return spec


_CNN_SETS = {
    # name: (log_n, q_bits, p_bits, conv dims, filters, fast per conv)
    # 12 levels: conv 1 + quad 2 per block, one mask level per fast conv, FC 1
    "cnn_toy": (12, [60] + [40] * 12, [60, 60], 1, [8, 16, 32], [False, True, True]),
    "cnn2d_toy": (12, [60] + [40] * 12, [60, 60], 2, [8, 16, 32], [False, True, True]),
    "cnn1d64": (15, [60] + [40] * 14, [60, 60], 1, [64, 128, 256], [False, True, True]),
    "cnn2d64": (15, [60] + [40] * 14, [60, 60], 2, [64, 128, 256], [False, True, True]),
}


def make_cnn(name: str, n_samples: int = 2) -> CnnNet:
    log_n, qb, pb, dims, filters, fast = _CNN_SETS[name]
    net = CnnNet(name, log_n, qb, pb, 40.0, 3.2, dims, list(filters), 2, list(fast))
    ri = np.random.default_rng(SEED_CNN_INPUTS)
    net.clips = skeleton_clips(ri, max(n_samples, 8))
    rw = np.random.default_rng(SEED_CNN_WEIGHTS)
    f = 3
    c_prev = 2
    h_all = [cnn_input_map(cl, dims) for cl in net.clips]
    for li, c_out in enumerate(filters):
        fh, fw = (1, f) if dims == 1 else (f, f)
        std = np.sqrt(2.0 / (c_prev * fh * fw + c_out))
        W = rw.normal(0.0, std, size=(c_out, c_prev, fh, fw))
        cv = dict(bias=rw.normal(0.0, 0.05, c_out), gamma=rw.uniform(0.8, 1.2, c_out),
                  beta=rw.normal(0.0, 0.05, c_out), mean=rw.normal(0.0, 0.05, c_out),
                  var=rw.uniform(0.5, 1.5, c_out),
                  act=tuple(np.array([0.25, 0.5, 0.125]) + rw.normal(0.0, 0.02, 3)))
        # rescale W so that the BN outputs over the generated clips stay inside [-1, 1]
        s = cv["gamma"] / np.sqrt(cv["var"] + BN_EPS)
        peak = 0.0
        for h in h_all:
            y = _conv_same(h, W, dims)
            sh = (-1,) + (1,) * (y.ndim - 1)
            z = s.reshape(sh) * (y + (cv["bias"] - cv["mean"]).reshape(sh)) + cv["beta"].reshape(sh)
            peak = max(peak, float(np.max(np.abs(z))))
        W = W / max(1.0, peak)
        cv["W"] = W
        net.convs.append(cv)
        nxt = []
        for h in h_all:
            y = _conv_same(h, W, dims)
            sh = (-1,) + (1,) * (y.ndim - 1)
            y = s.reshape(sh) * (y + (cv["bias"] - cv["mean"]).reshape(sh)) + cv["beta"].reshape(sh)
            a, b, c = cv["act"]
            y = a * y * y + b * y + c
            nxt.append(_pool_avg(y, dims) if li < len(filters) - 1 else y)
        h_all = nxt
        c_prev = c_out
    std = np.sqrt(2.0 / (c_prev + 2))
    net.fc_w = rw.normal(0.0, std, size=(2, c_prev))
    net.fc_b = rw.normal(0.0, 0.05, 2)
    net.clips = net.clips[:n_samples]
    return net


# Convolutional layers of the paper's homomorphic convolution microbenchmark (Table 1):
# (network, layer, conv dims, map (h, w) at the layer input, row pitch, puncture stride,
#  input channels, output channels).  The maps are those after one / two poolings of the
# 32 x 15 (2D) or 480-long (1D) input; the parameter set is N = 2^14 (16 channels of 512
# slots per ciphertext), q = 60 + 7x40 bits, p = 60 bits.
TABLE1_LAYERS = [
    ("1D-CNN-64", "conv2", 1, (1, 240), 240, 2, 64, 128),
    ("1D-CNN-64", "conv3", 1, (1, 120), 120, 4, 128, 256),
    ("1D-CNN-128", "conv2", 1, (1, 240), 240, 2, 128, 256),
    ("1D-CNN-128", "conv3", 1, (1, 120), 120, 4, 256, 512),
    ("2D-CNN-64", "conv2", 2, (16, 7), 15, 2, 64, 128),
    ("2D-CNN-64", "conv3", 2, (8, 3), 15, 4, 128, 256),
    ("2D-CNN-128", "conv2", 2, (16, 7), 15, 2, 128, 256),
    ("2D-CNN-128", "conv3", 2, (8, 3), 15, 4, 256, 512),
]
CONV_BENCH_PARAMS = (14, [60] + [40] * 7, [60])


def conv_bench_layer(index: int, fast: bool, n_samples: int = 1):
    """(spec of the single punctured conv layer, input slot vectors [n_samples][n_ct][N/2]).
    Weights Xavier-normal; every input slot (valid map positions and the junk between them
    alike) U(-1, 1)."""
    net, layer, dims, (h, w), pitch, stride, c_in, c_out = TABLE1_LAYERS[index]
    f = 3
    fh, fw = (1, f) if dims == 1 else (f, f)
    rw = np.random.default_rng(SEED_CNN_WEIGHTS + 7 * index)
    std = np.sqrt(2.0 / (c_in * fh * fw + c_out))
    W = rw.normal(0.0, std, size=(c_out, c_in, fh, fw))
    spec = {"conv_dims": dims, "c_in": c_in, "h": h, "w": w, "pitch": pitch, "stride": stride,
            "layers": [("conv", W, bool(fast))]}
    log_n = CONV_BENCH_PARAMS[0]
    slots = 1 << (log_n - 1)
    dist = 1
    while dist < stride * h * pitch:
        dist *= 2
    n_ct = c_in // (slots // dist)
    ri = np.random.default_rng(SEED_CNN_INPUTS + 7 * index)
    xs = ri.uniform(-1.0, 1.0, size=(n_samples, n_ct, slots))
    return spec, xs
