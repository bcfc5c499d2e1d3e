"""Seeded synthetic workloads: CKKS parameter sets, clip features and network weights.

This module holds no homomorphic arithmetic.  It only draws the FP64 inputs that both
the CUDA library and the CPU oracle consume, so both sides see identical data.

The paper evaluates skeleton CNNs on a private test set (608 clips of 2x32x15
min-max-normalised joint coordinates, Methods "Data preprocessing"); that data and the
trained weights are not available, so these synthetic inputs stand in for them:

* ``toy``   -- N = 2^12, q = 50 + 40 + 40 bits, one 50-bit special prime; one 64-dim
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
        w.clips = ri.uniform(-1.0, 1.0, size=(1, 64))
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
