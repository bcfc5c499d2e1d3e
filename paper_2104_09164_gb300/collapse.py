"""Collapse of a skeleton CNN's non-convolutional layers into the form the encrypted
network evaluates (Methods, "Non-convolutional layers"): the convolution bias, batch
normalisation and the quadratic activation of each block become one quadratic
A*y^2 + B*y + C per feature map (y = the bias-free convolution output), and the 1/2
(1D) or 1/4 (2D) scale of each average pooling and the 1/(h*w) of the global average
pooling move into the weights of the next linear layer, so that pooling is a plain sum.

With BN(y + bias) = s*y + t, s = gamma / sqrt(var + eps), t = s*(bias - mean) + beta and
the activation a*z^2 + b*z + c:  A = a*s^2, B = 2*a*s*t + b*s, C = a*t^2 + b*t + c.

The result is a plain dict (host data only):
  {"conv_dims": 1|2, "c_in": 2, "h": H, "w": W,
   "layers": [("conv", W[c_out][c_in][fh][fw], fast), ("quad", A, B, C), ("pool",),
              ("gap",), ("fc", W[n_cls][c], bias[n_cls])]}
"""
import numpy as np

from .workloads import BN_EPS, CnnNet


def collapse_cnn(net: CnnNet) -> dict:
    dims = net.conv_dims
    h, w = (1, 480) if dims == 1 else (32, 15)
    spec = {"conv_dims": dims, "c_in": 2, "h": h, "w": w, "layers": []}
    pool_scale = 1.0
    n = len(net.convs)
    for li, cv in enumerate(net.convs):
        spec["layers"].append(("conv", cv["W"] * pool_scale, bool(net.fast[li])))
        s = cv["gamma"] / np.sqrt(cv["var"] + BN_EPS)
        t = s * (cv["bias"] - cv["mean"]) + cv["beta"]
        a, b, c = cv["act"]
        spec["layers"].append(("quad", a * s * s, 2 * a * s * t + b * s, a * t * t + b * t + c))
        if li < n - 1:
            spec["layers"].append(("pool",))
            pool_scale = 0.5 if dims == 1 else 0.25
            if dims == 1:
                w //= 2
            else:
                h, w = h // 2, w // 2
        else:
            spec["layers"].append(("gap",))
    spec["layers"].append(("fc", net.fc_w / float(h * w), np.asarray(net.fc_b, dtype=np.float64)))
    return spec
