"""Plain FP64 numpy reference of the warm-start network (test infrastructure only).

The paper has no counterpart: this checks the library's own forward/backward
kernels and its tensor-core inference.  Layout of the flat parameter vector:
W1 [64][32], b1 [64], W2 [64][64], b2, W3 [64][64], b3, W4 [16][64], b4 [16],
input mean [32], input std [32], target scale [16].  Network: standardise the
32 features, three GELU hidden layers of 64, a linear layer of 16;
loss = mean squared error over the first 9 outputs against targets divided by
the target scale.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT, N_USED = 32, 64, 16, 9
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,)),
          ("in_mean", (N_IN,)), ("in_std", (N_IN,)), ("out_scale", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
N_TRAINABLE = N_PARAMS - 2 * N_IN - N_OUT


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715


def gelu(z):
    """GELU in its tanh form (Hendrycks and Gimpel, arXiv 1606.08415):
    x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    z = np.asarray(z, np.float64)
    u = GELU_C * (z + GELU_A * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def forward(p, feats):
    q = unpack(p)
    x = (np.asarray(feats, np.float64) - q["in_mean"]) / q["in_std"]
    z1 = x @ q["W1"].T + q["b1"]
    h1 = gelu(z1)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = gelu(z2)
    z3 = h2 @ q["W3"].T + q["b3"]
    h3 = gelu(z3)
    y = h3 @ q["W4"].T + q["b4"]
    return y, (x, z1, h1, z2, h2, z3, h3)


def loss_and_grad(p, feats, targets):
    q = unpack(p)
    y, (x, z1, h1, z2, h2, z3, h3) = forward(p, feats)
    n = y.shape[0]
    t = np.asarray(targets, np.float64) / q["out_scale"]
    diff = np.zeros_like(y)
    diff[:, :N_USED] = y[:, :N_USED] - t[:, :N_USED]
    loss = float((diff ** 2).sum() / (n * N_USED))
    dy = 2.0 * diff / (n * N_USED)
    g = {}
    g["W4"] = dy.T @ h3
    g["b4"] = dy.sum(0)
    dz3 = (dy @ q["W4"]) * gelu_grad(z3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ q["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ q["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    flat = np.concatenate([g[name].ravel() if name in g else np.zeros(int(np.prod(s)))
                           for name, s in SHAPES])
    return loss, flat
