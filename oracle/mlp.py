"""Oracle for the candidate scorer of the learned proposal (numpy, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The scorer is a perceptron with two hidden ReLU layers and one logit,
    H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  s = H2 w3 + b3,
trained by minimising the weighted binary cross-entropy of the logits,
    L = sum_i w_i (softplus(s_i) - y_i s_i),
with Adam (Kingma & Ba 2015: first and second moment estimates, both
bias-corrected).  In the BF16 network X, W1, W2, H1, H2 and the back-propagated
pre-activation gradients dZ2, dZ1 are stored as bfloat16 (8 significant bits,
round to nearest, ties to even, applied to the FP32 value); every product is
accumulated in FP32 or wider.  `quant=False` gives the plain FP64 network.

Parameters are one flat FP32 vector: W1 [in_pad][H] (in_pad = in_dim rounded
up to a multiple of 16, padded rows zero), b1 [H], W2 [H][H], b2 [H], w3 [H],
b3 [1].
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to bfloat16 (returned as float64): fl32 first, then keep the top
    16 bits of the binary32 pattern, rounding to nearest with ties to even."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def in_pad(in_dim: int) -> int:
    return (in_dim + 15) // 16 * 16


def split(flat, in_dim: int, hidden: int) -> dict:
    P, H = in_pad(in_dim), hidden
    out, o = {}, 0
    for name, shp in (("W1", (P, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def param_count(in_dim: int, hidden: int) -> int:
    P, H = in_pad(in_dim), hidden
    return P * H + H + H * H + H + H + 1


def forward(flat, x, in_dim: int, hidden: int, quant: bool = True):
    """Logits and the cached activations."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    p = split(flat, in_dim, hidden)
    x = np.asarray(x, np.float64)
    X = np.zeros((x.shape[0], in_pad(in_dim)))
    X[:, :in_dim] = x
    X = q(X)
    W1, W2 = q(p["W1"]), q(p["W2"])
    H1 = q(np.maximum(X @ W1 + p["b1"], 0.0))
    H2 = q(np.maximum(H1 @ W2 + p["b2"], 0.0))
    s = H2 @ p["w3"] + p["b3"][0]
    return s, {"X": X, "W2": W2, "H1": H1, "H2": H2, "p": p}


def softplus(s):
    """log(1 + e^s), written to avoid overflow."""
    s = np.asarray(s, np.float64)
    return np.maximum(s, 0.0) + np.log1p(np.exp(-np.abs(s)))


def loss(flat, x, y, w, in_dim, hidden, quant=True):
    s, _ = forward(flat, x, in_dim, hidden, quant)
    return float(np.sum(np.asarray(w, np.float64) * (softplus(s) - np.asarray(y, np.float64) * s)))


def gradients(flat, x, y, w, in_dim: int, hidden: int, quant: bool = True):
    """(loss, flat gradient) of the weighted cross-entropy, by back-propagation
    through the network above (ReLU derivative 1 where the output is > 0)."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    s, c = forward(flat, x, in_dim, hidden, quant)
    y, w = np.asarray(y, np.float64), np.asarray(w, np.float64)
    p = c["p"]
    sig = 1.0 / (1.0 + np.exp(-s))
    dS = w * (sig - y)
    L = float(np.sum(w * (softplus(s) - y * s)))
    g = {}
    g["w3"] = c["H2"].T @ dS
    g["b3"] = np.array([dS.sum()])
    dZ2 = q(dS[:, None] * p["w3"][None, :] * (c["H2"] > 0))
    g["W2"] = c["H1"].T @ dZ2
    g["b2"] = dZ2.sum(0)
    dH1 = dZ2 @ c["W2"].T
    dZ1 = q(dH1 * (c["H1"] > 0))
    g["W1"] = c["X"].T @ dZ1
    g["b1"] = dZ1.sum(0)
    flat_g = np.concatenate([g[k].ravel() for k in ("W1", "b1", "W2", "b2", "w3", "b3")])
    return L, flat_g


def adam(param, grad, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (param, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v
