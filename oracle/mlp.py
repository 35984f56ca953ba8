"""FP64 reference of the surrogate network (test infrastructure only).

The 4-64-64-2 perceptron of the split selector: z1 = x W1 + b1, h1 = tanh z1,
z2 = h1 W2 + b2, h2 = tanh z2, y = h2 W3 + b3, with inputs and targets
standardised by given means and standard deviations, and the loss
L = mean over samples and outputs of (y - t)^2 in standardised units.  The
backward pass is the chain rule written out layer by layer (plain numpy,
FP64); parameters use the library's flat layout
W1[4][64] b1[64] W2[64][64] b2[64] W3[64][2] b3[2].  Pinned against central
finite differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 4, 64, 2
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p, x, norm):
    """Predictions in target units and the cached activations."""
    w = unpack(p)
    xm, xs, ym, ys = (np.asarray(a, np.float64) for a in norm)
    xn = (np.asarray(x, np.float64) - xm) / xs
    h1 = np.tanh(xn @ w["W1"] + w["b1"])
    h2 = np.tanh(h1 @ w["W2"] + w["b2"])
    yn = h2 @ w["W3"] + w["b3"]
    return yn * ys + ym, (xn, h1, h2, yn)


def loss_and_grad(p, x, t, norm):
    """Loss (standardised mean squared error) and its gradient, flat layout."""
    w = unpack(p)
    _, (xn, h1, h2, yn) = forward(p, x, norm)
    ym, ys = np.asarray(norm[2], np.float64), np.asarray(norm[3], np.float64)
    tn = (np.asarray(t, np.float64) - ym) / ys
    n = xn.shape[0]
    e = yn - tn
    loss = float(np.mean(e ** 2))
    dy = 2.0 * e / (n * N_OUT)
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dz2 = (dy @ w["W3"].T) * (1.0 - h2 ** 2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"].T) * (1.0 - h1 ** 2)
    g["W1"] = xn.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(p, g, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at 1-based step t."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** t)
    vh = m2 / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
