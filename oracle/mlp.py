"""FP64 CPU reference of the surrogate inverse-CDF network (test
infrastructure only, like the rest of ``oracle``).

The network maps x = (x0, x1) to a scalar z with three SiLU hidden layers of
width 64:
    a1 = x W1 + b1,  h1 = silu(a1)
    a2 = h1 W2 + b2, h2 = silu(a2)
    a3 = h2 W3 + b3, h3 = silu(a3)
    z  = h3 W4 + b4
silu(a) = a / (1 + exp(-a)).  The loss of a batch is the mean of (z - t)^2.

Parameters travel as one flat float array in the order W1[2][64], b1[64],
W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4[1] (8577 values), the
format the C ABI uses.  The backward pass is written out by hand (chain rule)
and pinned by central finite differences in the CPU tests.
"""
from __future__ import annotations

import numpy as np

H = 64
SHAPES = [("W1", (2, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
          ("b3", (H,)), ("W4", (H,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def forward(flat, x):
    p = unpack(flat)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 2)
    a1 = x @ p["W1"] + p["b1"]
    h1 = silu(a1)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = silu(a2)
    a3 = h2 @ p["W3"] + p["b3"]
    h3 = silu(a3)
    z = h3 @ p["W4"] + p["b4"][0]
    return z, (x, a1, h1, a2, h2, a3, h3)


def loss_and_grad(flat, x, t):
    """Mean squared error and its gradient with respect to the flat parameters."""
    p = unpack(flat)
    z, (x, a1, h1, a2, h2, a3, h3) = forward(flat, x)
    t = np.asarray(t, dtype=np.float64).ravel()
    n = z.size
    r = z - t
    loss = np.mean(r * r)
    dz = 2.0 * r / n                      # dL/dz
    g = {"W4": h3.T @ dz, "b4": np.array([dz.sum()])}
    dh3 = np.outer(dz, p["W4"])
    da3 = dh3 * dsilu(a3)
    g["W3"] = h2.T @ da3
    g["b3"] = da3.sum(0)
    dh2 = da3 @ p["W3"].T
    da2 = dh2 * dsilu(a2)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * dsilu(a1)
    g["W1"] = x.T @ da1
    g["b1"] = da1.sum(0)
    return loss, pack(g)


def adam_step(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), bias-corrected; step counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed=0):
    """Uniform(+-sqrt(6/(fan_in+fan_out))) weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shp)
        else:
            fan_in = shp[0]
            fan_out = shp[1] if len(shp) > 1 else 1
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            p[name] = rng.uniform(-lim, lim, shp)
    return pack(p)
