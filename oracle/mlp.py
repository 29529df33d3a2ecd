"""FP64 oracle of the warm-start network (numpy).

TEST INFRASTRUCTURE ONLY: the CUDA kernels of the network are checked against this
file; the solver never imports it.

The network maps the 6 parameters of a Couette problem to its steady profiles:
x -> z1 = W1 x + b1 -> h1 = gelu(z1) -> z2 = W2 h1 + b2 -> h2 = gelu(z2) -> y = W3 h2 + b3,
with gelu(z) = z (1 + erf(z / sqrt 2)) / 2 and the loss L = mean over the batch and the
outputs of (y - t)^2.  The CUDA path multiplies in BF16 with FP32 accumulation: every
operand of a matrix product (weights, inputs, activations and, in the backward pass,
the incoming gradients) is rounded to BF16 (round to nearest even) before the product.
This oracle applies the same roundings and otherwise computes in FP64, so the two agree
up to accumulation order.  Adam follows Kingma & Ba (2015) with bias correction.
"""
import math

import numpy as np
from scipy.special import erf


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _identity(a):
    return np.asarray(a, dtype=np.float64)


def forward(params, x, rounding=True):
    """params: dict W1 (256x6), b1, W2, b2, W3, b3 (FP64 masters); x: (B, 6).
    rounding=False drops the BF16 roundings (used to check the derivatives)."""
    r = bf16 if rounding else _identity
    W1, W2, W3 = (r(params[k]) for k in ("W1", "W2", "W3"))
    z1 = r(x) @ W1.T + params["b1"]
    h1 = gelu(z1)
    z2 = r(h1) @ W2.T + params["b2"]
    h2 = gelu(z2)
    y = r(h2) @ W3.T + params["b3"]
    return y, (x, z1, h1, z2, h2)


def loss_and_grads(params, x, t, rounding=True):
    """MSE loss and its gradients with respect to every parameter."""
    r = bf16 if rounding else _identity
    y, (x, z1, h1, z2, h2) = forward(params, x, rounding)
    B, M = y.shape
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (B * M)
    W2, W3 = r(params["W2"]), r(params["W3"])
    g = {}
    g["W3"] = r(dy).T @ r(h2)
    g["b3"] = dy.sum(0)
    dz2 = (r(dy) @ W3) * gelu_grad(z2)
    g["W2"] = r(dz2).T @ r(h1)
    g["b2"] = dz2.sum(0)
    dz1 = (r(dz2) @ W2) * gelu_grad(z1)
    g["W1"] = r(dz1).T @ r(x)
    g["b1"] = dz1.sum(0)
    return L, g


def init_params(rng, sizes=(6, 256, 256, 512)):
    """He-style initial weights (the same recipe the CUDA path is seeded with in tests)."""
    p = {}
    for i, (a, b) in enumerate(zip(sizes[:-1], sizes[1:]), start=1):
        p["W%d" % i] = rng.standard_normal((b, a)) * math.sqrt(2.0 / a)
        p["b%d" % i] = np.zeros(b)
    return p


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the FP64 master parameters (state: m, v, step)."""
    state["step"] = state.get("step", 0) + 1
    k = state["step"]
    for name, g in grads.items():
        m = state.setdefault("m_" + name, np.zeros_like(g))
        v = state.setdefault("v_" + name, np.zeros_like(g))
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** k)
        vh = v / (1 - beta2 ** k)
        params[name] = params[name] - lr * mh / (np.sqrt(vh) + eps)
    return params
