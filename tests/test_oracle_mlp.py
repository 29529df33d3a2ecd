"""Pins of the warm-start network's oracle: GELU, BF16 rounding, back-propagation by
finite differences, and the closed form of Adam's first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding():
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0                 # tie, rounds to even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie, rounds up to even mantissa
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7       # representable
    assert mlp.bf16(-3.0) == -3.0
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2 ** -8)


def test_gelu_closed_form():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15  # Phi(1)
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-9)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(rng, sizes=(6, 16, 12, 10))
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((7, 6))
    t = rng.standard_normal((7, 10))
    L, g = mlp.loss_and_grads(p, x, t, rounding=False)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp = mlp.loss_and_grads(p, x, t, rounding=False)[0]
            flat[idx] = old - h
            Lm = mlp.loss_and_grads(p, x, t, rounding=False)[0]
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (name, idx)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    p = {"W": rng.standard_normal((3, 4))}
    g = {"W": rng.standard_normal((3, 4))}
    old = p["W"].copy()
    st = {}
    mlp.adam_step(p, g, st, lr=0.01)
    # m_hat = g, v_hat = g^2: the step is lr g / (|g| + eps)
    assert np.allclose(p["W"], old - 0.01 * np.sign(g["W"]), rtol=0, atol=1e-8)


def test_gpu_error_bounds_catch_a_wrong_column():
    """The element-wise check of the GPU network (tests/test_gpu_mlp.py) has the power to
    see a plausible kernel mistake: a gradient whose column k of W1 is replaced by
    column k+1 (planted in the oracle's own gradient, on the CPU), or a bias gradient
    with one row doubled, fails it."""
    from tests.test_gpu_mlp import _within, error_bounds
    om = mlp
    rng = np.random.default_rng(7)
    sizes, B = (6, 32, 32, 40), 37
    p = om.init_params(rng, sizes)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x, t = rng.standard_normal((B, 6)), rng.standard_normal((B, 40))
    E = error_bounds(p, x, t)
    _, g = om.loss_and_grads(p, x, t)
    assert all(_within(g[k], g[k], E[k]) for k in g)
    wrong = g["W1"].copy()
    wrong[:, 2] = g["W1"][:, 3]
    assert not _within(wrong, g["W1"], E["W1"])
    wrong = g["b2"].copy()
    wrong[5] *= 2.0
    assert not _within(wrong, g["b2"], E["b2"])
