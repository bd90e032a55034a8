"""Pins of the FP64 surrogate-network oracle: finite differences, closed-form
derivatives, the bfloat16 rounding definition, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp


def test_silu_derivative_closed_form():
    z = np.linspace(-8, 8, 41)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.silu_grad(z))) < 1e-8
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu_grad(0.0) - 0.5) < 1e-15


def test_one_hidden_unit_network_by_hand():
    # all weights zero except W1[0,0] = a, W2[0,0] = b, W3[0,0] = c: the
    # output is c * SiLU(b * SiLU(a * x0)) in output 0, biases elsewhere
    theta = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    a, b, c = 0.7, -1.3, 2.1
    W1[0, 0], W2[0, 0], W3[0, 0] = a, b, c
    b3[:] = [0.1, 0.2, 0.3, 0.4]
    th = mlp.pack([W1, b1, W2, b2, W3, b3])
    x = np.array([[0.9, 5, 6, 7, 8]])
    o, _ = mlp.forward(th, x)
    s = lambda v: v / (1 + np.exp(-v))
    hidden = b * s(a * 0.9)
    # unit 0 of layer 2 sees b * SiLU(a x0); every other unit of layer 2 has
    # zero input and SiLU(0) = 0
    assert abs(o[0, 0] - (c * s(hidden) + 0.1)) < 1e-14
    assert np.allclose(o[0, 1:], [0.2, 0.3, 0.4], atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_analytic_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed)
    theta += rng.normal(0, 0.01, size=theta.shape)  # nonzero biases
    x = rng.normal(size=(7, 5))
    t = rng.normal(size=(7, 4))
    g, _ = mlp.backward(theta, x, t)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [0, mlp.N_PARAMS - 1]])
    fd = mlp.finite_difference_grad(theta, x, t, idx)
    assert np.max(np.abs(fd - g[idx])) <= 1e-7 * max(1.0, np.max(np.abs(g[idx])))


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 3.0e38, 1e-40], np.float32)
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # exact tie rounds to even (down)
    assert r[2] == 1.0 + 2 ** -7            # representable
    assert r[3] == 1.0 + 2 ** -6            # tie rounds to even (up)
    assert r[4] == -2.5 and r[5] == 0.0
    # bfloat16 has an 8-bit exponent: large values stay finite, 7 fraction bits
    assert np.isfinite(r[6]) and abs(r[6] / 3.0e38 - 1) < 2 ** -8
    rng = np.random.default_rng(3)
    x = rng.normal(size=10000).astype(np.float32)
    rel = np.abs(mlp.bf16_round(x) - x) / np.abs(x)
    assert rel.max() <= 2 ** -8 + 1e-12


def test_adam_first_step_moves_each_parameter_by_lr():
    # with bias correction the first step is lr * g / (|g| + eps) = lr * sign(g)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01, eps=1e-12)
    assert np.allclose(th[:3], -0.01 * np.sign(g[:3]), rtol=1e-6) and th[3] == 0.0


def test_weight_average_closed_form():
    # a constant weight c, averaged from a0 over k steps: c + (a0 - c) d^k;
    # with decay 0 the average is the latest weight, with decay 1 the start
    a, c, d = np.array([2.0, -1.0]), np.array([0.5, 3.0]), 0.9
    avg = a.copy()
    for _ in range(25):
        avg = mlp.weight_average(avg, c, d)
    assert np.allclose(avg, c + (a - c) * d ** 25, rtol=1e-12)
    assert np.array_equal(mlp.weight_average(a, c, 0.0), c)
    assert np.array_equal(mlp.weight_average(a, c, 1.0), a)
