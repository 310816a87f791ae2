"""Pins of the warm-start network's FP64 oracle: finite differences, closed forms, properties."""
import math

import numpy as np
import pytest

import cgp_inputs as ci
from oracle import mlp


def tiny(seed=3, n=17, hidden=8):
    params = [p.astype(np.float64) for p in ci.mlp_init_params(n, hidden, seed)]
    rng = np.random.default_rng(seed)
    params[1] = 0.1 * rng.standard_normal(hidden)
    params[3] = 0.1 * rng.standard_normal(hidden)
    params[5] = 0.1 * rng.standard_normal(n)
    b = rng.standard_normal((3, n))
    p = rng.standard_normal((3, n))
    mask = np.ones(n)
    mask[0] = 0.0
    return params, b, p, mask


def test_gradients_match_central_differences():
    params, b, p, mask = tiny()
    L, grads = mlp.loss_and_grads(params, b, p, mask)
    h = 1e-6
    for k, (P, G) in enumerate(zip(params, grads)):
        flat = P.reshape(-1)
        num = np.zeros_like(flat)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            Lp, _ = mlp.loss_and_grads(params, b, p, mask)
            flat[i] = old - h
            Lm, _ = mlp.loss_and_grads(params, b, p, mask)
            flat[i] = old
            num[i] = (Lp - Lm) / (2 * h)
        err = np.linalg.norm(num - G.reshape(-1)) / max(np.linalg.norm(num), 1e-30)
        assert err < 1e-6, (k, err)


def test_gelu_closed_forms():
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-15
    z = np.linspace(-6, 6, 101)
    # tanh form: gelu(z) - gelu(-z) = z exactly (odd part), and gelu(z) -> z for large z
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    assert abs(mlp.gelu(30.0) - 30.0) < 1e-12 and abs(mlp.gelu(-30.0)) < 1e-12
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding_special_cases():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1.0 + 2 ** -7])
    got = mlp.bf16_round(x)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, -2.5, 0.0, 1.0 + 2 ** -7])   # ties to even
    np.testing.assert_array_equal(got, want)
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0).standard_normal(1000) * 100
    ref = torch.tensor(r, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(r), ref)


def test_homogeneous_in_the_right_hand_side():
    params, b, _, mask = tiny()
    p1, _ = mlp.forward(params, b, mask)
    p2, _ = mlp.forward(params, 7.5 * b, mask)
    np.testing.assert_allclose(p2, 7.5 * p1, rtol=1e-13)
    assert np.all(p1[:, 0] == 0.0)


def test_adam_first_step_is_signed_lr():
    P = [np.array([1.0, -2.0, 3.0])]
    G = [np.array([0.5, -4.0, 1e-3])]
    Pn, m, v = mlp.adam_step(P, G, [np.zeros(3)], [np.zeros(3)], 1, lr=0.01)
    np.testing.assert_allclose(Pn[0], P[0] - 0.01 * np.sign(G[0]), atol=1e-7)
