"""Pins for the warm-start network reference: gradients against central finite differences,
the Adam step against its closed form on a quadratic, and bf16 rounding against exact cases."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    H = 8
    theta = rng.standard_normal(mlp.n_params(H)) * 0.5
    X = rng.standard_normal((40, 4))
    t = rng.standard_normal(40) * 0.3
    _, g = mlp.loss_and_grad(theta, X, t, H)
    eps = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = eps
        fd[i] = (mlp.loss_and_grad(theta + e, X, t, H)[0] - mlp.loss_and_grad(theta - e, X, t, H)[0]) / (2 * eps)
    assert np.abs(fd - g).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_adam_closed_form_first_step():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -4.0])
    th, m, v = mlp.adam_step(theta, np.zeros(2), np.zeros(2), g, 1, lr=0.1)
    # first step of Adam moves every coordinate by lr * sign(g) (up to eps)
    assert np.allclose(th, theta - 0.1 * np.sign(g), atol=1e-7)


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.5], dtype=np.float32)
    r = mlp.bf16_round(a)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie to even
    assert r[2] == np.float32(1.0 + 2 ** -7)
    assert r[3] == np.float32(1.0 + 2 ** -6)  # tie rounds up to even
    assert r[4] == -3.5
