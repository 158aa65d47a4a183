"""Pins of the FP64 network oracle (oracle/mlp.py) used to check the GPU trainer.

The analytic gradient is checked against central finite differences; the
forward pass against closed forms (SiLU values; a network with zero weights
returns 1 + b3).
"""
import numpy as np

from oracle import mlp


def _rand_theta(rng, scale=0.3):
    return rng.normal(0.0, scale, mlp.N_PARAMS)


def test_parameter_count_and_silu():
    assert mlp.N_PARAMS == 7491
    z = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=0, atol=1e-15)
    assert mlp.silu(np.array([0.0]))[0] == 0.0


def test_zero_weights_give_bias():
    th = np.zeros(mlp.N_PARAMS)
    th[-3:] = [0.1, -0.2, 0.3]
    X = np.random.default_rng(0).uniform(0.05, 2.0, (5, 48))
    assert np.allclose(mlp.forward(th, X), 1.0 + th[-3:], atol=1e-15)


def test_analytic_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    th = _rand_theta(rng)
    X = rng.uniform(0.05, 2.0, (40, 48))
    T = rng.uniform(0.1, 2.0, (40, 3))
    loss, g = mlp.loss_grad(th, X, T)
    h = 1e-6
    idx = np.concatenate([rng.choice(48 * 64, 25, replace=False),          # W1
                          48 * 64 + rng.choice(64, 5, replace=False),        # b1
                          48 * 64 + 64 + rng.choice(64 * 64, 25, replace=False),
                          48 * 64 + 64 + 64 * 64 + rng.choice(64, 5, replace=False),
                          mlp.N_PARAMS - 3 - 192 + rng.choice(192, 10, replace=False),
                          mlp.N_PARAMS - 3 + np.arange(3)])
    for q in idx:
        tp, tm = th.copy(), th.copy()
        tp[q] += h
        tm[q] -= h
        fd = (mlp.loss_grad(tp, X, T)[0] - mlp.loss_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 + 1e-6 * abs(g[q]), (q, fd, g[q])
    # the loss is the stated mean squared error
    y = mlp.forward(th, X)
    assert abs(loss - ((y - T) ** 2).mean()) < 1e-12
