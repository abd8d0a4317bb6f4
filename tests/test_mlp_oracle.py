"""Pins of the FP64 network reference (oracle/mlp_oracle.py): its backward pass
against central finite differences of its own loss, its feature map against
the definition, and its parameter count."""
import numpy as np

from oracle import mlp_oracle as mo


def test_parameter_count():
    assert mo.N_PARAMS == 3 * (64 * 64 + 64) + 64 * 8 + 8 == 13000


def test_features_definition():
    B = np.array([[1.0, 0.0], [0.5, -2.0]] + [[0.0, 0.0]] * 30)
    x = np.array([[0.25, 0.5]])
    f = mo.features(x, B)
    assert np.isclose(f[0, 0], np.sin(np.pi * 0.25)) and np.isclose(f[0, 32], np.cos(np.pi * 0.25))
    assert np.isclose(f[0, 1], np.sin(np.pi * (0.125 - 1.0)))
    assert np.isclose(f[0, 2], 0.0) and np.isclose(f[0, 34], 1.0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    B = rng.normal(0, 3.0, (32, 2))
    theta = mo.init_params(1) + rng.normal(0, 0.05, mo.N_PARAMS)
    x = rng.uniform(-1, 1, (7, 2))
    t = rng.normal(0, 1, (7, 8))
    g = mo.backward(theta, B, x, t)
    h = 1e-6
    for k in list(rng.choice(mo.N_PARAMS, 40, replace=False)) + [0, 4159, 12999, 12480]:
        e = np.zeros(mo.N_PARAMS)
        e[k] = h
        fd = (mo.loss(theta + e, B, x, t) - mo.loss(theta - e, B, x, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-6 * abs(fd), k
