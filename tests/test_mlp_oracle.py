"""Pins of the CPU oracle of the learned warm start's network: its gradient against central
finite differences of its own loss, in FP64."""
import numpy as np

from oracle import mlp


def _params(rng):
    p = rng.normal(0, 0.2, mlp.NPARAM)
    p[mlp.SLICES["mu"]] = rng.normal(0, 1, mlp.NF)
    p[mlp.SLICES["sd"]] = rng.uniform(0.5, 2.0, mlp.NF)
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.normal(0, 1, (64, mlp.NF))
    y = rng.normal(0, 1, 64)
    loss, g = mlp.loss_and_gradient(p, X, y)
    assert loss == np.mean((mlp.forward(p, X) - y) ** 2)
    idx = np.concatenate([rng.choice(np.arange(mlp.SLICES[k].start, mlp.SLICES[k].stop), 6, replace=False)
                          for k in ("W1", "b1", "W2", "b2", "w3", "b3") for _ in [0] if mlp.SLICES[k].stop -
                          mlp.SLICES[k].start >= 6] + [np.array([mlp.SLICES["b3"].start])])
    eps = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = eps
        fd = (mlp.loss_and_gradient(p + e, X, y)[0] - mlp.loss_and_gradient(p - e, X, y)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
    assert np.all(g[mlp.SLICES["mu"]] == 0) and np.all(g[mlp.SLICES["sd"]] == 0)


def test_forward_of_a_linear_network():
    # ReLU layers acting on positive activations and identity-like weights reduce to a linear map
    p = np.zeros(mlp.NPARAM)
    p[mlp.SLICES["sd"]] = 1.0
    W1 = np.zeros((mlp.NF, mlp.NH))
    W1[np.arange(mlp.NF), np.arange(mlp.NF)] = 1.0
    W2 = np.eye(mlp.NH)
    p[mlp.SLICES["W1"]] = W1.ravel()
    p[mlp.SLICES["W2"]] = W2.ravel()
    w3 = np.zeros(mlp.NH)
    w3[:mlp.NF] = np.arange(mlp.NF)
    p[mlp.SLICES["w3"]] = w3
    p[mlp.SLICES["b3"]] = 0.5
    X = np.abs(np.random.default_rng(1).normal(size=(5, mlp.NF)))
    np.testing.assert_allclose(mlp.forward(p, X), X @ np.arange(mlp.NF) + 0.5, rtol=1e-14)
