"""ORACLE (test infrastructure) of the learned warm start's network: forward pass and gradient of
the mean squared error in plain FP64 numpy, with the parameter layout of include/sphc.h:
feature means [32], scales [32], W1 [32 x 128], b1 [128], W2 [128 x 128], b2 [128], w3 [128], b3.
"""
import numpy as np

NF, NH = 32, 128
SLICES = {}
_o = 0
for _name, _n in [("mu", NF), ("sd", NF), ("W1", NF * NH), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("w3", NH),
                  ("b3", 1)]:
    SLICES[_name] = slice(_o, _o + _n)
    _o += _n
NPARAM = _o


def unpack(params):
    p = np.asarray(params, np.float64)
    return dict(mu=p[SLICES["mu"]], sd=p[SLICES["sd"]], W1=p[SLICES["W1"]].reshape(NF, NH), b1=p[SLICES["b1"]],
                W2=p[SLICES["W2"]].reshape(NH, NH), b2=p[SLICES["b2"]], w3=p[SLICES["w3"]], b3=p[SLICES["b3"]][0])


def normalise(P, X):
    sd = P["sd"]
    inv = np.where(sd > 0, 1.0 / np.where(sd > 0, sd, 1.0), 0.0)
    return (np.asarray(X, np.float64) - P["mu"]) * inv


def forward(params, X):
    P = unpack(params)
    x = normalise(P, X)
    z1 = x @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    return h2 @ P["w3"] + P["b3"]


def loss_and_gradient(params, X, y):
    """Mean squared error and its gradient (zero for the normalisation entries)."""
    P = unpack(params)
    x = normalise(P, X)
    B = x.shape[0]
    z1 = x @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ P["w3"] + P["b3"]
    e = out - np.asarray(y, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    g = np.zeros(NPARAM)
    g[SLICES["w3"]] = h2.T @ dy
    g[SLICES["b3"]] = dy.sum()
    dz2 = np.outer(dy, P["w3"]) * (z2 > 0)
    g[SLICES["W2"]] = (h1.T @ dz2).ravel()
    g[SLICES["b2"]] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"].T) * (z1 > 0)
    g[SLICES["W1"]] = (x.T @ dz1).ravel()
    g[SLICES["b1"]] = dz1.sum(0)
    return loss, g
