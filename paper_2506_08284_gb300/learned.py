"""Learned warm start of the edge prolongator: training data from plain energy minimisation on
seeded meshes, initialisation and GPU training through the C ABI (sphc_mlp_train), and the
stored parameters.  Not part of the paper.

Training recipe: meshes of n^3 cells with n uniform in [24, 64] (seed 100 + m), jitter uniform in
[0, 0.25] h, log-normal sigma (log10 sigma ~ N(0, 2^2) clipped to [-6, 2]); targets are
P_e - P0 after `target_emin` plain energy-minimisation steps on levels 0 and 1 (the setup applies
the network on every level); a fixed number of pattern entries is sampled from every level of
every mesh.
"""
from __future__ import annotations

import os

import numpy as np

from . import sphc

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "mlp_warmstart.npy")


def training_mesh(m: int):
    import meshgen
    rng = np.random.default_rng(100 + m)
    n = int(rng.integers(24, 65))
    jit = float(rng.uniform(0.0, 0.25))
    return meshgen.MeshSpec(n, jitter=jit, seed_jitter=1000 + m, sigma="lognormal", sigma_in=2.0,
                            seed_sigma=2000 + m)


def samples_from_mesh(spec, per_mesh: int, target_emin: int = 4, seed: int = 0, levels=(0,)):
    import meshgen
    p = meshgen.generate(spec)
    o = sphc.default_opts(emin_iters=target_emin, vcycle_fp32=1)
    h = sphc.setup((p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val),
                   (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val), p.coords, p.sigma_edge, o)
    Xs, ys = [], []
    for l in levels:
        if l + 1 >= h.nlevels:
            continue
        X, y = h.features(l)
        rng = np.random.default_rng(seed + 7 * l)
        k = min(per_mesh, X.shape[0])
        sel = rng.choice(X.shape[0], size=k, replace=False)
        Xs.append(X[sel])
        ys.append(y[sel])
    h.destroy()
    return np.concatenate(Xs), np.concatenate(ys)


def training_set(n_meshes: int = 40, per_mesh: int = 100_000, target_emin: int = 4, levels=(0,)):
    Xs, ys = [], []
    for m in range(n_meshes):
        X, y = samples_from_mesh(training_mesh(m), per_mesh, target_emin, seed=m, levels=levels)
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def init_params(X, seed: int = 0) -> np.ndarray:
    """Feature means/scales from the data, He-initialised weights, zero biases."""
    rng = np.random.default_rng(seed)
    nf, nh = sphc.MLP_NFEAT, sphc.MLP_HIDDEN
    mu = X.mean(0)
    sd = X.std(0)
    sd = np.where(sd > 1e-8, sd, 0.0)
    W1 = rng.normal(0, np.sqrt(2.0 / nf), (nf, nh))
    W2 = rng.normal(0, np.sqrt(2.0 / nh), (nh, nh))
    w3 = rng.normal(0, np.sqrt(1.0 / nh), nh) * 0.1
    parts = [mu, sd, W1.ravel(), np.zeros(nh), W2.ravel(), np.zeros(nh), w3, np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == sphc.MLP_NPARAM
    return p


def train(X, y, steps: int = 3000, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    params = init_params(X, seed)
    opts = sphc.default_train_opts(steps=steps, batch=batch, lr=lr, seed=seed + 1)
    hist = sphc.mlp_train(X, y, params, opts)
    return params, hist


def save(params, path: str = WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, np.asarray(params, np.float32))


def load_weights(path: str = WEIGHTS):
    return np.load(path).astype(np.float32) if os.path.exists(path) else None


if __name__ == "__main__":
    import sys
    import time
    n_meshes = int(sys.argv[1]) if len(sys.argv) > 1 else 40
    levels = tuple(int(v) for v in sys.argv[2].split(",")) if len(sys.argv) > 2 else (0, 1)
    t0 = time.time()
    X, y = training_set(n_meshes, levels=levels)
    t1 = time.time()
    params, hist = train(X, y)
    t2 = time.time()
    save(params)
    print(f"samples {X.shape[0]}  data {t1 - t0:.1f}s  train {t2 - t1:.1f}s  loss {hist[:5].mean():.3e} -> "
          f"{hist[-100:].mean():.3e}  target var {y.var():.3e}")
