"""Learned warm start on the GPU: tensor-core inference and training kernels against the FP64
oracle of the network, the exact constraint projection of the prediction, and what a trained
network gains over the plain method."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import paper_2506_08284_gb300 as pkg
from oracle import mlp

pytestmark = pytest.mark.gpu


def _params(rng, scale=0.15):
    p = rng.normal(0, scale, mlp.NPARAM).astype(np.float32)
    p[mlp.SLICES["mu"]] = rng.normal(0, 1, mlp.NF)
    p[mlp.SLICES["sd"]] = rng.uniform(0.5, 2.0, mlp.NF)
    return p


def test_inference_matches_oracle():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.normal(0, 1.5, (1000, mlp.NF)).astype(np.float32)     # not a multiple of the 128-row tile
    out = pkg.sphc.mlp_predict(p, X)
    ref = mlp.forward(p.astype(np.float64), X)
    # BF16 weights and activations: about three significant digits
    assert np.abs(out - ref).max() <= 3e-2 * (np.abs(ref).max() + 1e-3)
    assert np.corrcoef(out, ref)[0, 1] > 0.9999


def test_training_gradient_matches_oracle():
    rng = np.random.default_rng(1)
    p = _params(rng)
    X = rng.normal(0, 1, (777, mlp.NF)).astype(np.float32)
    y = rng.normal(0, 1, 777).astype(np.float32)
    g, loss = pkg.sphc.mlp_gradient(p, X, y)
    loss_ref, g_ref = mlp.loss_and_gradient(p.astype(np.float64), X, y)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        a, b = g[mlp.SLICES[k]], g_ref[mlp.SLICES[k]]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), k


def _hierarchy(p, **kw):
    o = pkg.sphc.default_opts(**kw)
    return pkg.sphc.setup((p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val),
                          (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val), p.coords, p.sigma_edge, o)


def _energy(h, p):
    rp, ci, v, shape = h.export(0, "Pe")
    P = sp.csr_matrix((v, ci, rp), shape=shape)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    return float((P.multiply(A @ P)).sum()), P


@pytest.fixture(scope="module")
def trained():
    from paper_2506_08284_gb300 import learned
    Xs, ys = [], []
    for m in range(6):
        spec = meshgen.MeshSpec(12 + 2 * m, jitter=0.2, seed_jitter=300 + m, sigma="lognormal", sigma_in=2.0,
                                seed_sigma=400 + m)
        X, y = learned.samples_from_mesh(spec, 30000, target_emin=4, seed=m)
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    params, hist = learned.train(X, y, steps=1500, batch=2048, lr=2e-3)
    return params, hist, float(y.var())


def test_training_reduces_loss(trained):
    params, hist, var = trained
    assert hist[-100:].mean() < 0.5 * hist[:20].mean()
    assert hist[-100:].mean() < var


def test_learned_warm_start_keeps_commuting_relation_and_gains(trained):
    params, _, _ = trained
    spec = meshgen.MeshSpec(24, jitter=0.2, seed_jitter=77, sigma="lognormal", sigma_in=2.0, seed_sigma=78)
    p = meshgen.generate(spec)
    b = meshgen.rhs(5, p.n_edges)
    res = {}
    for name, kw in [("P0", dict(emin_iters=0)), ("plain1", dict(emin_iters=1)), ("plain4", dict(emin_iters=4)),
                     ("learned0", dict(learned=1, learned_emin_iters=0, mlp_params=params)),
                     ("learned1", dict(learned=1, learned_emin_iters=1, mlp_params=params))]:
        h = _hierarchy(p, **kw)
        E, P = _energy(h, p)
        rp, ci, v, shape = h.export(0, "DH")
        DH = sp.csr_matrix((v, ci, rp), shape=shape)
        rp, ci, v, shape = h.export(0, "Pn")
        Pn = sp.csr_matrix((v, ci, rp), shape=shape)
        D = sp.csr_matrix((p.D_val, p.D_col, p.D_rowptr), shape=(p.n_edges, p.n_nodes))
        rhs = D @ Pn
        assert abs(P @ DH - rhs).max() <= 1e-12 * max(1.0, abs(rhs).max()), name
        x = np.zeros_like(b)
        rc, it, rr = h.solve(b, x)
        assert rc == 0, name
        res[name] = (E, it[0])
        h.destroy()
    print("A-energy / CG iterations:", res)
    # the network has learned a correction towards the minimiser: lower energy than the
    # least-norm start it corrects, and no worse than one plain step
    assert res["learned0"][0] < res["P0"][0]
    assert res["learned1"][0] <= res["plain1"][0] * 1.001
    assert res["learned1"][1] <= res["plain1"][1] + 1
