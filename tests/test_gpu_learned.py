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


@pytest.mark.parametrize("which", ["trained", "random"])
def test_fused_inference_matches_oracle(which):
    # the kernel setup runs: features computed in the tensor-core kernel from the level's
    # operators, against the network's FP64 definition on the exported FP32 features
    from paper_2506_08284_gb300 import learned
    spec = meshgen.MeshSpec(12, jitter=0.2, seed_jitter=31, sigma="lognormal", sigma_in=2.0, seed_sigma=32)
    p = meshgen.generate(spec)
    params = learned.load_weights() if which == "trained" else _params(np.random.default_rng(5), 0.1)
    h = _hierarchy(p, max_coarse=100)
    for level in range(h.nlevels - 1):
        X, _ = h.features(level)
        out = h.predict_level(params, level)
        ref = mlp.forward(np.asarray(params, np.float64), X)
        assert out.shape == ref.shape and np.all(np.isfinite(out))
        assert np.abs(out - ref).max() <= 3e-2 * (np.abs(ref).max() + 1e-3), level
        assert np.corrcoef(out, ref)[0, 1] > 0.999, level
    h.destroy()


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
    assert res["learned1"][1] <= res["plain1"][1]


def test_exported_features_follow_their_definitions():
    """The features (include/sphc.h) restated in numpy from the exported level arrays: unit edge
    tangent, single-node flag, row sizes, A_e row scaling, log10 sigma, and the six T / P_n
    lookups at the coarse edge's ends (tail = lower node id, a single node is the head)."""
    spec = meshgen.MeshSpec(10, jitter=0.15, seed_jitter=3, sigma="lognormal", sigma_in=2.0, seed_sigma=4)
    p = meshgen.generate(spec)
    h = _hierarchy(p, max_coarse=100)
    X, y = h.features(0)
    csr = lambda name: (lambda rp, ci, v, shape: sp.csr_matrix((v, ci, rp), shape=shape))(*h.export(0, name))
    N, T, DH, Pn = csr("Pe"), csr("T"), csr("DH"), csr("Pn")
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    D = sp.csr_matrix((p.D_val, p.D_col, p.D_rowptr))
    rows = np.repeat(np.arange(N.shape[0]), np.diff(N.indptr))
    cols = N.indices
    assert X.shape == (N.nnz, 32)
    # edge ends and tangent
    two = np.diff(D.indptr)[rows] == 2
    np.testing.assert_array_equal(X[:, 0], two.astype(np.float32))
    norms = np.linalg.norm(X[two, 1:4], axis=1)
    np.testing.assert_allclose(norms, 1.0, atol=1e-5)
    # coarse edge ends by the orientation of D_H
    hl = np.diff(DH.indptr)[cols]
    first = DH.indices[DH.indptr[cols]]
    second = DH.indices[np.minimum(DH.indptr[cols] + 1, DH.nnz - 1)]
    ja = np.where(hl == 2, first, -1)
    jb = np.where(hl == 2, second, first)
    np.testing.assert_array_equal(X[:, 10], (hl == 1).astype(np.float32))
    np.testing.assert_allclose(X[:, 11], np.diff(N.indptr)[rows] / 32.0, rtol=1e-6)
    np.testing.assert_allclose(X[:, 12], np.diff(T.indptr)[rows] / 16.0, rtol=1e-6)
    # lookups: T at (i, ja / jb), P_n at (u / v, ja / jb)
    Td, Pd = T.tolil(), Pn.tocsr()
    look = lambda M, r, c: np.array([M[a, b] if a >= 0 and b >= 0 else 0.0 for a, b in zip(r, c)])
    np.testing.assert_allclose(X[:, 13], look(Td, rows, ja), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(X[:, 14], look(Td, rows, jb), rtol=1e-6, atol=1e-7)
    u = np.full(D.shape[0], -1)
    v = np.full(D.shape[0], -1)
    for i in range(D.shape[0]):
        for k in range(D.indptr[i], D.indptr[i + 1]):
            if D.data[k] < 0: u[i] = D.indices[k]
            else: v[i] = D.indices[k]
    np.testing.assert_allclose(X[:, 15], look(Pd, u[rows], ja), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(X[:, 16], look(Pd, u[rows], jb), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(X[:, 17], look(Pd, v[rows], ja), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(X[:, 18], look(Pd, v[rows], jb), rtol=1e-6, atol=1e-7)
    assert np.all(X[:, 19] == 0)
    # A_e row scaling and sigma
    diag = A.diagonal()
    l1 = np.asarray(abs(A).sum(axis=1)).ravel()
    np.testing.assert_allclose(X[:, 20], (diag / l1)[rows], rtol=1e-5)
    np.testing.assert_allclose(X[:, 21], (np.log10(p.sigma_edge) / 6.0)[rows], rtol=1e-5, atol=1e-6)
    h.destroy()


def test_prolongator_energy_and_vcycle_factor():
    """The two yardsticks of the learned warm start, against host computations: trace(P^T A P)
    from the exported matrices (scipy), and the V-cycle's contraction factor restated with the
    oracle's V-cycle from the same splitmix64 start vector (FP64 V-cycle on both sides)."""
    import oracle
    from prio import splitmix64
    spec = meshgen.MeshSpec(8, jitter=0.2, seed_jitter=5, sigma="lognormal", sigma_in=1.0, seed_sigma=6)
    p = meshgen.generate(spec)
    h = _hierarchy(p, vcycle_fp32=0, max_coarse=100)
    E, _ = _energy(h, p)
    assert h.energy(0) == pytest.approx(E, rel=1e-12)
    f = h.vcycle_factor(30, 10, seed=3)
    o = oracle.setup_problem(p, max_coarse=100)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    x = np.array([2.0 * ((splitmix64(3, i) >> 11) * 2.0**-53) - 1.0 for i in range(p.n_edges)])
    en = lambda v: np.sqrt(v @ (A @ v))
    e_prev, logs = en(x), []
    for k in range(30):
        x = x + o.vcycle(-(A @ x))
        e = en(x)
        logs.append(np.log(e / e_prev))
        e_prev = e
    f_ref = float(np.exp(np.mean(logs[-10:])))
    assert 0.0 < f < 1.0
    assert f == pytest.approx(f_ref, rel=1e-6)
