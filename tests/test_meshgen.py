"""Pins of the synthetic input generator against closed forms and the paper's mesh sizes."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen


def _csr(rp, ci, v, shape):
    return sp.csr_matrix((v, ci, rp), shape=shape)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8])
def test_count_polynomials(n):
    c = meshgen.counts(meshgen.MeshSpec(n))
    assert c["n_edges"] == 7 * n**3 - 9 * n**2 + 3 * n
    assert c["nnz_A"] == 115 * n**3 - 261 * n**2 + 195 * n - 48
    assert c["n_nodes"] == (n - 1) ** 3
    cn = meshgen.counts(meshgen.MeshSpec(n, natural=True))
    assert cn["n_edges"] == 7 * n**3 + 9 * n**2 + 3 * n
    assert cn["n_nodes"] == (n + 1) ** 3
    p = meshgen.generate(meshgen.MeshSpec(n), with_matrix=False)
    single = int(np.sum(np.diff(p.D_rowptr) == 1))
    assert single == 24 * n**2 - 60 * n + 38


def test_paper_tet_edge_counts():
    # Table of 3D tetrahedral results (Sec. 6.1): 10^3, 28^3, 82^3 nodal meshes -> 5,859 / 144,423 /
    # 3,779,379 edges with natural boundary conditions.
    for nodes, edges in [(10, 5859), (28, 144423), (82, 3779379)]:
        p = meshgen.generate(meshgen.MeshSpec(nodes - 1, natural=True), with_matrix=False)
        assert p.n_edges == edges


@pytest.mark.parametrize("natural", [True, False])
def test_curl_of_gradient_vanishes(natural):
    # S_h D_h = 0 (Sec. 1, eq. (3)), to rounding.
    spec = meshgen.MeshSpec(4, natural=natural, jitter=0.2, seed_jitter=3)
    S = meshgen.generate(spec, which="S")
    Sm = _csr(S.A_rowptr, S.A_col, S.A_val, (S.n_edges, S.n_edges))
    D = _csr(S.D_rowptr, S.D_col, S.D_val, (S.n_edges, S.n_nodes))
    assert abs(Sm @ D).max() <= 1e-12 * abs(Sm).max()
    assert abs(Sm - Sm.T).max() <= 1e-14 * abs(Sm).max()


def _p1_stiffness(X, tets, sigma, nall):
    """sigma-weighted P1 stiffness int sigma grad phi_i . grad phi_j, assembled element by element."""
    rows, cols, vals = [], [], []
    for t, s in zip(tets, sigma):
        P = X[t]
        J = (P[1:] - P[0]).T           # columns v_k - v_0
        G = np.linalg.inv(J)           # rows = grad lambda_1..3
        grads = np.vstack([-G.sum(0), G])
        vol = abs(np.linalg.det(J)) / 6
        K = s * vol * grads @ grads.T
        for a in range(4):
            for b in range(4):
                rows.append(t[a]); cols.append(t[b]); vals.append(K[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nall, nall))


@pytest.mark.parametrize("natural", [True, False])
def test_mass_on_gradients_is_p1_stiffness(natural):
    # D_h^T M_sigma D_h equals the sigma-weighted nodal P1 stiffness (the gradient of a P1
    # function is a Whitney field whose edge values are D_h times its nodal values).
    spec = meshgen.MeshSpec(3, natural=natural, jitter=0.2, seed_jitter=5, sigma="lognormal",
                            sigma_in=1.0, seed_sigma=9)
    M = meshgen.generate(spec, which="M", raw_mesh=True)
    Mm = _csr(M.A_rowptr, M.A_col, M.A_val, (M.n_edges, M.n_edges))
    D = _csr(M.D_rowptr, M.D_col, M.D_val, (M.n_edges, M.n_nodes))
    X, tets, sig = M.extra["coords_all"], M.extra["tets"], M.extra["tet_sigma"]
    K = _p1_stiffness(X, tets, sig, X.shape[0])
    n = spec.n
    N = n + 1
    g = np.arange(N**3)
    i, j, k = g % N, (g // N) % N, g // (N * N)
    keep = g if natural else g[(i > 0) & (j > 0) & (k > 0) & (i < n) & (j < n) & (k < n)]
    K = K[keep][:, keep]
    lhs = (D.T @ Mm @ D).toarray()
    assert np.abs(lhs - K.toarray()).max() <= 1e-12 * np.abs(K.toarray()).max()


def test_constant_field():
    # For a constant field c, u_e = c.(x_head - x_tail) is curl-free (S u = 0) and
    # u^T M u = sum_T sigma_T |T| |c|^2.
    spec = meshgen.MeshSpec(3, natural=True, jitter=0.2, seed_jitter=1, sigma="lognormal",
                            sigma_in=1.0, seed_sigma=2)
    S = meshgen.generate(spec, which="S", raw_mesh=True)
    M = meshgen.generate(spec, which="M")
    X, tets, sig = S.extra["coords_all"], S.extra["tets"], S.extra["tet_sigma"]
    c = np.array([0.3, -1.2, 0.7])
    u = (X[S.edge_ends[:, 1]] - X[S.edge_ends[:, 0]]) @ c
    Sm = _csr(S.A_rowptr, S.A_col, S.A_val, (S.n_edges, S.n_edges))
    Mm = _csr(M.A_rowptr, M.A_col, M.A_val, (M.n_edges, M.n_edges))
    assert np.abs(Sm @ u).max() <= 1e-12 * abs(Sm).max()
    vols = np.abs(np.linalg.det(X[tets[:, 1:]] - X[tets[:, :1]])) / 6
    assert u @ (Mm @ u) == pytest.approx(np.sum(sig * vols) * (c @ c), rel=1e-12)


def test_jitter_keeps_volumes_positive():
    spec = meshgen.MeshSpec(6, jitter=0.2, seed_jitter=11)
    p = meshgen.generate(spec, raw_mesh=True)
    X, tets = p.extra["coords_all"], p.extra["tets"]
    det = np.linalg.det(X[tets[:, 1:]] - X[tets[:, :1]])
    ref = np.linalg.det(meshgen.generate(meshgen.MeshSpec(6), raw_mesh=True).extra["coords_all"][tets[:, 1:]]
                        - meshgen.generate(meshgen.MeshSpec(6), raw_mesh=True).extra["coords_all"][tets[:, :1]])
    assert np.all(np.sign(det) == np.sign(ref)) and np.all(np.abs(det) > 0)


def test_sigma_fields():
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    assert np.all(p.sigma_edge == 1.0)
    spec = meshgen.MeshSpec(8, sigma="lognormal", sigma_in=2.0, seed_sigma=5)
    q = meshgen.generate(spec, raw_mesh=True)
    ls = np.log10(q.extra["tet_sigma"])
    assert ls.min() >= -6 - 1e-12 and ls.max() <= 2 + 1e-12
    # moments of clip(N(0, 2^2), -6, 2)
    from scipy import stats
    z = np.linspace(-12, 12, 200001)
    w = stats.norm.pdf(z, scale=2.0)
    w /= w.sum()
    zc = np.clip(z, -6, 2)
    mu = (w * zc).sum()
    sd = np.sqrt((w * (zc - mu) ** 2).sum())
    assert abs(ls.mean() - mu) < 0.05 and abs(ls.std() - sd) < 0.05
    b = meshgen.rhs(6, 1000)
    assert b.min() >= -1 and b.max() <= 1 and abs(b.mean()) < 0.1
