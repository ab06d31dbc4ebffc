"""Pins of the CPU oracle against what the paper and the mathematics fix."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import oracle
from conftest import load_golden_matrices
from prio import adjacency, jp_colour, mis2_rounds


# ---------------------------------------------------------------- local least-norm systems
@pytest.mark.parametrize("name", ["fig2a", "fig2b", "fig2c", "fig2d"])
def test_fig2_local_systems(name):
    G, rank = load_golden_matrices("fig2_local_dh.txt")[name]
    assert np.linalg.matrix_rank(G) == rank == G.shape[1] - 1       # Sec. 4.2 text
    rng = np.random.default_rng(1)
    r = G.T @ rng.normal(size=G.shape[0])                             # consistent right side
    p = oracle.minnorm(G, r, singular=True)
    np.testing.assert_allclose(G.T @ p, r, atol=1e-13)
    np.testing.assert_allclose(p, np.linalg.pinv(G.T) @ r, atol=1e-13)   # library least-norm
    x = rng.normal(size=G.shape[0])
    y = oracle.project(G, x, singular=True)
    np.testing.assert_allclose(G.T @ y, 0, atol=1e-13)
    np.testing.assert_allclose(y, x - G @ np.linalg.pinv(G) @ x, atol=1e-13)


def test_fig2_with_dirichlet_edge_is_full_rank():
    G, _ = load_golden_matrices("fig2_local_dh.txt")["fig2c"]
    Gd = np.vstack([G, np.eye(6)[2]])            # a single-node (Dirichlet) coarse edge
    r = np.arange(6.0)                           # any right side is consistent now
    p = oracle.minnorm(Gd, r, singular=False)
    np.testing.assert_allclose(Gd.T @ p, r, atol=1e-12)
    np.testing.assert_allclose(p, np.linalg.lstsq(Gd.T, r, rcond=None)[0], atol=1e-12)


def test_fig3_is_infeasible():
    G, rank = load_golden_matrices("fig2_local_dh.txt")["fig3"]
    assert np.linalg.matrix_rank(G) == rank and G.shape[1] - rank == 2   # two-dimensional null space
    with pytest.raises(RuntimeError):
        oracle.minnorm(G, np.array([1.0, -1.0, 0.5, -0.5]), singular=True)


# ---------------------------------------------------------------- integer steps
def _graph(n):
    h = oracle.setup_problem(meshgen.generate(meshgen.MeshSpec(n, jitter=0.2, seed_jitter=1)), max_levels=2)
    return h.matrix(0, "An"), h.matrix(0, "A")


def test_aggregation_matches_parallel_rounds():
    An, _ = _graph(6)
    adj = adjacency(An.rowptr, An.col)
    for seed in (1, 7, 1001):
        agg, nagg = oracle.aggregate(An.rowptr, An.col, seed)
        roots = mis2_rounds(adj, seed)
        assert nagg == len(roots)
        # aggregate ids follow root ids; each root heads its own aggregate
        assert [agg[r] for r in sorted(roots)] == list(range(nagg))
        # root + neighbours
        for r in roots:
            assert all(agg[w] == agg[r] for w in adj[r])
        # every node is assigned, every aggregate is connected
        for a in range(nagg):
            members = set(np.nonzero(agg == a)[0].tolist())
            start = next(iter(members))
            seen, stack = {start}, [start]
            while stack:
                v = stack.pop()
                for w in adj[v]:
                    if w in members and w not in seen:
                        seen.add(w); stack.append(w)
            assert seen == members


def test_leftover_nodes_join_most_connected_aggregate():
    An, _ = _graph(5)
    adj = adjacency(An.rowptr, An.col)
    agg, nagg = oracle.aggregate(An.rowptr, An.col, 3)
    roots = mis2_rounds(adj, 3)
    core = {r: r for r in roots}
    phase2 = {}
    for r in roots:
        phase2[r] = r
        for w in adj[r]:
            phase2[w] = r
    rid = {r: i for i, r in enumerate(sorted(roots))}
    for v in range(len(adj)):
        if v in phase2:
            assert agg[v] == rid[phase2[v]]
        else:
            counts = {}
            for w in adj[v]:
                if w in phase2:
                    counts[rid[phase2[w]]] = counts.get(rid[phase2[w]], 0) + 1
            best = max(counts.values())
            assert agg[v] == min(a for a, c in counts.items() if c == best)


def test_colouring_matches_jones_plassmann():
    An, A = _graph(4)
    for M in (An, A):
        adj = adjacency(M.rowptr, M.col)
        col, nc = oracle.color(M.rowptr, M.col, 42)
        ref = jp_colour(adj, 42)
        np.testing.assert_array_equal(col, ref)
        assert nc == col.max() + 1
        for v in range(len(adj)):
            assert all(col[v] != col[w] for w in adj[v])


def _blocks(n):
    """3-node blocks per axis {0,1},{2,3,4},...,{n-1,n} on the (n+1)^3 natural-BC grid."""
    N = n + 1
    b = np.zeros(N, int)
    k, idx = 1, 2
    while idx < N:
        b[idx:idx + 3] = k
        idx += 3
        k += 1
    nb = b.max() + 1
    g = np.arange(N**3)
    i, j, kk = g % N, (g // N) % N, g // (N * N)
    return (b[i] + nb * (b[j] + nb * b[kk])).astype(np.int32), int(nb**3)


@pytest.mark.parametrize("n,expected", [(27, 5859), (81, 144423)])
def test_rs_coarse_edges_of_block_aggregates(n, expected):
    # 3-node blocks on the 82^3 (28^3) nodal Kuhn mesh coarsen to the 28^3 (10^3) Kuhn mesh;
    # eq. (4) then yields exactly its edges, the level-1 (level-2) prolongator row count of the
    # 3D least-squares table (Sec. 6.1): 144,423 (and 5,859 edges of the 10^3 mesh).
    p = meshgen.generate(meshgen.MeshSpec(n, natural=True), with_matrix=False)
    agg, nagg = _blocks(n)
    H = oracle.coarse_gradient(p.n_edges, p.n_nodes, (p.D_rowptr, p.D_col, p.D_val), agg, nagg)
    assert H.shape[0] == expected
    assert np.all(np.diff(H.rowptr) == 2)


# ---------------------------------------------------------------- hierarchy invariants
@pytest.fixture(scope="module")
def hier12():
    spec = meshgen.MeshSpec(12, jitter=0.2, seed_jitter=4, sigma="lognormal", sigma_in=2.0, seed_sigma=5)
    p = meshgen.generate(spec)
    S = meshgen.generate(spec, which="S")
    h = oracle.setup_problem(p, max_coarse=200)
    return p, S, h


def _sp(m):
    return m.to_scipy()


def test_hierarchy_has_levels(hier12):
    _, _, h = hier12
    assert h.status == 0 and h.nlevels >= 3


def test_commuting_relation(hier12):
    # P_e D_H = D_h P_n (eq. (6)) to 1e-12 on every level
    _, _, h = hier12
    for l in range(h.nlevels - 1):
        Pe, DH, D, Pn = (_sp(h.matrix(l, k)) for k in ("Pe", "DH", "D", "Pn"))
        rhs = D @ Pn
        assert abs(Pe @ DH - rhs).max() <= 1e-12 * max(1.0, abs(rhs).max())
        P0 = _sp(h.matrix(l, "P0"))
        assert abs(P0 @ DH - rhs).max() <= 1e-12 * max(1.0, abs(rhs).max())


def test_nodal_prolongator_definition(hier12):
    # P_n = rowscale((I - w D^-1 A_n) Pbar), rows sum to one (Sec. 4.2)
    _, _, h = hier12
    for l in range(h.nlevels - 1):
        An, Pn = _sp(h.matrix(l, "An")), _sp(h.matrix(l, "Pn"))
        agg = h.ivec(l, "agg")
        Pb = sp.csr_matrix((np.ones(len(agg)), (np.arange(len(agg)), agg)), shape=Pn.shape)
        w = h.scalars(l)["omega_sa"]
        Q = (Pb - w * sp.diags(1 / An.diagonal()) @ An @ Pb).tocsr()
        rs = np.asarray(Q.sum(1)).ravel()
        keep = rs > 0.125                      # rows below this keep their tentative values
        Q = sp.diags(np.where(keep, 1 / np.where(keep, rs, 1), 0)) @ Q + sp.diags((~keep).astype(float)) @ Pb
        assert abs(Q - Pn).max() <= 1e-13
        assert (~keep).sum() == h.sizes(l)["n_rows_unsmoothed"]
        np.testing.assert_allclose(np.asarray(Pn.sum(1)).ravel(), 1.0, atol=1e-14)


def test_coarse_gradient_structure(hier12):
    _, _, h = hier12
    for l in range(h.nlevels - 1):
        DH = h.matrix(l, "DH")
        lens = np.diff(DH.rowptr)
        assert set(np.unique(lens)) <= {1, 2}
        two = np.nonzero(lens == 2)[0]
        tails = DH.col[DH.rowptr[two]]
        heads = DH.col[DH.rowptr[two] + 1]
        assert np.all(tails < heads)
        assert np.all(DH.val[DH.rowptr[two]] == -1) and np.all(DH.val[DH.rowptr[two] + 1] == 1)
        keys = tails.astype(np.int64) * (1 << 32) + heads
        assert np.all(np.diff(keys) > 0)                                  # sorted, unique
        assert np.all(two == np.arange(len(two)))                         # two-node edges first
        D = h.matrix(l, "D")
        agg = h.ivec(l, "agg")
        single_fine = D.col[D.rowptr[:-1][np.diff(D.rowptr) == 1]]
        singles = DH.col[DH.rowptr[:-1][lens == 1]]
        np.testing.assert_array_equal(singles, np.unique(agg[single_fine]))


def test_structure_preservation(hier12):
    # S_H D_H = 0 (Sec. 2) and D_H^T A_H D_H = P_n^T A_n P_n on every level
    p, S, h = hier12
    Sl = sp.csr_matrix((S.A_val, S.A_col, S.A_rowptr), shape=(S.n_edges, S.n_edges))
    for l in range(h.nlevels - 1):
        Pe, DH = _sp(h.matrix(l, "Pe")), _sp(h.matrix(l, "DH"))
        Sl = (Pe.T @ Sl @ Pe).tocsr()
        assert abs(Sl @ DH).max() <= 1e-12 * abs(Sl).max()
        A1, An, Pn, An1 = (_sp(h.matrix(l + 1, "A")), _sp(h.matrix(l, "An")), _sp(h.matrix(l, "Pn")),
                           _sp(h.matrix(l + 1, "An")))
        A = _sp(h.matrix(l, "A"))
        assert abs(Pe.T @ A @ Pe - A1).max() <= 1e-12 * abs(A1).max()
        assert abs(Pn.T @ An @ Pn - An1).max() <= 1e-12 * abs(An1).max()
        assert abs(DH.T @ A1 @ DH - An1).max() <= 1e-10 * abs(An1).max()


def test_pattern_is_alg2(hier12):
    # N_ij = 1 iff every node of coarse edge j lies in T_i = pattern(|D_h||P_n|)
    _, _, h = hier12
    for l in range(h.nlevels - 1):
        T, Pe, DH = h.matrix(l, "T"), h.matrix(l, "Pe"), h.matrix(l, "DH")
        D, Pn = _sp(h.matrix(l, "D")), _sp(h.matrix(l, "Pn"))
        Ds, Ps = D.copy(), Pn.copy()
        Ds.data[:] = 1.0
        Ps.data[:] = 1.0                       # structural product: no cancellation, no drops
        Tref = (Ds @ Ps).tocsr()
        Tref.sort_indices()
        np.testing.assert_array_equal(T.rowptr, Tref.indptr)
        np.testing.assert_array_equal(T.col, Tref.indices)
        nodes = [set(DH.col[DH.rowptr[j]:DH.rowptr[j + 1]].tolist()) for j in range(DH.shape[0])]
        byn = {}
        for j, s in enumerate(nodes):
            for u in s:
                byn.setdefault(u, []).append(j)
        for i in range(0, T.shape[0], 7):
            Ti = set(T.col[T.rowptr[i]:T.rowptr[i + 1]].tolist())
            ref = sorted({j for u in Ti for j in byn.get(u, []) if nodes[j] <= Ti})
            np.testing.assert_array_equal(Pe.col[Pe.rowptr[i]:Pe.rowptr[i + 1]], ref)


def test_rs_special_case():
    # piecewise-constant P_n, natural BCs: every P_e row is empty or a single +-1 (Sec. 2)
    p = meshgen.generate(meshgen.MeshSpec(6, natural=True))
    for it in (0, 1, 3):
        h = oracle.setup_problem(p, max_levels=2, max_coarse=10, unsmoothed_pn=True, emin_iters=it)
        Pe = h.matrix(0, "Pe")
        lens = np.diff(Pe.rowptr)
        assert set(np.unique(lens)) <= {0, 1}
        np.testing.assert_array_equal(np.abs(Pe.val), 1.0)
        D, agg = h.matrix(0, "D"), h.ivec(0, "agg")
        a = agg[D.col[D.rowptr[:-1]]]
        b = agg[D.col[D.rowptr[:-1] + 1]]
        np.testing.assert_array_equal(lens, (a != b).astype(int))


def _kkt_optimum(h):
    """Dense solve of the constrained minimisation (eqs. (7)-(8)) on level 0."""
    A, D, Pn, DH, Pe = (_sp(h.matrix(0, k)) for k in ("A", "D", "Pn", "DH", "Pe"))
    Pe = Pe.tocoo()
    rows, cols = Pe.row, Pe.col
    nvar = len(rows)
    # objective sum_j P_:j^T A P_:j on the pattern
    Ad = A.toarray()
    H = np.zeros((nvar, nvar))
    bycol = {}
    for k, (i, j) in enumerate(zip(rows, cols)):
        bycol.setdefault(j, []).append((k, i))
    for j, lst in bycol.items():
        ks = [k for k, _ in lst]
        ii = [i for _, i in lst]
        H[np.ix_(ks, ks)] += Ad[np.ix_(ii, ii)]
    # constraints (P D_H)_{iu} = (D_h P_n)_{iu}
    R = (D @ Pn).toarray()
    DHd = DH.toarray()
    cons, rhs = [], []
    nf, nc = R.shape
    for i in range(nf):
        ks = np.nonzero(rows == i)[0]
        for u in range(nc):
            row = np.zeros(nvar)
            row[ks] = DHd[cols[ks], u]
            if row.any() or R[i, u] != 0:
                cons.append(row); rhs.append(R[i, u])
    X = np.array(cons)
    K = np.block([[2 * H, X.T], [X, np.zeros((len(cons), len(cons)))]])
    sol = np.linalg.lstsq(K, np.concatenate([np.zeros(nvar), rhs]), rcond=None)[0]
    x = sol[:nvar]
    return x @ H @ x, x, rows, cols


def test_emin_decreases_energy_towards_kkt_optimum():
    p = meshgen.generate(meshgen.MeshSpec(3, natural=True, jitter=0.2, seed_jitter=2))
    h0 = oracle.setup_problem(p, max_levels=2, max_coarse=10, emin_iters=0)
    E_opt, x_opt, rows, cols = _kkt_optimum(h0)
    E0 = h0.scalars(0)["energy0"]
    h1 = oracle.setup_problem(p, max_levels=2, max_coarse=10, emin_iters=1)
    E1 = h1.scalars(0)["energy1"]
    assert E_opt <= E1 < E0
    hk = oracle.setup_problem(p, max_levels=2, max_coarse=10, emin_iters=3000)
    Ek = hk.scalars(0)["energy1"]
    assert Ek == pytest.approx(E_opt, rel=1e-8)
    Pe = _sp(hk.matrix(0, "Pe")).tocoo()
    np.testing.assert_allclose(np.asarray(_sp(hk.matrix(0, "Pe"))[rows, cols]).ravel(), x_opt,
                               atol=1e-3 * np.abs(x_opt).max())


# ---------------------------------------------------------------- solve
def test_pcg_matches_dense_solve():
    spec = meshgen.MeshSpec(4, jitter=0.2, seed_jitter=1, sigma="lognormal", sigma_in=1.0, seed_sigma=3)
    p = meshgen.generate(spec)
    h = oracle.setup_problem(p, max_coarse=50)
    assert h.nlevels >= 2
    b = meshgen.rhs(7, p.n_edges)
    r = h.solve(b, tol=1e-13, max_iter=500)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr)).toarray()
    x = np.linalg.solve(A, b)
    assert r["status"] == 0
    assert np.linalg.norm(r["x"] - x) <= 1e-9 * np.linalg.norm(x)


def test_vcycle_is_symmetric_and_contracting(hier12):
    p, _, h = hier12
    rng = np.random.default_rng(3)
    r1, r2 = rng.normal(size=p.n_edges), rng.normal(size=p.n_edges)
    a, b = h.vcycle(r1) @ r2, r1 @ h.vcycle(r2)
    assert abs(a - b) <= 1e-12 * abs(a)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    x = rng.uniform(-1, 1, p.n_edges)
    en = lambda v: np.sqrt(v @ (A @ v))
    e0 = en(x)
    for _ in range(10):
        x = x + h.vcycle(-(A @ x))
    assert (en(x) / e0) ** (1 / 10) < 0.9


def test_config1_iterations():
    spec, seed = meshgen.workload("kuhn8")
    p = meshgen.generate(spec)
    h = oracle.setup_problem(p)
    r = h.solve(meshgen.rhs(seed, p.n_edges))
    assert r["status"] == 0 and r["relres"] <= 1e-8 and r["iters"] <= 30


def test_make_irreducible_joins_every_local_graph():
    """make_irreducible (Alg. 2, Sec. 4.2): on an input with reducible local graphs it adds coarse
    edges; afterwards every row's local graph (T_i, two-node edges of N_i) is connected, each
    added edge joins two coarse nodes of one T_i with Z_uv = (P_n^T D_h^T D_h P_n)_uv != 0, and
    the prolongator still satisfies P_e D_H = D_h P_n."""
    import scipy.sparse as sp
    from irr_case import coupled_problem
    p, arp, aci, av = coupled_problem()
    o = oracle.setup(p.n_edges, p.n_nodes, (arp, aci, av), (p.D_rowptr, p.D_col, p.D_val), max_coarse=50)
    assert o.status == 0
    s = o.sizes(0)
    assert s["n_infeasible0"] > 0 and s["n_added"] > 0
    csr = lambda name: (lambda M: sp.csr_matrix((M.val, M.col, M.rowptr), shape=M.shape))(o.matrix(0, name))
    T, DH, Pn, Pe, N = csr("T"), csr("DH"), csr("Pn"), csr("Pe"), csr("Pe")
    D = sp.csr_matrix((p.D_val, p.D_col, p.D_rowptr), shape=(p.n_edges, p.n_nodes))
    # every local graph connected
    pairs = {}
    for j in range(DH.shape[0]):
        c = DH.indices[DH.indptr[j]:DH.indptr[j + 1]]
        if len(c) == 2:
            pairs[j] = (int(c[0]), int(c[1]))
    for i in range(T.shape[0]):
        J = list(T.indices[T.indptr[i]:T.indptr[i + 1]])
        if len(J) <= 1:
            continue
        par = {u: u for u in J}
        def find(u):
            while par[u] != u:
                u = par[u]
            return u
        for j in N.indices[N.indptr[i]:N.indptr[i + 1]]:
            if j in pairs:
                a, b = pairs[j]
                par[find(a)] = find(b)
        assert len({find(u) for u in J}) == 1, i
    # added edges: not in the RS gradient of the aggregates, Z != 0, inside some T_i
    Z = (T.T @ T).tocsr()
    n2 = DH.nnz - DH.shape[0]
    agg = o.ivec(0, "agg")
    Pbar = sp.csr_matrix((np.ones(p.n_nodes), (np.arange(p.n_nodes), agg)), shape=(p.n_nodes, agg.max() + 1))
    rs = (Pbar.T @ D.T @ D @ Pbar).tocsr()
    Tsets = [set(T.indices[T.indptr[i]:T.indptr[i + 1]]) for i in range(T.shape[0])]
    added = [pairs[j] for j in range(n2) if rs[pairs[j][0], pairs[j][1]] == 0]
    assert len(added) == s["n_added"]
    for u, v in added:
        assert Z[u, v] != 0
        assert any(u in t and v in t for t in Tsets)
    # commuting relation
    lhs = (Pe @ DH).toarray()
    rhs = (D @ Pn).toarray()
    assert np.abs(lhs - rhs).max() <= 1e-12 * max(1.0, np.abs(rhs).max())
