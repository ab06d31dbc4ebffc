"""Pins of oracle parts that the invariants of test_oracle.py leave loose, each against a
computation written here independently of the oracle's C code.

- rho(D^-1 A_n) (Sec. 3, the omega of the prolongator smoothing read as 4 / (3 rho)): the
  oracle's 15 power-iteration steps equal a numpy restatement from the same splitmix64 start
  vector, and lie below, and close to, the largest eigenvalue of the pencil (A_n, D) from LAPACK.
- The symmetric Hiptmair sweep inside the V-cycle (Sec. 6.1): the oracle's V-cycle equals a
  sparse restatement of the sweep's steps (SGS on A; r = b - A x; nodal SGS on A_n c = D^T r
  from c = 0; x += D c; SGS on A) around the Galerkin coarse correction.  The restatements
  that drop the nodal correction or take D^T r before the first SGS differ from it, and at
  small sigma only the nodal correction removes the gradient-space residual.
- Reading R14' of the initial guess (Sec. 6.1): with 3-node block aggregates on natural-BC
  Kuhn meshes and sigma = 1, the least-norm P0 gives nearly mesh-independent CG counts (the
  paper's 3D tet table has 11 and 12 at 10^3 and 28^3 nodes), while the literal reading (the
  all-ones row projected onto the constraints) grows with the mesh.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import meshgen
import oracle
from prio import splitmix64
from test_oracle import _blocks


# ---------------------------------------------------------------- rho(D^-1 A_n)
def _power_rho(An, seed, iters):
    """Power iteration on D^-1 A_n from v_i = uniform01(splitmix64(seed, i)); the estimate is
    ||w|| / ||v|| of the last step."""
    n = An.shape[0]
    d = An.diagonal()
    v = np.array([(splitmix64(seed, i) >> 11) * 2.0**-53 for i in range(n)])
    est = 1.0
    for _ in range(iters):
        w = (An @ v) / d
        est = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return est


@pytest.mark.parametrize("spec", [meshgen.MeshSpec(6),
                                  meshgen.MeshSpec(6, jitter=0.2, seed_jitter=3, sigma="lognormal", sigma_in=2.0,
                                                   seed_sigma=4)], ids=["kuhn6", "jit6"])
def test_power_rho_restated(spec):
    p = meshgen.generate(spec)
    h = oracle.setup_problem(p, max_coarse=50)
    An = h.matrix(0, "An").to_scipy()
    rho = h.scalars(0)["rho"]
    seed = 0 + 1000 * 0 + 4                       # level-0 seed of the smoothing estimate
    assert rho == pytest.approx(_power_rho(An, seed, 15), rel=1e-12)
    # the step count matters at this size: 14 or 16 steps would fail the line above
    assert abs(_power_rho(An, seed, 14) - rho) > 1e-4 * rho
    assert abs(_power_rho(An, seed, 16) - rho) > 1e-4 * rho
    lam = sla.eigh(An.toarray(), np.diag(An.diagonal()), eigvals_only=True).max()
    assert rho <= lam * (1 + 1e-12)
    assert rho >= 0.9 * lam
    assert h.scalars(0)["omega_sa"] == pytest.approx(4.0 / (3.0 * rho), rel=1e-15)


# ---------------------------------------------------------------- Hiptmair composition
def _sgs(A, col, b, x):
    """Multicolour symmetric Gauss-Seidel: colours 0..C-1, then C-1..0; the rows of one colour
    do not couple, so each colour is one simultaneous update."""
    d = A.diagonal()
    off = (A - sp.diags(d)).tocsr()
    ncol = int(col.max()) + 1
    for c in list(range(ncol)) + list(range(ncol - 1, -1, -1)):
        rows = np.nonzero(col == c)[0]
        x[rows] = (b[rows] - off[rows] @ x) / d[rows]
    return x


def _hiptmair(L, b, x, variant="paper"):
    A, D, An, ce, cn = L
    if variant == "pre_residual":                 # wrong order: D^T r before the first SGS
        g = D.T @ (b - A @ x)
        _sgs(A, ce, b, x)
    else:
        _sgs(A, ce, b, x)
        g = D.T @ (b - A @ x)
    if variant != "no_nodal":
        x += D @ _sgs(An, cn, g, np.zeros(An.shape[0]))
    _sgs(A, ce, b, x)
    return x


def _vcycle(levels, Pe, l, b, variant="paper"):
    if l == len(levels) - 1:
        return np.linalg.solve(levels[l][0].toarray(), b)
    A = levels[l][0]
    x = _hiptmair(levels[l], b, np.zeros_like(b), variant)
    x += Pe[l] @ _vcycle(levels, Pe, l + 1, Pe[l].T @ (b - A @ x), variant)
    return _hiptmair(levels[l], b, x, variant)


def _levels(h):
    L, Pe = [], []
    for l in range(h.nlevels):
        L.append((h.matrix(l, "A").to_scipy(), h.matrix(l, "D").to_scipy(), h.matrix(l, "An").to_scipy(),
                  h.ivec(l, "col_e"), h.ivec(l, "col_n")))
        if l < h.nlevels - 1:
            Pe.append(h.matrix(l, "Pe").to_scipy())
    return L, Pe


def test_vcycle_is_the_restated_hiptmair_composition():
    p = meshgen.generate(meshgen.MeshSpec(4, jitter=0.2, seed_jitter=3))
    h = oracle.setup_problem(p, max_coarse=20)
    assert h.nlevels >= 2
    L, Pe = _levels(h)
    r = meshgen.rhs(5, p.n_edges)
    z = h.vcycle(r)
    zt = _vcycle(L, Pe, 0, r)
    assert np.abs(z - zt).max() <= 1e-13 * np.abs(z).max()
    for wrong in ("no_nodal", "pre_residual"):
        zw = _vcycle(L, Pe, 0, r, wrong)
        assert np.abs(z - zw).max() > 1e-3 * np.abs(z).max(), wrong


def test_nodal_correction_removes_the_gradient_residual():
    # sigma = 1e-4: A is nearly singular on gradients, which SGS on A cannot reduce
    p = meshgen.generate(meshgen.MeshSpec(4, jitter=0.2, seed_jitter=3, sigma_in=1e-4))
    h = oracle.setup_problem(p, max_coarse=20)
    L, Pe = _levels(h)
    A, D = L[0][0], L[0][1]
    b = meshgen.rhs(5, p.n_edges)
    g0 = np.linalg.norm(D.T @ b)
    full = np.linalg.norm(D.T @ (b - A @ _hiptmair(L[0], b, np.zeros_like(b)))) / g0
    sgs_only = np.linalg.norm(D.T @ (b - A @ _hiptmair(L[0], b, np.zeros_like(b), "no_nodal"))) / g0
    assert full < 0.25 and sgs_only > 0.99
    # the oracle's V-cycle is the composition with the correction (at the conditioning 1/sigma
    # of this case, rounding differences are amplified to about 1e-10)
    r = meshgen.rhs(7, p.n_edges)
    z, zt = h.vcycle(r), _vcycle(L, Pe, 0, r)
    assert np.abs(z - zt).max() <= 1e-9 * np.abs(z).max()
    assert np.abs(z - _vcycle(L, Pe, 0, r, "no_nodal")).max() > 1e-2 * np.abs(z).max()


# ---------------------------------------------------------------- reading R14' of P0
@pytest.mark.slow
def test_least_norm_initial_guess_gives_mesh_independent_counts():
    its = {}
    for n in (9, 27):
        p = meshgen.generate(meshgen.MeshSpec(n, natural=True))
        agg, _ = _blocks(n)
        b = meshgen.rhs(1, p.n_edges)
        for name, p0 in (("least_norm", 0.0), ("literal", 1.0)):
            h = oracle.setup_problem(p, agg0=agg, p0_value=p0)
            r = h.solve(b, max_iter=300)
            assert r["status"] == 0
            its[name, n] = r["iters"]
    # least-norm: close to the paper's 11 / 12 and nearly flat from 10^3 to 28^3 nodes
    assert 9 <= its["least_norm", 9] <= 14 and 9 <= its["least_norm", 27] <= 16
    assert its["least_norm", 27] - its["least_norm", 9] <= 3
    # literal: already worse on the small mesh and more than doubling on the larger one
    assert its["literal", 9] > its["least_norm", 9]
    assert its["literal", 27] >= 2 * its["literal", 9]


# ---------------------------------------------------------------- projected CG energy minimisation
def test_projected_cg_energy_minimisation():
    """Projected CG on eq. (8) (Sec. 3): its first step is an exact line search along the
    direction of the projected Jacobi step of eq. (9), so no damping of eq. (9) gives lower
    energy; the energy falls with every step; enough steps reach the KKT optimum (dense solve);
    the commuting relation holds throughout."""
    from test_oracle import _kkt_optimum
    p = meshgen.generate(meshgen.MeshSpec(3, natural=True, jitter=0.2, seed_jitter=2))
    kw = dict(max_levels=2, max_coarse=10)
    h0 = oracle.setup_problem(p, emin_iters=0, **kw)
    E_opt, _, _, _ = _kkt_optimum(h0)
    E0 = h0.scalars(0)["energy0"]
    cg = [oracle.setup_problem(p, emin_iters=k, emin_method=1, **kw).scalars(0)["energy1"] for k in range(1, 7)]
    for omega in (0.25, 0.5, 1.0):
        Ej = oracle.setup_problem(p, emin_iters=1, emin_omega=omega, **kw).scalars(0)["energy1"]
        assert cg[0] <= Ej * (1 + 1e-12), omega
    assert E0 > cg[0] and all(b <= a * (1 + 1e-12) for a, b in zip(cg, cg[1:]))
    hk = oracle.setup_problem(p, emin_iters=400, emin_method=1, **kw)
    assert hk.scalars(0)["energy1"] == pytest.approx(E_opt, rel=1e-9)
    # the steps the paper uses (1-4) keep the relation to rounding; over hundreds of steps the
    # rounding of the feasible updates accumulates slowly
    for h, bound in ((oracle.setup_problem(p, emin_iters=4, emin_method=1, **kw), 1e-12), (hk, 1e-8)):
        Pe, DH = h.matrix(0, "Pe").to_scipy(), h.matrix(0, "DH").to_scipy()
        D, Pn = h.matrix(0, "D").to_scipy(), h.matrix(0, "Pn").to_scipy()
        rhs = D @ Pn
        assert abs(Pe @ DH - rhs).max() <= bound * max(1.0, abs(rhs).max())


# ---------------------------------------------------------------- setup reuse (Sec. 3 warm start)
def _related(seed_sigma):
    return meshgen.MeshSpec(8, jitter=0.2, seed_jitter=3, sigma="lognormal", sigma_in=1.0, seed_sigma=seed_sigma)


def test_update_with_unchanged_values_continues_the_iteration():
    """Updating a hierarchy with the values it was built from keeps P_e feasible, so the
    projection of the warm start is the identity (to rounding) and one more step of eq. (9)
    follows: the result equals a fresh setup with twice the steps."""
    p = meshgen.generate(_related(4))
    h1 = oracle.setup_problem(p, max_coarse=100, emin_iters=1)
    hu = h1.update(p.A_val, max_coarse=100, emin_iters=1)
    h2 = oracle.setup_problem(p, max_coarse=100, emin_iters=2)
    assert hu.status == 0 and hu.nlevels == h2.nlevels
    for l in range(h2.nlevels - 1):
        a, b = hu.matrix(l, "Pe"), h2.matrix(l, "Pe")
        np.testing.assert_array_equal(a.col, b.col)
        assert np.abs(a.val - b.val).max() <= 1e-12 * np.abs(b.val).max()


def test_update_to_a_related_system():
    """New conductivities on the same mesh: the structure is kept, the commuting relation holds
    on every level, and the updated hierarchy solves the new system."""
    p, q = meshgen.generate(_related(4)), meshgen.generate(_related(5))
    np.testing.assert_array_equal(p.A_col, q.A_col)
    h = oracle.setup_problem(p, max_coarse=100)
    hu = h.update(q.A_val, max_coarse=100)
    assert hu.status == 0 and hu.nlevels == h.nlevels
    for l in range(hu.nlevels - 1):
        np.testing.assert_array_equal(hu.ivec(l, "agg"), h.ivec(l, "agg"))
        np.testing.assert_array_equal(hu.matrix(l, "DH").col, h.matrix(l, "DH").col)
        Pe, DH = hu.matrix(l, "Pe").to_scipy(), hu.matrix(l, "DH").to_scipy()
        D, Pn = hu.matrix(l, "D").to_scipy(), hu.matrix(l, "Pn").to_scipy()
        rhs = D @ Pn
        assert abs(Pe @ DH - rhs).max() <= 1e-12 * max(1.0, abs(rhs).max())
    b = meshgen.rhs(3, q.n_edges)
    r = hu.solve(b)
    fresh = oracle.setup_problem(q, max_coarse=100).solve(b)
    assert r["status"] == 0 and r["iters"] <= fresh["iters"] + 2


# ---------------------------------------------------------------- f1: drop tolerance and Alg. 1
def test_tiny_drop_tolerance_changes_nothing():
    # jittered, so no structural entry is exactly zero: theta = 1e-300 drops nothing and the
    # lumping adds nothing, which must reproduce the theta = 0 hierarchy bit for bit
    p = meshgen.generate(meshgen.MeshSpec(8, jitter=0.2, seed_jitter=9, sigma="lognormal", sigma_in=1.0, seed_sigma=2))
    h0 = oracle.setup_problem(p, max_coarse=100)
    h1 = oracle.setup_problem(p, max_coarse=100, sa_theta=1e-300)
    for l in range(h0.nlevels - 1):
        np.testing.assert_array_equal(h0.ivec(l, "agg"), h1.ivec(l, "agg"))
        np.testing.assert_array_equal(h0.matrix(l, "Pe").val, h1.matrix(l, "Pe").val)


def _strong_graph(An, theta):
    d = An.diagonal()
    C = An.tocoo()
    keep = (C.row != C.col) & (np.abs(C.data) >= theta * np.sqrt(d[C.row] * d[C.col]))
    return sp.csr_matrix((np.ones(keep.sum()), (C.row[keep], C.col[keep])), shape=An.shape)


def test_drop_tolerance_aggregates_respect_the_strong_graph():
    """theta = 0.1 on the box conductivity (1 inside, 1e-3 outside): every aggregate is connected
    in the strong graph (restated here from A_n with the symmetric SA criterion), P_n rows sum to
    one, and fewer aggregates straddle the material interface than with theta = 0."""
    import scipy.sparse.csgraph as csg
    p = meshgen.generate(meshgen.MeshSpec(12, jitter=0.15, seed_jitter=8, sigma="box", sigma_in=1.0, sigma_out=1e-3))
    hs = {th: oracle.setup_problem(p, max_coarse=200, sa_theta=th) for th in (0.0, 0.1)}
    h = hs[0.1]
    An = h.matrix(0, "An").to_scipy()
    S = _strong_graph(An, 0.1)
    agg = h.ivec(0, "agg")
    for a in range(agg.max() + 1):
        nodes = np.nonzero(agg == a)[0]
        ncomp, _ = csg.connected_components(S[nodes][:, nodes], directed=False)
        assert ncomp == 1, a
    Pn = h.matrix(0, "Pn").to_scipy()
    np.testing.assert_allclose(np.asarray(Pn.sum(axis=1)).ravel(), 1.0, atol=1e-12)
    X = p.coords
    inside = np.all((X > 0.25 + 1 / 24) & (X < 0.75 - 1 / 24), axis=1)
    outside = np.any((X < 0.25 - 1 / 24) | (X > 0.75 + 1 / 24), axis=1)
    def straddling(hh):
        g = hh.ivec(0, "agg")
        return sum(1 for a in range(g.max() + 1) if inside[g == a].any() and outside[g == a].any())
    assert straddling(hs[0.1]) < straddling(hs[0.0])


def _alg1_restated(P, passes):
    """The oracle's reading of Alg. 1, restated with numpy on a scipy CSR matrix."""
    m, nc = P.shape
    nnz = P.nnz
    Pt = P.T.tocsr()
    assign = -np.ones(m, int)
    cnt = np.diff(Pt.indptr)
    nass = -(-(-(-(cnt * m) // nnz)) // passes)
    for _ in range(passes):
        best, bcol = -np.ones(m), -np.ones(m, int)
        props = []
        for j in range(nc):
            rows, vals = Pt.indices[Pt.indptr[j]:Pt.indptr[j + 1]], np.abs(Pt.data[Pt.indptr[j]:Pt.indptr[j + 1]])
            cand = sorted((-a, r) for r, a in zip(rows, vals) if assign[r] < 0)[:nass[j]]
            props += [(j, r, -na) for na, r in cand]
        for j, r, a in props:
            if a > best[r] or (a == best[r] and (bcol[r] < 0 or j < bcol[r])):
                best[r], bcol[r] = a, j
        assign[bcol >= 0] = bcol[bcol >= 0]
    for r in np.nonzero(assign < 0)[0]:
        cols, vals = P.indices[P.indptr[r]:P.indptr[r + 1]], np.abs(P.data[P.indptr[r]:P.indptr[r + 1]])
        assign[r] = min(zip(-vals, cols))[1]
    count = np.bincount(assign, minlength=nc)
    for j in range(nc):
        rows, vals = Pt.indices[Pt.indptr[j]:Pt.indptr[j + 1]], np.abs(Pt.data[Pt.indptr[j]:Pt.indptr[j + 1]])
        if count[j] > 0 or rows.size == 0:
            continue
        r = min(zip(-vals, rows))[1]
        if count[assign[r]] >= 2:
            count[assign[r]] -= 1
            assign[r] = j
            count[j] += 1
    return assign


def test_alg1_reading_restated_and_special_case():
    p = meshgen.generate(meshgen.MeshSpec(6, jitter=0.2, seed_jitter=2))
    h = oracle.setup_problem(p, max_coarse=50)
    Pn = h.matrix(0, "Pn")
    for passes in (1, 2, 3):
        got = oracle.gen_piecewise_const(Pn, passes)
        np.testing.assert_array_equal(got, _alg1_restated(Pn.to_scipy(), passes))
        S = Pn.to_scipy()
        assert all(S[r, got[r]] != 0 for r in range(S.shape[0]))      # a column of the row
    # Alg. 1 of a piecewise-constant P returns it: every column keeps all its rows
    agg = h.ivec(0, "agg")
    Pbar = oracle.CSR(np.arange(agg.size + 1, dtype=np.int64), agg.astype(np.int32), np.ones(agg.size), Pn.shape)
    np.testing.assert_array_equal(oracle.gen_piecewise_const(Pbar, 2), agg)
    # with Alg. 1 the hierarchy still satisfies the commuting relation and solves
    ha = oracle.setup_problem(p, max_coarse=50, pn_alg1=1)
    assert ha.status == 0
    Pe, DH = ha.matrix(0, "Pe").to_scipy(), ha.matrix(0, "DH").to_scipy()
    rhs = ha.matrix(0, "D").to_scipy() @ ha.matrix(0, "Pn").to_scipy()
    assert abs(Pe @ DH - rhs).max() <= 1e-12 * max(1.0, abs(rhs).max())
    assert ha.solve(meshgen.rhs(2, p.n_edges))["status"] == 0
