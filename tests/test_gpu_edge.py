"""Edge cases and error reporting of the GPU library through the C ABI."""
import numpy as np
import pytest

import meshgen
import paper_2506_08284_gb300 as pkg
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


def test_single_level_direct_solve():
    p = meshgen.generate(meshgen.MeshSpec(3, jitter=0.1, seed_jitter=2))
    h = gpu_setup(p, vcycle_fp32=0)                 # 117 edges <= max_coarse: one level
    assert h.nlevels == 1
    b = meshgen.rhs(1, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    assert rc == 0 and it[0] == 1 and rr[0] < 1e-12


def test_two_node_mesh_with_forced_coarsening():
    p = meshgen.generate(meshgen.MeshSpec(4, natural=True))
    h = gpu_setup(p, vcycle_fp32=0, max_coarse=20)
    o = oracle_setup(p, max_coarse=20)
    assert h.nlevels == o.nlevels
    b = meshgen.rhs(2, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    ref = o.solve(b)
    assert rc == 0 and abs(it[0] - ref["iters"]) <= 1


def test_zero_rhs():
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    h = gpu_setup(p)
    b = np.zeros(p.n_edges)
    x = np.ones_like(b)
    rc, it, rr = h.solve(b, x)
    assert rc == 0 and it[0] == 0 and np.all(x == 0)


def test_multiple_rhs():
    # one right-hand side after another (the block solve has its own tests)
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    h = gpu_setup(p, block_rhs=0)
    B = meshgen.rhs(6, p.n_edges, nrhs=3)
    X = np.zeros_like(B)
    rc, it, rr = h.solve(B, X, nrhs=3)
    assert rc == 0 and all(r <= 1.01e-8 for r in rr)
    for k in range(3):
        x1 = np.zeros(p.n_edges)
        h.solve(B[k].copy(), x1)
        np.testing.assert_allclose(X[k], x1, rtol=0, atol=1e-12 * np.abs(x1).max())


def test_invalid_gradient_is_rejected():
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    bad = p.D_val.copy()
    bad[5] = 2.0
    o = pkg.sphc.default_opts()
    with pytest.raises(pkg.sphc.SphcError) as e:
        pkg.sphc.setup((p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val),
                       (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, bad), opts=o)
    assert e.value.code == -1 and "D_h" in str(e.value)


def test_missing_diagonal_is_rejected():
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    ci = p.A_col.copy()
    # replace the diagonal of row 0 by a duplicate-free off-diagonal column outside the row
    r0 = slice(p.A_rowptr[0], p.A_rowptr[1])
    cols = ci[r0]
    spare = max(cols) + 1
    while spare in cols:
        spare += 1
    k = int(np.nonzero(cols == 0)[0][0])
    cols = np.sort(np.concatenate([np.delete(cols, k), [spare]]))
    ci[r0] = cols
    with pytest.raises(pkg.sphc.SphcError) as e:
        pkg.sphc.setup((p.n_edges, p.n_edges, p.A_rowptr, ci, p.A_val),
                       (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val))
    assert e.value.code == -1


def test_device_resident_inputs():
    import torch
    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    dev = lambda a: torch.from_numpy(a).cuda()
    A = (p.n_edges, p.n_edges, dev(p.A_rowptr), dev(p.A_col), dev(p.A_val))
    D = (p.n_edges, p.n_nodes, dev(p.D_rowptr), dev(p.D_col), dev(p.D_val))
    h = pkg.sphc.setup(A, D)
    b = dev(meshgen.rhs(1, p.n_edges))
    x = torch.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    torch.cuda.synchronize()
    h2 = gpu_setup(p)
    x2 = np.zeros(p.n_edges)
    h2.solve(meshgen.rhs(1, p.n_edges), x2)
    assert rc == 0
    np.testing.assert_allclose(x.cpu().numpy(), x2, rtol=0, atol=1e-12 * np.abs(x2).max())


def test_autotuned_widths_give_the_same_solve():
    spec = meshgen.MeshSpec(24, jitter=0.2, seed_jitter=9, sigma="lognormal", sigma_in=2.0, seed_sigma=10)
    p = meshgen.generate(spec)
    b = meshgen.rhs(3, p.n_edges)
    res = []
    for tune in (0, 1):
        h = gpu_setup(p, autotune=tune)
        x = np.zeros_like(b)
        rc, it, rr = h.solve(b, x)
        assert rc == 0 and rr[0] <= 1.01e-8
        res.append((it[0], x))
    assert abs(res[0][0] - res[1][0]) <= 1
    assert np.linalg.norm(res[0][1] - res[1][1]) <= 1e-6 * np.linalg.norm(res[0][1])
