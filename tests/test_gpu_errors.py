"""Every failure code sphc_solve and sphc_setup declare, driven through the C ABI by inputs made
on the host; none of them faults or hangs the GPU.

- SPHC_ENOTCONV: an iteration cap below what CG needs.
- SPHC_ESTAGNATION: a tolerance below the FP64 rounding floor.  Sec. 7 states the criterion:
  CG stops when two consecutive iterations give the same solution.  The recursive residual
  keeps shrinking past the floor until alpha p rounds away against every entry of x.
- SPHC_EBREAKDOWN: a non-finite right-hand side, which makes p^T A p non-finite.
- SPHC_ETIMEOUT: the learned warm start's tensor-core completion waits limited to one
  non-blocking check.  The kernel gives up, drains the MMA in flight with its full wait, frees
  its tensor memory and returns.  The next call in the same process must succeed.
"""
import numpy as np
import pytest

import meshgen
import paper_2506_08284_gb300 as pkg
from gpu_util import gpu_setup

pytestmark = pytest.mark.gpu

ENOTCONV, EBREAKDOWN, ETIMEOUT, ESTAGNATION = -4, -5, -7, -8


@pytest.fixture(scope="module")
def kuhn8():
    return meshgen.generate(meshgen.workload("kuhn8")[0])


@pytest.mark.parametrize("graph", [1, 0])
def test_iteration_cap_gives_enotconv(kuhn8, graph):
    h = gpu_setup(kuhn8, vcycle_fp32=0, max_iter=2, cg_graph=graph)
    b = meshgen.rhs(1, kuhn8.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-8)
    assert rc == ENOTCONV and it[0] == 2
    assert 1e-8 < rr[0] < 1.0                      # x is the last iterate, its true residual reported
    assert b"tolerance" in pkg.sphc.load().sphc_last_error()


@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("fp32", [0, 1])
def test_unreachable_tolerance_gives_estagnation(kuhn8, graph, fp32):
    h = gpu_setup(kuhn8, vcycle_fp32=fp32, cg_graph=graph, max_iter=400)
    b = meshgen.rhs(1, kuhn8.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-30)
    assert rc == ESTAGNATION, (rc, it)
    assert it[0] < 400
    assert rr[0] < 1e-12                           # stagnated at the rounding floor, not earlier
    assert b"stagnated" in pkg.sphc.load().sphc_last_error()
    # the same handle solves a reachable tolerance afterwards
    x2 = np.zeros_like(b)
    rc2, _, rr2 = h.solve(b, x2, tol=1e-8)
    assert rc2 == 0 and rr2[0] <= 1.01e-8


def test_nonfinite_rhs_gives_ebreakdown(kuhn8):
    h = gpu_setup(kuhn8, vcycle_fp32=0)
    b = meshgen.rhs(1, kuhn8.n_edges)
    b[17] = np.nan
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-8)
    assert rc == EBREAKDOWN and it[0] == 1 and np.isnan(rr[0])
    assert b"breakdown" in pkg.sphc.load().sphc_last_error()
    b[17] = 0.5
    rc, it, rr = h.solve(b, x, tol=1e-8)
    assert rc == 0


def test_batched_stagnation_is_reported(kuhn8):
    import torch
    p = kuhn8
    o = pkg.sphc.default_opts(vcycle_fp32=0, max_iter=400)
    sys_ = [((p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val), (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val))]
    B = pkg.sphc.setup_batched(sys_, o)
    b = meshgen.rhs(1, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = B.solve([b], [x], tol=1e-30)
    assert rc == ESTAGNATION and it[0, 0] < 400
    B.destroy()
    torch.cuda.synchronize()


def test_tensor_core_wait_limit_gives_etimeout_and_recovers(kuhn8):
    from paper_2506_08284_gb300 import learned
    params = learned.load_weights()
    p = kuhn8
    kw = dict(vcycle_fp32=1, learned=1, learned_emin_iters=1, mlp_params=params)
    A = (p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val)
    D = (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val)
    with pytest.raises(pkg.sphc.SphcError) as e:
        pkg.sphc.setup(A, D, p.coords, p.sigma_edge, pkg.sphc.default_opts(mlp_wait_polls=1, **kw))
    assert e.value.code == ETIMEOUT and "completion wait" in str(e.value)
    # the context is intact: the same setup with the default wait succeeds and solves
    h = pkg.sphc.setup(A, D, p.coords, p.sigma_edge, pkg.sphc.default_opts(**kw))
    b = meshgen.rhs(1, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    assert rc == 0 and rr[0] <= 1.01e-8


def test_setup_reports_device_bytes(kuhn8):
    used0, _ = pkg.sphc.memory_usage(0)
    h = gpu_setup(kuhn8, vcycle_fp32=1)
    st = h.stats()
    used1, _ = pkg.sphc.memory_usage(0)
    nb = st["device_bytes"]
    assert nb > 0
    # temporaries of earlier calls may still be returning to the pool when used0 is read
    assert abs((used1 - used0) - nb) <= 0.01 * nb
    h.destroy()
