"""The persistent grid sweep of the smoothers (sphc_opts.sweep_form 3): one cooperative launch per
forward + backward multicolour sweep, a grid barrier between colours instead of a kernel boundary.

- PCG with the CG graph (the cooperative launches captured into the body of its device-side loop)
  and with the host loop, FP64 and FP32 V-cycles, against the oracle's solve: FP64 to the
  oracle's iteration count +-1 and x to 1e-9, FP32 to x within 1e-6.  The grid sweeps must still
  be in place after the solve (the graph capture did not fall back to per-colour launches).
- The FP32 V-cycle with grid sweeps against the same V-cycle with a launch per colour.
- The barrier's bounded waits: a barrier that counts one arrival more than the grid has thread
  blocks cannot complete; every wait gives up after its polls, the call reports it, and the
  device keeps working (a barrier with the right count completes, a solve after it converges).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import paper_2506_08284_gb300 as pkg
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu

OPTS = dict(max_coarse=200)


@pytest.fixture(scope="module")
def case():
    p = meshgen.generate(meshgen.MeshSpec(16, jitter=0.2, seed_jitter=4, sigma="lognormal", sigma_in=2.0,
                                          seed_sigma=5))
    return p, oracle_setup(p, **OPTS)


def _edge_kinds(h):
    return [h.level_info(l)["sweep_kind_edge"] for l in range(h.stats()["n_levels"] - 1)]


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("graph", [1, 0])
def test_grid_sweep_pcg_matches_oracle(case, fp32, graph):
    p, o = case
    h = gpu_setup(p, vcycle_fp32=fp32, sweep_form=3, cg_graph=graph, **OPTS)
    kinds = _edge_kinds(h)
    assert kinds[0] == 3
    b = meshgen.rhs(5, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-8)
    assert rc == 0 and rr[0] <= 1.01e-8
    ref = o.solve(b, tol=1e-8)
    assert ref["status"] == 0
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    if fp32:
        assert err <= 1e-6 and it[0] <= ref["iters"] + 3, (err, it[0], ref["iters"])
    else:
        assert err <= 1e-9 and abs(it[0] - ref["iters"]) <= 1, (err, it[0], ref["iters"])
    assert _edge_kinds(h) == kinds
    # a second solve on the same handle (the barrier state carries over between launches)
    x2 = np.zeros_like(b)
    rc2, it2, _ = h.solve(b, x2, tol=1e-8)
    assert rc2 == 0 and it2[0] == it[0]
    np.testing.assert_array_equal(x2, x)
    h.destroy()


def test_grid_sweep_matches_per_colour_launches(case):
    import torch
    p, _ = case
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    r = meshgen.rhs(12, p.n_edges)
    zs = []
    for form in (3, 1):
        h = gpu_setup(p, vcycle_fp32=1, sweep_form=form, **OPTS)
        assert (_edge_kinds(h)[0] == 3) == (form == 3)
        rt = torch.tensor(r, device="cuda")
        zt = torch.empty_like(rt)
        h.vcycle(rt, zt)
        torch.cuda.synchronize()
        zs.append(zt.cpu().numpy())
        h.destroy()
    e = zs[0] - zs[1]
    assert np.sqrt(e @ (A @ e)) <= 1e-5 * np.sqrt(zs[1] @ (A @ zs[1]))


def test_grid_barrier_wait_gives_up(case):
    assert pkg.sphc.grid_barrier_check(0) is False
    assert pkg.sphc.grid_barrier_check(1, polls=20000) is True
    assert pkg.sphc.grid_barrier_check(3, polls=1) is True
    assert pkg.sphc.grid_barrier_check(0) is False            # the device keeps working
    p, o = case
    h = gpu_setup(p, vcycle_fp32=1, sweep_form=3, **OPTS)
    b = meshgen.rhs(6, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-8)
    assert rc == 0 and rr[0] <= 1.01e-8
    h.destroy()
