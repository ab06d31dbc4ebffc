"""Block right-hand sides through sphc_solve (opts.block_rhs, the default): up to 16 columns per
block share every operator read, each with its own CG.  Every column is checked against the CPU
oracle's solve of that column alone: FP64 V-cycle to the oracle's iteration count +-1 and x to
1e-9, FP32 V-cycle to x within 1e-6 and at most three iterations more.  Padding columns (nrhs
not a power of two), a zero column, a second block (nrhs = 17), host and device buffers, the
host-loop and graph forms, and the stagnation code per column are covered."""
import numpy as np
import pytest

import meshgen
import paper_2506_08284_gb300 as pkg
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


def _spec(name):
    if name == "kuhn8":
        return meshgen.workload("kuhn8")[0], dict()
    return meshgen.MeshSpec(12, jitter=0.2, seed_jitter=4, sigma="lognormal", sigma_in=2.0, seed_sigma=5), \
        dict(max_coarse=200)


@pytest.fixture(scope="module", params=["kuhn8", "jit12"])
def case(request):
    spec, opts = _spec(request.param)
    p = meshgen.generate(spec)
    o = oracle_setup(p, **opts)
    return request.param, p, o, opts


def _check_columns(o, B, X, it, rr, fp32, skip=()):
    for k in range(B.shape[0]):
        if k in skip:
            continue
        ref = o.solve(B[k], tol=1e-8)
        assert ref["status"] == 0
        err = np.linalg.norm(X[k] - ref["x"]) / np.linalg.norm(ref["x"])
        assert rr[k] <= 1.01e-8, (k, rr[k])
        if fp32:
            assert err <= 1e-6, (k, err)
            assert it[k] <= ref["iters"] + 3, (k, it[k], ref["iters"])
        else:
            assert err <= 1e-9, (k, err)
            assert abs(it[k] - ref["iters"]) <= 1, (k, it[k], ref["iters"])


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("nrhs", [2, 3, 5, 16])
def test_block_columns_match_oracle(case, fp32, nrhs):
    name, p, o, opts = case
    h = gpu_setup(p, vcycle_fp32=fp32, **opts)
    B = meshgen.rhs(60, p.n_edges, nrhs=nrhs)
    X = np.zeros_like(B)
    rc, it, rr = h.solve(B, X, nrhs=nrhs)
    assert rc == 0
    _check_columns(o, B, X, it, rr, fp32)
    h.destroy()


def test_two_blocks_zero_column_and_device_buffers(case):
    import torch
    name, p, o, opts = case
    h = gpu_setup(p, vcycle_fp32=1, **opts)
    nrhs = 17                                   # a block of 16 and a block of 1 (padded to 2)
    B = meshgen.rhs(70, p.n_edges, nrhs=nrhs)
    B[4] = 0.0
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.full_like(Bd, 7.0)
    rc, it, rr = h.solve(Bd, Xd, nrhs=nrhs)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy()
    assert rc == 0
    assert it[4] == 0 and rr[4] == 0.0 and np.all(X[4] == 0.0)
    _check_columns(o, B, X, it, rr, 1, skip=(4,))
    # host-loop form of the same block solve gives the same result
    hl = gpu_setup(p, vcycle_fp32=1, cg_graph=0, **opts)
    X2 = np.zeros_like(B)
    rc2, it2, rr2 = hl.solve(B, X2, nrhs=nrhs)
    assert rc2 == 0 and list(it2) == list(it)
    np.testing.assert_array_equal(X2, X)
    h.destroy()
    hl.destroy()


def test_block_agrees_with_one_at_a_time(case):
    name, p, o, opts = case
    B = meshgen.rhs(80, p.n_edges, nrhs=4)
    res = []
    for blk in (1, 0):
        h = gpu_setup(p, vcycle_fp32=0, block_rhs=blk, **opts)
        X = np.zeros_like(B)
        rc, it, rr = h.solve(B, X, nrhs=4)
        assert rc == 0
        res.append((it, X))
        h.destroy()
    for k in range(4):
        assert abs(res[0][0][k] - res[1][0][k]) <= 1
        assert np.linalg.norm(res[0][1][k] - res[1][1][k]) <= 1e-9 * np.linalg.norm(res[1][1][k])


def test_block_stagnation_per_column(case):
    name, p, o, opts = case
    h = gpu_setup(p, vcycle_fp32=0, max_iter=400, **opts)
    B = meshgen.rhs(90, p.n_edges, nrhs=3)
    X = np.zeros_like(B)
    rc, it, rr = h.solve(B, X, nrhs=3, tol=1e-30)
    assert rc == -8
    assert all(i < 400 for i in it) and all(r < 1e-12 for r in rr)
    assert b"stagnation" in pkg.sphc.load().sphc_last_error()
    h.destroy()
