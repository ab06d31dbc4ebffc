"""Batched uneven systems through the C ABI: every system's whole CG as one branch of a single
CUDA graph; results match the single-system solves and, system by system, the CPU oracle
(FP64: iterations +-1 and x to 1e-9; FP32 V-cycle: x to 1e-6 of the FP64 oracle)."""
import numpy as np
import pytest

import meshgen
import paper_2506_08284_gb300 as pkg
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


def _systems():
    out = []
    for k, n in enumerate([6, 11, 8, 14, 9]):
        spec = meshgen.MeshSpec(n, jitter=0.2, seed_jitter=500 + k, sigma="lognormal", sigma_in=2.0, seed_sigma=600 + k)
        out.append(meshgen.generate(spec))
    return out


@pytest.mark.parametrize("fp32", [0, 1])
def test_batched_matches_single(fp32):
    probs = _systems()
    systems = [((p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val), (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col,
                p.D_val), p.coords, p.sigma_edge) for p in probs]
    opts = pkg.sphc.default_opts(vcycle_fp32=fp32, max_coarse=200)
    batch = pkg.sphc.setup_batched(systems, opts)
    nrhs = 2
    bs = [meshgen.rhs(40 + k, p.n_edges, nrhs=nrhs) for k, p in enumerate(probs)]
    xs = [np.zeros_like(b) for b in bs]
    rc, it, rr = batch.solve(bs, xs, nrhs=nrhs)
    assert rc == 0
    assert np.all(rr <= 1.01e-8)
    for k, p in enumerate(probs):
        h = gpu_setup(p, vcycle_fp32=fp32, max_coarse=200)
        o = oracle_setup(p, max_coarse=200)
        for r in range(nrhs):
            x1 = np.zeros(p.n_edges)
            rc1, it1, rr1 = h.solve(bs[k][r].copy(), x1)
            assert abs(it1[0] - it[k, r]) <= 1
            assert np.linalg.norm(xs[k][r] - x1) <= 1e-7 * np.linalg.norm(x1)
            ref = o.solve(bs[k][r], tol=1e-8)
            assert ref["status"] == 0
            err = np.linalg.norm(xs[k][r] - ref["x"]) / np.linalg.norm(ref["x"])
            if fp32:
                assert err <= 1e-6, (k, r, err)
                assert it[k, r] <= ref["iters"] + 3
            else:
                assert err <= 1e-9, (k, r, err)
                assert abs(int(it[k, r]) - ref["iters"]) <= 1
        h.destroy()
    # a second solve on the same graph reuses it
    xs2 = [np.zeros_like(b) for b in bs]
    rc2, it2, rr2 = batch.solve(bs, xs2, nrhs=nrhs)
    assert rc2 == 0 and np.array_equal(it2, it)
    for k in range(len(probs)):
        np.testing.assert_array_equal(xs2[k], xs[k])
    batch.destroy()
