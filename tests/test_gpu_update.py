"""sphc_setup_update (setup reuse for related systems, Sec. 3 warm-start remark) on the GPU
against the oracle's update of the same hierarchy: structure kept bit for bit, prolongators and
coarse operators to 1e-10, CG iterations +-1, and a sequence of updates."""
import numpy as np
import pytest

import meshgen
from gpu_util import assert_csr_close, gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


def _spec(seed_sigma, n=12):
    return meshgen.MeshSpec(n, jitter=0.2, seed_jitter=3, sigma="lognormal", sigma_in=1.0, seed_sigma=seed_sigma)


@pytest.mark.parametrize("fp32", [0, 1])
def test_update_matches_oracle(fp32):
    p, q = meshgen.generate(_spec(4)), meshgen.generate(_spec(5))
    h = gpu_setup(p, vcycle_fp32=fp32, max_coarse=200)
    o = oracle_setup(p, max_coarse=200)
    agg0 = [h.export(l, "agg") for l in range(h.nlevels - 1)]
    h.update(q.A_val)
    ou = o.update(q.A_val, max_coarse=200)
    assert h.nlevels == ou.nlevels
    for l in range(ou.nlevels):
        assert_csr_close(h.export(l, "A"), ou.matrix(l, "A"), f"L{l} A", 1e-10)
        if l == ou.nlevels - 1:
            continue
        np.testing.assert_array_equal(h.export(l, "agg"), agg0[l])
        np.testing.assert_array_equal(h.export(l, "agg"), ou.ivec(l, "agg"))
        assert_csr_close(h.export(l, "DH"), ou.matrix(l, "DH"), f"L{l} D_H", 0.0)
        for what in ("Pn", "P0", "Pe"):
            assert_csr_close(h.export(l, what), ou.matrix(l, what), f"L{l} {what}", 1e-10)
    b = meshgen.rhs(7, q.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    ref = ou.solve(b)
    assert rc == 0 and rr[0] <= 1.01e-8
    assert abs(it[0] - ref["iters"]) <= (3 if fp32 else 1)
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= (1e-6 if fp32 else 1e-9)


def test_sequence_of_updates_and_block_solve():
    h = gpu_setup(meshgen.generate(_spec(4)), vcycle_fp32=1, max_coarse=200)
    for k in range(3):
        q = meshgen.generate(_spec(10 + k))
        h.update(q.A_val)
        B = meshgen.rhs(20 + k, q.n_edges, nrhs=3)
        X = np.zeros_like(B)
        rc, it, rr = h.solve(B, X, nrhs=3)
        assert rc == 0 and max(rr) <= 1.01e-8
        fresh = gpu_setup(q, vcycle_fp32=1, max_coarse=200)
        X1 = np.zeros_like(B)
        rc1, it1, _ = fresh.solve(B, X1, nrhs=3)
        assert max(it) <= max(it1) + 2
        fresh.destroy()
