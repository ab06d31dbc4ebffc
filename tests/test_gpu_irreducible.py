"""make_irreducible on the GPU (Alg. 2, Sec. 4.2) against the oracle, on an input whose local
coarse graphs are reducible (tests/irr_case.py).  Integer work bit-exact: the coarse gradient
with its added edges, the pattern; FP64 values within 1e-10."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from irr_case import coupled_problem

pytestmark = pytest.mark.gpu


def test_make_irreducible_matches_oracle():
    import torch

    import paper_2506_08284_gb300 as pkg

    p, arp, aci, av = coupled_problem()
    opts = dict(max_coarse=50)
    o = oracle.setup(p.n_edges, p.n_nodes, (arp, aci, av), (p.D_rowptr, p.D_col, p.D_val), **opts)
    assert o.status == 0
    h = pkg.sphc.setup((p.n_edges, p.n_edges, arp, aci, av), (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val),
                       p.coords, p.sigma_edge, pkg.sphc.default_opts(vcycle_fp32=0, **opts))
    assert h.nlevels == o.nlevels
    s0 = o.sizes(0)
    assert s0["n_added"] > 0
    for l in range(o.nlevels - 1):
        assert h.level_info(l)["n_added_edges"] == o.sizes(l)["n_added"], l
        for name in ("DH", "Pe"):
            rp, ci, v, shape = h.export(l, name)
            M = o.matrix(l, name)
            np.testing.assert_array_equal(rp, M.rowptr, err_msg=f"{name} level {l}")
            np.testing.assert_array_equal(ci, M.col, err_msg=f"{name} level {l}")
            if name == "DH":
                np.testing.assert_array_equal(v, M.val)
            else:
                scale = np.abs(M.val).max()
                np.testing.assert_allclose(v, M.val, rtol=0, atol=1e-10 * scale, err_msg=f"{name} level {l}")
    # the hierarchy solves
    b = np.random.default_rng(5).uniform(-1, 1, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x)
    assert rc == 0 and rr[0] <= 1e-8
    r = o.solve(b, tol=1e-8)
    assert abs(int(it[0]) - int(r["iters"])) <= 1
    h.destroy()
