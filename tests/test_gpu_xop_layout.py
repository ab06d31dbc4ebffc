"""Every layout and product kernel of the V-cycle's transfer operators (P_e, P_eᵀ, P_n and A D)
gives the oracle's V-cycle, forced through the test switch SPHC_XOP_LAYOUT (a bit mask read at
setup): 1 CSR for every operator instead of SELL where its slices pad little; 2 the lanes-per-row
product for every CSR operator; 4 the row-block product (a warp's 32 rows streamed in tiles of
staged products, lane k summing row k) for every CSR operator, long rows included, so that rows
spanning several tiles occur.  By default the row-block product serves CSR operators with at most
24 entries per row on average.  FP64 V-cycle against the oracle's in the A-norm to 1e-10; FP32
V-cycle CG solution to 1e-6 of the oracle's."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu

OPTS = dict(max_coarse=200)


@pytest.fixture(scope="module")
def case():
    p = meshgen.generate(meshgen.MeshSpec(14, jitter=0.2, seed_jitter=6, sigma="lognormal", sigma_in=2.0,
                                          seed_sigma=7))
    return p, oracle_setup(p, **OPTS)


@pytest.mark.parametrize("layout", ["0", "1", "3", "5"])
def test_transfer_layouts_match_oracle(case, layout, monkeypatch):
    import torch
    p, o = case
    monkeypatch.setenv("SPHC_XOP_LAYOUT", layout)
    h = gpu_setup(p, vcycle_fp32=0, **OPTS)
    r = meshgen.rhs(17, p.n_edges)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    h.vcycle(rt, zt)
    torch.cuda.synchronize()
    z, zo = zt.cpu().numpy(), o.vcycle(r)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
    e = z - zo
    assert np.sqrt(e @ (A @ e)) <= 1e-10 * np.sqrt(zo @ (A @ zo))
    h.destroy()

    h32 = gpu_setup(p, vcycle_fp32=1, **OPTS)
    b = meshgen.rhs(19, p.n_edges)
    x = np.zeros_like(b)
    rc, it, rr = h32.solve(b, x, tol=1e-8)
    ref = o.solve(b, tol=1e-8)
    assert rc == 0 and rr[0] <= 1.01e-8
    assert np.linalg.norm(x - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    assert it[0] <= ref["iters"] + 3
    h32.destroy()
