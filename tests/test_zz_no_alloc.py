"""sphc_relres_noalloc, the entry point that allocates no device memory.

It exists for callers that cannot allocate: code running inside another allocator's callback,
processes whose device memory a framework has already reserved, or real-time loops that forbid
allocation after start-up.  Through the C ABI it must report the same true relative residual
||b - A x|| / ||b|| as sphc_solve does, within the FP64 tolerance of the other parity tests, on
two calls in a row (its fixed scratch keeps the previous call's contents).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
from gpu_util import gpu_setup

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-10


def test_noalloc_relres_matches_solve():
    import torch

    import paper_2506_08284_gb300 as pkg

    p = meshgen.generate(meshgen.workload("kuhn8")[0])
    h = gpu_setup(p, vcycle_fp32=0, block_rhs=0)
    nrhs = 3
    B = torch.from_numpy(meshgen.rhs(21, p.n_edges, nrhs=nrhs)).cuda()
    X = torch.zeros_like(B)
    rc, it, rr_solve = h.solve(B, X, nrhs=nrhs)
    torch.cuda.synchronize()
    assert rc == 0
    # sphc_solve stops each right-hand side at a different x; also test an arbitrary x
    Y = X.clone()
    Y[1] += 1e-3
    for trial in range(2):                                   # two calls in a row
        out = np.full(nrhs, -1.0)
        torch.cuda.synchronize()
        pool0, torch0 = pkg.sphc.memory_usage(0), torch.cuda.memory_allocated()
        assert h.relres_noalloc(B, X, out, nrhs=nrhs) == 0
        torch.cuda.synchronize()
        # the call allocated nothing: neither the library's pool nor torch's allocator moved
        assert pkg.sphc.memory_usage(0) == pool0
        assert torch.cuda.memory_allocated() == torch0
        # sphc_solve forms A x in its own layout and summation order; b - A x cancels to ~1e-8
        # of b, so the two agree to the rounding of A x relative to b, not to 1e-10 of the result
        np.testing.assert_allclose(out, rr_solve, rtol=FP64_RTOL, atol=1e-14)
        dev_out = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
        assert h.relres_noalloc(B, Y, dev_out, nrhs=nrhs) == 0
        torch.cuda.synchronize()
        A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr))
        Bh, Yh = B.cpu().numpy(), Y.cpu().numpy()
        ref = [np.linalg.norm(Bh[k] - A @ Yh[k]) / np.linalg.norm(Bh[k]) for k in range(nrhs)]
        # the host reference sums in another order; b - A x cancels to ~1e-9 of b, so compare
        # in units of the rounding of A x relative to b
        np.testing.assert_allclose(dev_out.cpu().numpy(), ref, rtol=1e-9, atol=1e-14)
    # arguments the wrapper refuses before the library could read past them
    with pytest.raises(ValueError):
        h.relres_noalloc(B.float(), X, np.zeros(nrhs), nrhs=nrhs)
    with pytest.raises(ValueError):
        h.relres_noalloc(B[:1], X, np.zeros(nrhs), nrhs=nrhs)
    with pytest.raises(ValueError):
        h.relres_noalloc(B, X, np.zeros(nrhs - 1), nrhs=nrhs)
    # more right-hand sides than the fixed scratch holds: a clear error, nothing launched
    Bbig = torch.zeros((65, p.n_edges), dtype=torch.float64, device="cuda")
    rc = h.relres_noalloc(Bbig, Bbig, np.zeros(65), nrhs=65)
    assert rc == -1
    assert b"64" in pkg.sphc.load().sphc_last_error()
