"""The paper's 3D tetrahedral model problems (Sec. 6.1, Table of 3D constant-sigma problems):
natural boundary conditions, unjittered Kuhn meshes with 10^3 and 28^3 nodes, constant sigma in
{1e2, 1e1, 1, 1e-1, 1e-2}, one V-cycle of PCG, x0 = 0, random right-hand side, tolerance 1e-8
capped at kappa(D^-1 A) / 1e16 (the paper's rounding rule).

- The 1-norm condition estimate (Hager's method on the GPU) against the exact kappa_1 of D^-1 A
  on a small mesh (dense inverse).
- Per sigma, the GPU (FP64 V-cycle) against the CPU oracle at the same tolerance: iterations +-1.
- The counts are printed beside the paper's; they are context, not a bound: the aggregation and
  the piecewise-constant prolongator differ from the paper's (readings 5 and 9).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
from gpu_util import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu

SIGMAS = [1e2, 1e1, 1.0, 1e-1, 1e-2]
PAPER = {9: [4, 9, 11, 12, 12], 27: [5, 12, 12, 13, 13], 81: [9, 12, 13, 13, 11]}


def test_condition_estimate_against_exact():
    p = meshgen.generate(meshgen.MeshSpec(4, natural=True, sigma="const", sigma_in=1e-2))
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr)).toarray()
    B = A / np.diag(A)[:, None]
    exact = np.linalg.norm(B, 1) * np.linalg.norm(np.linalg.inv(B), 1)
    h = gpu_setup(p, vcycle_fp32=0, max_coarse=50)
    kappa, nb, ni = h.cond_estimate(5)
    assert nb == pytest.approx(np.linalg.norm(B, 1), rel=1e-12)
    assert kappa <= exact * (1 + 1e-6)            # Hager's estimate is a lower bound
    assert kappa >= 0.3 * exact
    print(f"\nkappa_1(D^-1 A), 4^3 cells, sigma 1e-2: estimate {kappa:.4e}, exact {exact:.4e}")


@pytest.mark.parametrize("n", [9, 27])
def test_paper_tet_table_against_oracle(n):
    its_gpu, its_orc, tols = [], [], []
    for sigma in SIGMAS:
        p = meshgen.generate(meshgen.MeshSpec(n, natural=True, sigma="const", sigma_in=sigma))
        b = meshgen.rhs(1, p.n_edges)
        h = gpu_setup(p, vcycle_fp32=0)
        kappa, _, _ = h.cond_estimate(5)
        tol = max(1e-8, kappa / 1e16)
        x = np.zeros_like(b)
        rc, it, rr = h.solve(b, x, tol=tol)
        assert rc == 0 and rr[0] <= 1.01 * tol
        ref = oracle_setup(p).solve(b, tol=tol)
        assert ref["status"] == 0
        assert abs(it[0] - ref["iters"]) <= 1, (sigma, it[0], ref["iters"])
        its_gpu.append(it[0])
        its_orc.append(ref["iters"])
        tols.append(tol)
        h.destroy()
    print(f"\n{n + 1}^3 nodes, sigma {SIGMAS}: GPU {its_gpu}, oracle {its_orc}, paper {PAPER[n]}, "
          f"tolerances {['%.2e' % t for t in tols]}")
