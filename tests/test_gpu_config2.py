"""The 48^3 box-conductivity workload (753,552 unknowns, jitter +-0.2h, sigma 1 inside
[0.25, 0.75]^3 and 1e-3 outside, RHS seed 3) on the GPU against the CPU oracle, element by
element: every integer array of the hierarchy bit for bit, every FP64 setup value to 1e-10 of
the largest entry, the FP64 solve to the oracle's iteration count +-1 and x to 1e-9, and the
FP32 V-cycle solve to x within 1e-6 of the FP64 oracle.  The measured errors are printed.
"""
import numpy as np
import pytest

import meshgen
from gpu_util import assert_csr_close, assert_csr_equal_pattern, gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kuhn48():
    spec, seed = meshgen.workload("kuhn48")
    p = meshgen.generate(spec)
    b = meshgen.rhs(seed, p.n_edges)
    o = oracle_setup(p)
    ref = o.solve(b, tol=1e-8)
    assert ref["status"] == 0
    return p, b, o, ref


def test_config2_fp64_hierarchy_matches_oracle(kuhn48):
    p, b, o, ref = kuhn48
    h = gpu_setup(p, vcycle_fp32=0)
    assert h.nlevels == o.nlevels
    for l in range(o.nlevels):
        np.testing.assert_array_equal(h.export(l, "col_e"), o.ivec(l, "col_e"))
        np.testing.assert_array_equal(h.export(l, "col_n"), o.ivec(l, "col_n"))
        assert_csr_close(h.export(l, "A"), o.matrix(l, "A"), f"L{l} A", 1e-10)
        if not o.sizes(l)["has_transfer"]:
            continue
        np.testing.assert_array_equal(h.export(l, "agg"), o.ivec(l, "agg"))
        assert_csr_close(h.export(l, "DH"), o.matrix(l, "DH"), f"L{l} D_H", 0.0)
        assert_csr_equal_pattern(h.export(l, "T"), o.matrix(l, "T"), f"L{l} T")
        for what in ("Pn", "P0", "Pe"):
            assert_csr_close(h.export(l, what), o.matrix(l, what), f"L{l} {what}", 1e-10)
    h.destroy()


@pytest.mark.parametrize("fp32", [0, 1])
def test_config2_solve_matches_oracle(kuhn48, fp32):
    p, b, o, ref = kuhn48
    h = gpu_setup(p, vcycle_fp32=fp32)
    x = np.zeros_like(b)
    rc, it, rr = h.solve(b, x, tol=1e-8)
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    print(f"\nconfig2 kuhn48 {'FP32' if fp32 else 'FP64'} V-cycle: {it[0]} CG iterations (oracle {ref['iters']}), "
          f"relres {rr[0]:.3e}, ||x - x_oracle|| / ||x_oracle|| = {err:.3e}")
    assert rc == 0 and rr[0] <= 1.01e-8
    if fp32:
        assert err <= 1e-6
        assert it[0] <= ref["iters"] + 3
    else:
        assert err <= 1e-9
        assert abs(it[0] - ref["iters"]) <= 1
    h.destroy()
