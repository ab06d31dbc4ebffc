"""The OpenMP build of the oracle (the timed CPU baseline) splits only independent rows, so it
must reproduce the plain build bit for bit: prolongators, coarse operators and the CG solution."""
import os
import subprocess
import sys

import numpy as np

import meshgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SPEC = "meshgen.MeshSpec(10, jitter=0.2, seed_jitter=3, sigma='lognormal', sigma_in=2.0, seed_sigma=4)"

DUMP = f"""
import sys; sys.path.insert(0, {ROOT!r})
import numpy as np, meshgen, oracle
p = meshgen.generate({SPEC})
h = oracle.setup_problem(p, max_coarse=100, emin_iters=2)
r = h.solve(meshgen.rhs(5, p.n_edges))
out = dict(x=r["x"], iters=r["iters"])
for l in range(h.nlevels - 1):
    out[f"Pe{{l}}"] = h.matrix(l, "Pe").val
    out[f"A{{l + 1}}"] = h.matrix(l + 1, "A").val
np.savez(sys.argv[1], **out)
"""


def test_openmp_build_is_bit_identical(tmp_path):
    out = str(tmp_path / "omp.npz")
    env = dict(os.environ, SPHC_ORACLE_OPENMP="1", OMP_NUM_THREADS="4")
    subprocess.run([sys.executable, "-c", DUMP, out], check=True, env=env, timeout=300)
    omp = np.load(out)
    p = meshgen.generate(eval(SPEC))
    h = oracle.setup_problem(p, max_coarse=100, emin_iters=2)
    r = h.solve(meshgen.rhs(5, p.n_edges))
    assert int(omp["iters"]) == r["iters"]
    np.testing.assert_array_equal(omp["x"], r["x"])
    for l in range(h.nlevels - 1):
        np.testing.assert_array_equal(omp[f"Pe{l}"], h.matrix(l, "Pe").val)
        np.testing.assert_array_equal(omp[f"A{l + 1}"], h.matrix(l + 1, "A").val)
