"""Every path of the structural SpGEMM gives the same hierarchy, forced through the test switch
SPHC_SPGEMM_PATHS (a bit mask read at each product): 1 the small-row bin's counting and writing
passes instead of its one pass into temporary slots; 2 the numeric pass binned by output row
length for any number of rows; 4 never binned by length; 8 the hash bins through counting and
numeric passes instead of their one pass into an arena; 16 sub-arenas so small that most one-pass
rows overflow into the counting path; 32 every transpose by the stable radix sort (by default only
large transposes with long rows take it); 64 the smaller one-pass tables of the upper-triangle
products (by default only on products of many rows).  The default choices depend on the free device memory and
on the number of rows, so the small test meshes would otherwise exercise one branch only (the
coarse levels' long rows also overflow the one-pass tables by themselves).  Each forced path against the CPU oracle: integer patterns bit for bit,
FP64 values (A_l, A_n, P_n, P_e on every level) to 1e-10 of the largest entry."""
import pytest

import meshgen
from gpu_util import assert_csr_close, assert_csr_equal_pattern, gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu

OPTS = dict(max_coarse=200)


@pytest.fixture(scope="module")
def case():
    p = meshgen.generate(meshgen.MeshSpec(12, jitter=0.2, seed_jitter=4, sigma="lognormal", sigma_in=2.0,
                                          seed_sigma=5))
    return p, oracle_setup(p, **OPTS)


@pytest.mark.parametrize("paths", ["0", "1", "16", "17", "8", "10", "12", "11", "13", "32", "49", "64", "80"])
def test_spgemm_paths_match_oracle(case, paths, monkeypatch):
    p, o = case
    monkeypatch.setenv("SPHC_SPGEMM_PATHS", paths)
    h = gpu_setup(p, vcycle_fp32=0, **OPTS)
    assert h.nlevels == o.nlevels
    for l in range(o.nlevels):
        assert_csr_close(h.export(l, "A"), o.matrix(l, "A"), f"L{l} A", 1e-10)
        assert_csr_close(h.export(l, "An"), o.matrix(l, "An"), f"L{l} A_n", 1e-10)
        if not o.sizes(l)["has_transfer"]:
            continue
        assert_csr_equal_pattern(h.export(l, "Pe"), o.matrix(l, "Pe"), f"L{l} N")
        for what in ("Pn", "Pe"):
            assert_csr_close(h.export(l, what), o.matrix(l, what), f"L{l} {what}", 1e-10)
    h.destroy()
