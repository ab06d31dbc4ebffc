"""Helpers of the GPU parity tests: run the library and the oracle on the same inputs."""
import numpy as np

import meshgen
import oracle
import paper_2506_08284_gb300 as pkg


def gpu_setup(p, **opts):
    o = pkg.sphc.default_opts(**opts)
    A = (p.n_edges, p.n_edges, p.A_rowptr, p.A_col, p.A_val)
    D = (p.n_edges, p.n_nodes, p.D_rowptr, p.D_col, p.D_val)
    return pkg.sphc.setup(A, D, p.coords, p.sigma_edge, o)


def oracle_setup(p, **opts):
    kw = dict(max_levels=opts.get("max_levels", 8), emin_iters=opts.get("emin_iters", 1),
              max_coarse=opts.get("max_coarse", 1000), emin_omega=opts.get("emin_omega", 0.5),
              seed=opts.get("seed", 0), power_iters=opts.get("power_iters", 15),
              emin_method=opts.get("emin_method", 0), sa_theta=opts.get("sa_theta", 0.0),
              pn_alg1=opts.get("pn_alg1", 0), alg1_passes=opts.get("alg1_passes", 2))
    return oracle.setup_problem(p, **kw)


def assert_csr_equal_pattern(g, o, what):
    rp, ci, v, shape = g
    assert shape == o.shape, (what, shape, o.shape)
    np.testing.assert_array_equal(rp, o.rowptr, err_msg=f"{what}: row pointers")
    np.testing.assert_array_equal(ci, o.col, err_msg=f"{what}: columns")


def assert_csr_close(g, o, what, rtol):
    assert_csr_equal_pattern(g, o, what)
    v = g[2]
    scale = max(np.abs(o.val).max() if o.val.size else 0.0, 1e-300)
    err = np.abs(v - o.val).max() if v.size else 0.0
    assert err <= rtol * scale, f"{what}: max |gpu - oracle| = {err:.3e} > {rtol:g} * {scale:.3e}"


def problem(name_or_spec):
    if isinstance(name_or_spec, str):
        spec, seed = meshgen.workload(name_or_spec)
    else:
        spec, seed = name_or_spec, 1
    return meshgen.generate(spec), seed
