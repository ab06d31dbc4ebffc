"""A seeded input whose local coarse graphs are reducible (Sec. 4.2, Fig. 3), so that
make_irreducible has work to do.

On the Kuhn-tet meshes every nodal neighbour lies in an aggregate joined to the node's own
aggregate by a fine edge, so the local graphs stay connected.  Adding a few symmetric positive
rank-1 couplings eps (e_i + e_j)(e_i + e_j)^T between distant edges to A_e (which keeps A_e SPD)
couples nodes that no fine edge joins; the smoothed P_n then reaches aggregates that are not
joined to the others in T_i by any coarse edge."""
import numpy as np
import scipy.sparse as sp

import meshgen


def coupled_problem(n=8, ncouple=40, seed=2):
    p = meshgen.generate(meshgen.MeshSpec(n))
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr)).tolil()
    ne = A.shape[0]
    rng = np.random.default_rng(seed)
    for _ in range(ncouple):
        i, j = (int(x) for x in rng.integers(0, ne, 2))
        if i == j:
            continue
        eps = 0.05 * A[i, i]
        A[i, j] += eps
        A[j, i] += eps
        A[i, i] += eps
        A[j, j] += eps
    A = A.tocsr()
    A.sort_indices()
    return p, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)
