"""The order of a symmetric multicolour Gauss-Seidel sweep (Sec. 6.1 smoother).

The oracle sweeps colours 0..C-1 forward and C-1..0 backward.  The GPU leaves out the backward
sweep's first colour, C-1: right after the forward sweep updated those rows their residual is
zero, and rows of one colour do not couple, so repeating the update changes x only by rounding.
These tests pin that reading on the oracle's own colouring, with plain numpy sweeps.
"""
import numpy as np
import scipy.sparse as sp

import meshgen
import oracle


def _problem():
    spec = meshgen.MeshSpec(6, jitter=0.2, seed_jitter=3, sigma="lognormal", sigma_in=2.0, seed_sigma=4)
    p = meshgen.generate(spec)
    A = sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr), shape=(p.n_edges, p.n_edges))
    color, ncol = oracle.color(p.A_rowptr, p.A_col, 0)
    return A, color, ncol


def _sweep(A, color, order, b, x):
    d = A.diagonal()
    for c in order:
        rows = np.flatnonzero(color == c)
        x[rows] += (b[rows] - A[rows] @ x) / d[rows]
    return x


def test_colouring_is_proper():
    A, color, ncol = _problem()
    C = A.tocoo()
    off = C.row != C.col
    assert ncol == color.max() + 1
    assert np.all(color[C.row[off]] != color[C.col[off]])


def test_repeated_middle_colour_changes_nothing_but_rounding():
    A, color, ncol = _problem()
    rng = np.random.default_rng(5)
    b = rng.uniform(-1, 1, A.shape[0])
    x0 = rng.uniform(-1, 1, A.shape[0])
    full = list(range(ncol)) + list(range(ncol - 1, -1, -1))
    short = list(range(ncol)) + list(range(ncol - 2, -1, -1))
    xf = _sweep(A, color, full, b, x0.copy())
    xs = _sweep(A, color, short, b, x0.copy())
    assert np.abs(xf - xs).max() <= 1e-12 * np.abs(xf).max()
    # and the sweep does something: x moved
    assert np.abs(xf - x0).max() > 1e-3 * np.abs(x0).max()


def test_last_colour_rows_have_zero_residual_after_their_update():
    A, color, ncol = _problem()
    rng = np.random.default_rng(6)
    b = rng.uniform(-1, 1, A.shape[0])
    x = _sweep(A, color, list(range(ncol)), b, rng.uniform(-1, 1, A.shape[0]))
    rows = np.flatnonzero(color == ncol - 1)
    r = b[rows] - A[rows] @ x
    assert np.abs(r).max() <= 1e-12 * (np.abs(A[rows]) @ np.abs(x)).max()
