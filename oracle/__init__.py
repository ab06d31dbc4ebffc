"""ORACLE -- test infrastructure.  A plain FP64 single-threaded CPU implementation of the
SpHcurlAMG setup and solve (``sphc_oracle.c``), written from the paper's definitions and
independent of the GPU library.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.

The C source is compiled with gcc on first use (or by ``build()``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sphc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lib = None

# matrix ids of orc_matrix_get
MAT = dict(A=0, D=1, An=2, Pn=3, DH=4, T=5, Pe=6, P0=7)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle: plain (single-threaded, the tests' build) or with -fopenmp (the timed
    CPU baseline; its pragmas split only independent rows, so results are bit-identical)."""
    src = open(_SRC, "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    so = os.path.join(_BUILD, f"liborc{'_omp' if openmp else ''}_{tag}.so")
    if force or not os.path.exists(so):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", *flags,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


class _Opts(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_int32), ("emin_iters", ctypes.c_int32),
                ("max_coarse", ctypes.c_int64), ("emin_omega", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("power_iters", ctypes.c_int32),
                ("unsmoothed_pn", ctypes.c_int32), ("agg0", ctypes.c_void_p),
                ("nagg0", ctypes.c_int64), ("p0_value", ctypes.c_double), ("emin_method", ctypes.c_int32),
                ("sa_theta", ctypes.c_double), ("pn_alg1", ctypes.c_int32), ("alg1_passes", ctypes.c_int32)]


_OPENMP = os.environ.get("SPHC_ORACLE_OPENMP", "0") == "1"


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build(openmp=_OPENMP))
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.orc_setup.argtypes = [I64, I64, P, P, P, P, P, P, ctypes.POINTER(_Opts), P]
        lib.orc_setup.restype = P
        lib.orc_update.argtypes = [P, P, ctypes.POINTER(_Opts), P]
        lib.orc_update.restype = P
        lib.orc_free.argtypes = [P]
        lib.orc_free.restype = None
        lib.orc_num_levels.argtypes = [P]
        lib.orc_status.argtypes = [P]
        lib.orc_level_sizes.argtypes = [P, I32, P]
        lib.orc_level_scalars.argtypes = [P, I32, P]
        lib.orc_level_hist.argtypes = [P, I32, P]
        lib.orc_matrix_nnz.argtypes = [P, I32, I32, P, P, P]
        lib.orc_matrix_get.argtypes = [P, I32, I32, P, P, P]
        lib.orc_level_ivec.argtypes = [P, I32, I32, P]
        lib.orc_vcycle.argtypes = [P, P, P]
        lib.orc_vcycle.restype = None
        lib.orc_solve.argtypes = [P, P, P, ctypes.c_double, I32, I32, P, P, P]
        lib.orc_color.argtypes = [I64, P, P, ctypes.c_uint64, P]
        lib.orc_aggregate.argtypes = [I64, P, P, ctypes.c_uint64, P]
        lib.orc_aggregate.restype = I64
        lib.orc_coarse_gradient.argtypes = [I64, I64, P, P, P, P, I64, I64, P, P, P]
        lib.orc_coarse_gradient.restype = I64
        lib.orc_minnorm.argtypes = [I32, I32, P, P, I32, P]
        lib.orc_project.argtypes = [I32, I32, P, I32, P]
        lib.orc_gen_piecewise_const.argtypes = [I64, I64, P, P, P, I32, P]
        lib.orc_gen_piecewise_const.restype = I64
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class CSR:
    """Minimal host CSR (rowptr int64, col int32, val float64)."""

    def __init__(self, rowptr, col, val, shape):
        self.rowptr, self.col, self.val, self.shape = rowptr, col, val, shape

    def to_dense(self):
        M = np.zeros(self.shape)
        for i in range(self.shape[0]):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            np.add.at(M[i], self.col[s:e], self.val[s:e])
        return M

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=self.shape)


class Hierarchy:
    """Result of ``setup``; owns the C hierarchy."""

    def __init__(self, ptr, setup_seconds):
        self._ptr = ptr
        self.setup_seconds = setup_seconds
        self._lib = _load()

    def __del__(self):
        if getattr(self, "_ptr", None):
            self._lib.orc_free(self._ptr)
            self._ptr = None

    @property
    def status(self):
        return self._lib.orc_status(self._ptr)

    @property
    def nlevels(self):
        return self._lib.orc_num_levels(self._ptr)

    def sizes(self, l):
        out = np.zeros(17, np.int64)
        self._lib.orc_level_sizes(self._ptr, l, _p(out))
        keys = ["ne", "nv", "nnzA", "nnzD", "nnzAn", "nagg", "nnzPn", "nH", "nnzDH", "nnzPe",
                "ncol_e", "ncol_n", "n_added", "nnzT", "n_infeasible0", "has_transfer",
                "n_rows_unsmoothed"]
        return dict(zip(keys, (int(v) for v in out)))

    def scalars(self, l):
        out = np.zeros(4)
        self._lib.orc_level_scalars(self._ptr, l, _p(out))
        return dict(rho=out[0], omega_sa=out[1], energy0=out[2], energy1=out[3])

    def hist(self, l):
        out = np.zeros((33, 33), np.int64)
        self._lib.orc_level_hist(self._ptr, l, _p(out))
        return out

    def matrix(self, l, name) -> CSR:
        nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = self._lib.orc_matrix_nnz(self._ptr, l, MAT[name], ctypes.byref(nr), ctypes.byref(nc),
                                      ctypes.byref(nnz))
        if rc != 0:
            raise KeyError((l, name))
        rp = np.empty(nr.value + 1, np.int64)
        ci = np.empty(nnz.value, np.int32)
        v = np.empty(nnz.value, np.float64)
        self._lib.orc_matrix_get(self._ptr, l, MAT[name], _p(rp), _p(ci), _p(v))
        return CSR(rp, ci, v, (nr.value, nc.value))

    def ivec(self, l, name):
        s = self.sizes(l)
        n = s["ne"] if name == "col_e" else s["nv"]
        out = np.empty(n, np.int32)
        rc = self._lib.orc_level_ivec(self._ptr, l, {"agg": 0, "col_e": 1, "col_n": 2}[name], _p(out))
        if rc != 0:
            raise KeyError((l, name))
        return out

    def update(self, A_values, max_levels=8, emin_iters=1, max_coarse=1000, emin_omega=0.5, seed=0,
               power_iters=15, emin_method=0):
        """Hierarchy of a related system: new values of A on this hierarchy's level-0 pattern, with
        this hierarchy's aggregates, D_H and pattern kept and its P_e as the initial guess."""
        av = _c(A_values, np.float64)
        o = _Opts(max_levels, emin_iters, max_coarse, emin_omega, seed, power_iters, 0, None, 0, 0.0,
                  int(emin_method), 0.0, 0, 2)
        st = ctypes.c_int()
        t0 = time.perf_counter()
        ptr = self._lib.orc_update(self._ptr, _p(av), ctypes.byref(o), ctypes.byref(st))
        h = Hierarchy(ptr, time.perf_counter() - t0)
        h._keep = (av, self)
        return h

    def vcycle(self, r):
        r = _c(r, np.float64)
        z = np.empty_like(r)
        self._lib.orc_vcycle(self._ptr, _p(r), _p(z))
        return z

    def solve(self, b, tol=1e-8, max_iter=200, precond=True):
        b = _c(b, np.float64)
        x = np.empty_like(b)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(max_iter)
        st = self._lib.orc_solve(self._ptr, _p(b), _p(x), tol, max_iter, int(precond),
                                 ctypes.byref(it), ctypes.byref(rel), _p(hist))
        return dict(x=x, status=st, iters=it.value, relres=rel.value, history=hist[:it.value])

    def operator_complexity(self):
        tot = sum(self.sizes(l)["nnzA"] for l in range(self.nlevels))
        return tot / self.sizes(0)["nnzA"]


def setup(ne, nv, A, D, max_levels=8, emin_iters=1, max_coarse=1000, emin_omega=0.5, seed=0,
          power_iters=15, unsmoothed_pn=False, agg0=None, p0_value=0.0, emin_method=0, sa_theta=0.0,
          pn_alg1=0, alg1_passes=2) -> Hierarchy:
    """A, D: (rowptr, col, val) triplets of A_e (ne x ne) and D_h (ne x nv)."""
    lib = _load()
    Arp, Aci, Av = _c(A[0], np.int64), _c(A[1], np.int32), _c(A[2], np.float64)
    Drp, Dci, Dv = _c(D[0], np.int64), _c(D[1], np.int32), _c(D[2], np.float64)
    aggarr = None
    nagg0 = 0
    if agg0 is not None:
        aggarr = _c(agg0, np.int32)
        nagg0 = int(aggarr.max()) + 1 if aggarr.size else 0
    o = _Opts(max_levels, emin_iters, max_coarse, emin_omega, seed, power_iters, int(unsmoothed_pn),
              None if aggarr is None else aggarr.ctypes.data, nagg0, p0_value, int(emin_method), float(sa_theta),
              int(pn_alg1), int(alg1_passes))
    st = ctypes.c_int()
    t0 = time.perf_counter()
    ptr = lib.orc_setup(ne, nv, _p(Arp), _p(Aci), _p(Av), _p(Drp), _p(Dci), _p(Dv), ctypes.byref(o),
                        ctypes.byref(st))
    h = Hierarchy(ptr, time.perf_counter() - t0)
    h._keep = (Arp, Aci, Av, Drp, Dci, Dv, aggarr)
    return h


def setup_problem(prob, **kw) -> Hierarchy:
    """Setup from a ``meshgen.Problem``."""
    return setup(prob.n_edges, prob.n_nodes, (prob.A_rowptr, prob.A_col, prob.A_val),
                 (prob.D_rowptr, prob.D_col, prob.D_val), **kw)


# ---------------------------------------------------------------- unit entry points
def color(rowptr, col, seed):
    lib = _load()
    n = len(rowptr) - 1
    out = np.empty(n, np.int32)
    rp, ci = _c(rowptr, np.int64), _c(col, np.int32)
    nc = lib.orc_color(n, _p(rp), _p(ci), seed, _p(out))
    return out, nc


def aggregate(rowptr, col, seed):
    lib = _load()
    n = len(rowptr) - 1
    out = np.empty(n, np.int32)
    rp, ci = _c(rowptr, np.int64), _c(col, np.int32)
    nagg = lib.orc_aggregate(n, _p(rp), _p(ci), seed, _p(out))
    if nagg < 0:
        raise RuntimeError("aggregation failed")
    return out, int(nagg)


def coarse_gradient(ne, nv, D, agg, nagg):
    lib = _load()
    rp, ci, v = _c(D[0], np.int64), _c(D[1], np.int32), _c(D[2], np.float64)
    a = _c(agg, np.int32)
    nH = lib.orc_coarse_gradient(ne, nv, _p(rp), _p(ci), _p(v), _p(a), nagg, 0, None, None, None)
    Hrp = np.empty(nH + 1, np.int64)
    Hci = np.empty(2 * nH, np.int32)
    Hv = np.empty(2 * nH, np.float64)
    lib.orc_coarse_gradient(ne, nv, _p(rp), _p(ci), _p(v), _p(a), nagg, nH, _p(Hrp), _p(Hci), _p(Hv))
    nnz = int(Hrp[-1])
    return CSR(Hrp, Hci[:nnz].copy(), Hv[:nnz].copy(), (int(nH), int(nagg)))


def minnorm(G, r, singular):
    """Least-norm p with G^T p = r (G: np x m; singular -> drop the last column)."""
    lib = _load()
    G = _c(G, np.float64)
    r = _c(r, np.float64)
    p = np.empty(G.shape[0])
    k = lib.orc_minnorm(G.shape[0], G.shape[1], _p(G), _p(r), int(singular), _p(p))
    if k < 0:
        raise RuntimeError("infeasible local system")
    return p


def project(G, x, singular):
    lib = _load()
    G = _c(G, np.float64)
    x = _c(x, np.float64).copy()
    rc = lib.orc_project(G.shape[0], G.shape[1], _p(G), int(singular), _p(x))
    if rc < 0:
        raise RuntimeError("infeasible local system")
    return x


def gen_piecewise_const(P: "CSR", passes=2):
    """Alg. 1 (Gen_Piecewise_Const) under the oracle's reading: the column of each row."""
    lib = _load()
    rp, ci, v = _c(P.rowptr, np.int64), _c(P.col, np.int32), _c(P.val, np.float64)
    out = np.empty(P.shape[0], np.int32)
    lib.orc_gen_piecewise_const(P.shape[0], P.shape[1], _p(rp), _p(ci), _p(v), int(passes), _p(out))
    return out
