"""Seeded synthetic inputs: Kuhn-tetrahedral cube meshes, Whitney edge-element matrices
A_e = S_e + M_e (Sec. 1, eqs. (1)-(2)), the discrete gradient D_h (Sec. 1), sigma fields and
right-hand sides.

This package manufactures inputs only and holds none of the AMG method.  The GPU library
and the CPU oracle both consume its arrays.  The C source is ``kuhn.c``; it is compiled on
first use (or by ``build()``) into ``meshgen/_build/``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kuhn.c")
_BUILD = os.path.join(_HERE, "_build")
_lib = None


def build(force: bool = False) -> str:
    """Compile kuhn.c (gcc, OpenMP) and return the shared-library path."""
    src = open(_SRC, "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    so = os.path.join(_BUILD, f"libkuhn_{tag}.so")
    if force or not os.path.exists(so):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("natural", ctypes.c_int32), ("jitter", ctypes.c_double),
                ("seed_jitter", ctypes.c_uint64), ("sigma_kind", ctypes.c_int32),
                ("sigma_in", ctypes.c_double), ("sigma_out", ctypes.c_double),
                ("log_lo", ctypes.c_double), ("log_hi", ctypes.c_double),
                ("seed_sigma", ctypes.c_uint64), ("which", ctypes.c_int32),
                ("nthreads", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.kg_count.argtypes = [ctypes.POINTER(_Params), P]
        lib.kg_count.restype = ctypes.c_int
        lib.kg_fill.argtypes = [ctypes.POINTER(_Params)] + [P] * 12
        lib.kg_fill.restype = ctypes.c_int
        lib.kg_rhs.argtypes = [ctypes.c_uint64, ctypes.c_int64, P]
        lib.kg_rhs.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class MeshSpec:
    """Recipe of one synthetic eddy-current problem."""
    n: int
    natural: bool = False
    jitter: float = 0.0          # fraction of h
    seed_jitter: int = 0
    sigma: str = "const"         # const | box | lognormal
    sigma_in: float = 1.0        # const value / inside-box value / std-dev of log10 sigma
    sigma_out: float = 1.0
    log_lo: float = -6.0
    log_hi: float = 2.0
    seed_sigma: int = 0

    def params(self, which: int = 0, nthreads: int = 0) -> _Params:
        kind = {"const": 0, "box": 1, "lognormal": 2}[self.sigma]
        return _Params(self.n, int(self.natural), self.jitter, self.seed_jitter, kind,
                       self.sigma_in, self.sigma_out, self.log_lo, self.log_hi, self.seed_sigma,
                       which, nthreads)


@dataclass
class Problem:
    """CSR arrays of A_e (or S_e / M_e) and D_h plus per-node / per-edge data (all numpy)."""
    spec: MeshSpec
    n_edges: int
    n_nodes: int
    A_rowptr: np.ndarray
    A_col: np.ndarray
    A_val: np.ndarray
    D_rowptr: np.ndarray
    D_col: np.ndarray
    D_val: np.ndarray
    coords: np.ndarray = None        # [n_nodes, 3]
    sigma_edge: np.ndarray = None    # [n_edges]
    edge_ends: np.ndarray = None     # [n_edges, 2] global node ids
    extra: dict = field(default_factory=dict)


def _threads(nthreads):
    if nthreads:
        return nthreads
    return max(1, min(os.cpu_count() or 1, 32))


def counts(spec: MeshSpec, nthreads: int = 0) -> dict:
    lib = _load()
    out = np.zeros(6, dtype=np.int64)
    p = spec.params(0, _threads(nthreads))
    rc = lib.kg_count(ctypes.byref(p), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"kg_count failed ({rc})")
    return dict(n_edges=int(out[0]), n_nodes=int(out[1]), nnz_A=int(out[2]), nnz_D=int(out[3]),
                n_tets=int(out[4]), n_grid_nodes=int(out[5]))


def generate(spec: MeshSpec, which: str = "A", with_matrix: bool = True, raw_mesh: bool = False,
             nthreads: int = 0) -> Problem:
    """Build the problem.  which = 'A' (S+M), 'S' (curl-curl only) or 'M' (sigma-mass only).
    with_matrix=False skips the operator (topology and D_h only).  raw_mesh=True also returns
    all grid coordinates, the tets and the per-tet sigma in ``extra``."""
    lib = _load()
    c = counts(spec, nthreads)
    ne, nv = c["n_edges"], c["n_nodes"]
    w = {"A": 0, "S": 1, "M": 2}[which]
    p = spec.params(w, _threads(nthreads))
    A_rp = np.empty(ne + 1, np.int64) if with_matrix else None
    A_ci = np.empty(c["nnz_A"], np.int32) if with_matrix else None
    A_v = np.empty(c["nnz_A"], np.float64) if with_matrix else None
    D_rp = np.empty(ne + 1, np.int64)
    D_ci = np.empty(c["nnz_D"], np.int32)
    D_v = np.empty(c["nnz_D"], np.float64)
    coords = np.empty((nv, 3), np.float64) if with_matrix else None
    sig = np.empty(ne, np.float64) if with_matrix else None
    ends = np.empty((ne, 2), np.int64)
    X = tets = tsig = None
    if raw_mesh:
        X = np.empty((c["n_grid_nodes"], 3), np.float64)
        tets = np.empty((c["n_tets"], 4), np.int64)
        tsig = np.empty(c["n_tets"], np.float64)
    rc = lib.kg_fill(ctypes.byref(p), _ptr(A_rp), _ptr(A_ci), _ptr(A_v), _ptr(D_rp), _ptr(D_ci),
                     _ptr(D_v), _ptr(coords), _ptr(sig), _ptr(ends), _ptr(X), _ptr(tets), _ptr(tsig))
    if rc != 0:
        raise RuntimeError(f"kg_fill failed ({rc})")
    extra = {}
    if raw_mesh:
        extra = dict(coords_all=X, tets=tets, tet_sigma=tsig)
    return Problem(spec, ne, nv, A_rp, A_ci, A_v, D_rp, D_ci, D_v, coords, sig, ends, extra)


def rhs(seed: int, length: int, nrhs: int = 1) -> np.ndarray:
    """Uniform[-1, 1] right-hand sides; vector k uses seed + k.  Shape [length] or [nrhs, length]."""
    lib = _load()
    out = np.empty((nrhs, length), np.float64)
    for k in range(nrhs):
        lib.kg_rhs(ctypes.c_uint64(seed + k), length, _ptr(out[k]))
    return out[0] if nrhs == 1 else out


def workload(name: str) -> tuple[MeshSpec, int]:
    """The named synthetic workloads (mesh recipe, RHS seed).

    kuhn8:   8^3 cells, no jitter, sigma = 1, Dirichlet (3,032 unknowns), RHS seed 1.
    kuhn48:  48^3 cells, +-0.2h jitter (seed 2), sigma 1 inside [0.25,0.75]^3 else 1e-3, RHS seed 3.
    kuhn128: 128^3 cells, +-0.2h jitter (seed 4), log10 sigma ~ N(0, 2^2) clipped to [-6, 2]
             (seed 5), RHS seed 6 (block: seeds 6..21).
    kuhn96:  96^3 cells, 0.2h jitter, log-normal sigma (the learned warm-start test mesh).
    """
    if name == "kuhn8":
        return MeshSpec(8), 1
    if name == "kuhn48":
        return MeshSpec(48, jitter=0.2, seed_jitter=2, sigma="box", sigma_in=1.0, sigma_out=1e-3), 3
    if name == "kuhn128":
        return MeshSpec(128, jitter=0.2, seed_jitter=4, sigma="lognormal", sigma_in=2.0,
                        seed_sigma=5), 6
    if name == "kuhn96":
        return MeshSpec(96, jitter=0.2, seed_jitter=7, sigma="lognormal", sigma_in=2.0,
                        seed_sigma=8), 9
    if name.startswith("kuhn"):
        n = int(name[4:])
        return MeshSpec(n, jitter=0.2, seed_jitter=10 + n, sigma="lognormal", sigma_in=2.0,
                        seed_sigma=20 + n), 30 + n
    raise KeyError(name)
