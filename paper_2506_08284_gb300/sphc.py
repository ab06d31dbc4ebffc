"""Thin ctypes binding of libsphc.so (the C ABI of ``include/sphc.h``).

Argument marshalling only: every step of the setup and the solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU fallback: loading fails
loudly when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SPHC_OK = 0
ERRORS = {-1: "SPHC_EINVAL", -2: "SPHC_ENOMEM", -3: "SPHC_ECUDA", -4: "SPHC_ENOTCONV", -5: "SPHC_EBREAKDOWN",
          -6: "SPHC_EINFEASIBLE", -7: "SPHC_ETIMEOUT", -8: "SPHC_ESTAGNATION", -9: "SPHC_ENUMERIC",
          -10: "SPHC_ELIMIT"}
X = dict(A=0, D=1, An=2, Pn=3, DH=4, T=5, Pe=6, P0=7, agg=16, col_e=17, col_n=18)


class SphcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class sphc_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class sphc_opts(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_int32), ("emin_iters", ctypes.c_int32), ("max_coarse", ctypes.c_int64),
                ("emin_omega", ctypes.c_double), ("seed", ctypes.c_uint64), ("power_iters", ctypes.c_int32),
                ("vcycle_fp32", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("flexible", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("cg_graph", ctypes.c_int32), ("learned", ctypes.c_int32),
                ("learned_emin_iters", ctypes.c_int32), ("mlp_params", ctypes.c_void_p),
                ("autotune", ctypes.c_int32), ("sweep_form", ctypes.c_int32), ("mlp_wait_polls", ctypes.c_int32),
                ("sell_lpr0", ctypes.c_int32), ("sell_ch0", ctypes.c_int32), ("emin_fp32", ctypes.c_int32),
                ("block_rhs", ctypes.c_int32), ("emin_method", ctypes.c_int32), ("pn_alg1", ctypes.c_int32),
                ("sa_theta", ctypes.c_double), ("alg1_passes", ctypes.c_int32), ("grid_wait_polls", ctypes.c_int32)]


class sphc_train_opts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("weight_decay", ctypes.c_float), ("pad", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("reserved", ctypes.c_int32 * 4)]


MLP_NFEAT, MLP_HIDDEN, MLP_NPARAM = 32, 128, 20929


class sphc_level_info(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("nnz_A", ctypes.c_int64),
                ("nnz_An", ctypes.c_int64), ("n_aggregates", ctypes.c_int64), ("n_coarse_edges", ctypes.c_int64),
                ("nnz_Pn", ctypes.c_int64), ("nnz_Pe", ctypes.c_int64), ("nnz_T", ctypes.c_int64),
                ("n_colors_edge", ctypes.c_int32), ("n_colors_node", ctypes.c_int32),
                ("n_added_edges", ctypes.c_int64), ("n_rows_unsmoothed", ctypes.c_int64),
                ("rho", ctypes.c_double), ("omega_sa", ctypes.c_double), ("max_pattern_row", ctypes.c_int64),
                ("max_T_row", ctypes.c_int64), ("sell_lpr_edge", ctypes.c_int32), ("sell_ch_edge", ctypes.c_int32),
                ("sell_lpr_node", ctypes.c_int32), ("sell_ch_node", ctypes.c_int32),
                ("sell_stored_edge", ctypes.c_int64), ("sell_stored_node", ctypes.c_int64),
                ("colour_rounds_edge", ctypes.c_int32), ("colour_rounds_node", ctypes.c_int32),
                ("sweep_kind_edge", ctypes.c_int32), ("sweep_kind_node", ctypes.c_int32)]


class sphc_stats(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("operator_complexity", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("last_iters", ctypes.c_int32),
                ("last_relres", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class sphc_timer(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_double), ("calls", ctypes.c_int64),
                ("bytes_per_call", ctypes.c_double)]


EXPORTED = ["sphc_default_opts", "sphc_setup", "sphc_solve", "sphc_vcycle", "sphc_get_stats",
            "sphc_get_level_info", "sphc_export_size", "sphc_export", "sphc_destroy", "sphc_last_error",
            "sphc_get_profile", "sphc_launch_count", "sphc_relres_noalloc", "sphc_default_train_opts",
            "sphc_mlp_train", "sphc_mlp_predict", "sphc_mlp_gradient", "sphc_export_features",
            "sphc_setup_batched", "sphc_solve_batched", "sphc_batch_destroy", "sphc_trim_memory",
            "sphc_memory_usage", "sphc_mlp_predict_level", "sphc_cond_estimate", "sphc_setup_update", "sphc_vcycle_factor", "sphc_prolongator_energy",
            "sphc_grid_barrier_check"]

_lib = None


def load(path: str | None = None):
    """Load (building first if needed) libsphc.so and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    so = path or _build.build()
    lib = ctypes.CDLL(so)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.sphc_default_opts.argtypes = [ctypes.POINTER(sphc_opts)]
    lib.sphc_setup.argtypes = [ctypes.POINTER(sphc_csr), ctypes.POINTER(sphc_csr), P, P, ctypes.POINTER(sphc_opts),
                               P, ctypes.POINTER(P)]
    lib.sphc_solve.argtypes = [P, P, P, I, ctypes.c_double, P, P, P]
    lib.sphc_vcycle.argtypes = [P, P, P, P]
    lib.sphc_get_stats.argtypes = [P, ctypes.POINTER(sphc_stats)]
    lib.sphc_get_level_info.argtypes = [P, I, ctypes.POINTER(sphc_level_info)]
    lib.sphc_export_size.argtypes = [P, I, I, P, P, P]
    lib.sphc_export.argtypes = [P, I, I, P, P, P, P, P]
    lib.sphc_destroy.argtypes = [P]
    lib.sphc_destroy.restype = None
    lib.sphc_get_profile.argtypes = [P, ctypes.POINTER(sphc_timer), I, ctypes.POINTER(I)]
    lib.sphc_relres_noalloc.argtypes = [P, P, P, I, P, P]
    lib.sphc_trim_memory.argtypes = [I, ctypes.c_uint64]
    lib.sphc_memory_usage.argtypes = [I, P, P]
    lib.sphc_default_train_opts.argtypes = [ctypes.POINTER(sphc_train_opts)]
    lib.sphc_mlp_train.argtypes = [P, P, I64, ctypes.POINTER(sphc_train_opts), P, P, P]
    lib.sphc_mlp_predict.argtypes = [P, P, I64, P, P]
    lib.sphc_mlp_gradient.argtypes = [P, P, P, I, P, P, P]
    lib.sphc_export_features.argtypes = [P, I, P, P, P]
    lib.sphc_mlp_predict_level.argtypes = [P, I, P, P, P]
    lib.sphc_cond_estimate.argtypes = [P, I, P, P, P, P]
    lib.sphc_setup_update.argtypes = [P, P, P]
    lib.sphc_vcycle_factor.argtypes = [P, I, I, ctypes.c_uint64, P, P]
    lib.sphc_prolongator_energy.argtypes = [P, I, P, P]
    lib.sphc_grid_barrier_check.argtypes = [I, I, P, P]
    lib.sphc_setup_batched.argtypes = [I, P, P, P, P, ctypes.POINTER(sphc_opts), P, ctypes.POINTER(P)]
    lib.sphc_solve_batched.argtypes = [P, P, P, I, ctypes.c_double, P, P, P]
    lib.sphc_batch_destroy.argtypes = [P]
    lib.sphc_batch_destroy.restype = None
    lib.sphc_launch_count.argtypes = []
    lib.sphc_launch_count.restype = ctypes.c_int64
    lib.sphc_last_error.argtypes = []
    lib.sphc_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("sphc_destroy", "sphc_last_error", "sphc_launch_count", "sphc_batch_destroy"):
            getattr(lib, name).restype = I
    if path is None:
        _lib = lib
    return lib


def _check(rc):
    if rc != SPHC_OK:
        raise SphcError(rc, load().sphc_last_error().decode())


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _require_f64(name, a, need):
    """Raise ValueError unless a is a contiguous float64 array/tensor with at least `need` entries."""
    if isinstance(a, np.ndarray):
        ok_t, ok_c, size = a.dtype == np.float64, a.flags["C_CONTIGUOUS"], a.size
    else:
        import torch
        ok_t, ok_c, size = a.dtype == torch.float64, a.is_contiguous(), a.numel()
    if not ok_t:
        raise ValueError(f"{name}: float64 required")
    if not ok_c:
        raise ValueError(f"{name}: contiguous storage required")
    if size < need:
        raise ValueError(f"{name}: {size} entries, at least {need} required")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_opts(**kw) -> sphc_opts:
    """Options with the library defaults, overridden by keyword.  mlp_params may be a float32
    numpy array or torch tensor; the options object keeps a reference to it."""
    o = sphc_opts()
    _check(load().sphc_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "mlp_params" and v is not None and not isinstance(v, int):
            o._keep = v
            v = _ptr(v)
        setattr(o, k, v)
    return o


def make_csr(nrows, ncols, rowptr, col, val):
    return sphc_csr(nrows, ncols, _ptr(rowptr), _ptr(col), _ptr(val))


class Handle:
    """An AMG hierarchy built by ``sphc_setup``; keeps the library handle."""

    def __init__(self, ptr):
        self._ptr = ctypes.c_void_p(ptr)

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            load().sphc_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(0)

    @property
    def ptr(self):
        return self._ptr

    def solve(self, b, x, tol=1e-8, nrhs=1, stream=None):
        """b, x: FP64 arrays/tensors of nrhs x n_e.  Returns (status, iters[], relres[])."""
        n = self.level_info(0)["n_edges"]
        _require_f64("b", b, nrhs * n)
        _require_f64("x", x, nrhs * n)
        it = (ctypes.c_int * nrhs)()
        rr = (ctypes.c_double * nrhs)()
        rc = load().sphc_solve(self._ptr, _ptr(b), _ptr(x), nrhs, tol, _stream(stream), it, rr)
        if rc not in (SPHC_OK, -4, -5, -8):
            _check(rc)
        return rc, list(it), list(rr)

    def update(self, A_values, stream=None):
        """Rebuild for new values of A_e on the same pattern (sphc_setup_update)."""
        _require_f64("A_values", A_values, self.level_info(0)["nnz_A"])
        _check(load().sphc_setup_update(self._ptr, _ptr(A_values), _stream(stream)))

    def vcycle_factor(self, iters=30, tail=10, seed=1, stream=None):
        """Geometric-mean A-norm contraction of the V-cycle as a stationary iteration (b = 0)."""
        f = ctypes.c_double()
        _check(load().sphc_vcycle_factor(self._ptr, int(iters), int(tail), int(seed), ctypes.byref(f),
                                         _stream(stream)))
        return f.value

    def energy(self, level=0, stream=None):
        """trace(P_e^T A P_e) of a level's edge prolongator."""
        e = ctypes.c_double()
        _check(load().sphc_prolongator_energy(self._ptr, int(level), ctypes.byref(e), _stream(stream)))
        return e.value

    def cond_estimate(self, max_steps=5, stream=None):
        """(kappa_1(D^-1 A_e) estimate, ||D^-1 A_e||_1, estimated ||(D^-1 A_e)^-1||_1)."""
        k, nb, ni = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().sphc_cond_estimate(self._ptr, int(max_steps), ctypes.byref(k), ctypes.byref(nb),
                                         ctypes.byref(ni), _stream(stream)))
        return k.value, nb.value, ni.value

    def vcycle(self, r, z, stream=None):
        _check(load().sphc_vcycle(self._ptr, _ptr(r), _ptr(z), _stream(stream)))

    def stats(self) -> dict:
        st = sphc_stats()
        _check(load().sphc_get_stats(self._ptr, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in sphc_stats._fields_}

    def level_info(self, level) -> dict:
        li = sphc_level_info()
        _check(load().sphc_get_level_info(self._ptr, level, ctypes.byref(li)))
        return {k: getattr(li, k) for k, _ in sphc_level_info._fields_}

    def relres_noalloc(self, b, x, relres, nrhs=1, stream=None):
        """||b - A x|| / ||b|| through sphc_relres_noalloc (b, x on the device; relres host or device).
        Returns the status code.  b and x must be contiguous float64 with at least nrhs * n_e
        entries and relres contiguous float64 with at least nrhs entries (checked here, before the
        library reads them)."""
        n = self.level_info(0)["n_edges"]
        for name, a, need in (("b", b, nrhs * n), ("x", x, nrhs * n), ("relres", relres, nrhs)):
            _require_f64(name, a, max(need, 0))
        return load().sphc_relres_noalloc(self._ptr, _ptr(b), _ptr(x), nrhs, _ptr(relres), _stream(stream))

    def features(self, level=0, stream=None):
        """(X [nnz(P_e) x 32], y = P_e - P0 [nnz(P_e)]) of a level, as numpy float32."""
        nr, nc, nz = self.export_size(level, "Pe")
        X = np.empty((nz, MLP_NFEAT), np.float32)
        y = np.empty(nz, np.float32)
        _check(load().sphc_export_features(self._ptr, level, _ptr(X), _ptr(y), _stream(stream)))
        return X, y

    def predict_level(self, params, level=0, stream=None):
        """Raw outputs of the fused tensor-core inference on every pattern entry of a level
        (numpy float32 [nnz(P_e)])."""
        nr, nc, nz = self.export_size(level, "Pe")
        params = np.ascontiguousarray(params, np.float32)
        if params.size != MLP_NPARAM:
            raise ValueError(f"params: {params.size} entries, {MLP_NPARAM} required")
        out = np.empty(nz, np.float32)
        _check(load().sphc_mlp_predict_level(self._ptr, level, _ptr(params), _ptr(out), _stream(stream)))
        return out

    def profile(self) -> dict:
        arr = (sphc_timer * 256)()
        n = ctypes.c_int()
        _check(load().sphc_get_profile(self._ptr, arr, 256, ctypes.byref(n)))
        return {arr[i].name.decode(): dict(ms=arr[i].ms, calls=arr[i].calls, bytes_per_call=arr[i].bytes_per_call)
                for i in range(min(n.value, 256))}

    @property
    def nlevels(self):
        return self.stats()["n_levels"]

    def export_size(self, level, what):
        nr, nc, nz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().sphc_export_size(self._ptr, level, X[what], ctypes.byref(nr), ctypes.byref(nc),
                                       ctypes.byref(nz)))
        return nr.value, nc.value, nz.value

    def export(self, level, what, stream=None):
        """Copy a level array to host numpy: CSR -> (rowptr, col, val, shape); vector -> int32 array."""
        nr, nc, nz = self.export_size(level, what)
        if X[what] >= 16:
            out = np.empty(nr, np.int32)
            _check(load().sphc_export(self._ptr, level, X[what], None, None, None, _ptr(out), _stream(stream)))
            return out
        rp = np.empty(nr + 1, np.int64)
        ci = np.empty(nz, np.int32)
        v = np.empty(nz, np.float64)
        _check(load().sphc_export(self._ptr, level, X[what], _ptr(rp), _ptr(ci), _ptr(v), None, _stream(stream)))
        return rp, ci, v, (nr, nc)


def default_train_opts(**kw) -> sphc_train_opts:
    o = sphc_train_opts()
    _check(load().sphc_default_train_opts(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def mlp_train(X, y, params, opts=None, stream=None):
    """Train in place on the GPU; X float32 [m, 32], y float32 [m], params float32 [NPARAM].
    Returns the loss history."""
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    o = opts if opts is not None else default_train_opts()
    hist = np.zeros(max(o.steps, 1), np.float32)
    _check(load().sphc_mlp_train(_ptr(X), _ptr(y), X.shape[0], ctypes.byref(o), _ptr(params), _ptr(hist),
                                 _stream(stream)))
    return hist[:o.steps]


def mlp_predict(params, X, stream=None):
    X = np.ascontiguousarray(X, np.float32)
    out = np.empty(X.shape[0], np.float32)
    _check(load().sphc_mlp_predict(_ptr(params), _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
    return out


def mlp_gradient(params, X, y, stream=None):
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    grad = np.zeros(MLP_NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().sphc_mlp_gradient(_ptr(params), _ptr(X), _ptr(y), X.shape[0], _ptr(grad), _ptr(loss),
                                    _stream(stream)))
    return grad, float(loss[0])


class Batch:
    """Independent systems solved together (sphc_setup_batched / sphc_solve_batched)."""

    def __init__(self, ptr, sizes, keep):
        self._ptr = ctypes.c_void_p(ptr)
        self.sizes = sizes
        self._keep = keep

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            load().sphc_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(0)

    def solve(self, bs, xs, tol=1e-8, nrhs=1, stream=None):
        """bs, xs: lists (one per system) of nrhs x n_e arrays.  Returns (status, iters, relres) with
        iters / relres of shape [nsys, nrhs]."""
        n = len(self.sizes)
        bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        it = np.zeros((n, nrhs), np.int32)
        rr = np.zeros((n, nrhs), np.float64)
        rc = load().sphc_solve_batched(self._ptr, bp, xp, nrhs, tol, _stream(stream), _ptr(it), _ptr(rr))
        if rc not in (SPHC_OK, -4, -5, -8):
            _check(rc)
        return rc, it, rr


def setup_batched(systems, opts=None, stream=None) -> Batch:
    """systems: list of (A, D, coords, sigma_edge) with A, D as for setup()."""
    n = len(systems)
    As = (sphc_csr * n)(*[make_csr(*s[0]) for s in systems])
    Ds = (sphc_csr * n)(*[make_csr(*s[1]) for s in systems])
    cs = (ctypes.c_void_p * n)(*[_ptr(s[2]) if len(s) > 2 else None for s in systems])
    ss = (ctypes.c_void_p * n)(*[_ptr(s[3]) if len(s) > 3 else None for s in systems])
    o = opts if opts is not None else default_opts()
    out = ctypes.c_void_p()
    _check(load().sphc_setup_batched(n, As, Ds, cs, ss, ctypes.byref(o), _stream(stream), ctypes.byref(out)))
    return Batch(out.value, [s[0][0] for s in systems], systems)


def launch_count() -> int:
    return int(load().sphc_launch_count())


def memory_usage(device: int = 0):
    """(used, reserved) bytes of the library's memory pool on `device`."""
    u, r = ctypes.c_int64(), ctypes.c_int64()
    _check(load().sphc_memory_usage(int(device), ctypes.byref(u), ctypes.byref(r)))
    return u.value, r.value


def grid_barrier_check(extra_arrivals: int, polls: int = 0, stream=None) -> bool:
    """Run the persistent sweep's grid barrier three times on the current device, counting
    `extra_arrivals` arrivals more than there are thread blocks; True when the waits gave up
    (always, for extra_arrivals > 0)."""
    t = ctypes.c_int()
    _check(load().sphc_grid_barrier_check(int(extra_arrivals), int(polls), ctypes.byref(t), _stream(stream)))
    return bool(t.value)


def trim_memory(device: int = 0, keep_bytes: int = 0) -> int:
    """Return the device memory the library caches beyond keep_bytes to the driver."""
    return int(load().sphc_trim_memory(int(device), int(keep_bytes)))


def setup(A, D, coords=None, sigma_edge=None, opts=None, stream=None) -> Handle:
    """A, D: (nrows, ncols, rowptr, col, val) with host (numpy) or device (torch) arrays."""
    Ac = make_csr(*A)
    Dc = make_csr(*D)
    h = ctypes.c_void_p()
    o = opts if opts is not None else default_opts()
    _check(load().sphc_setup(ctypes.byref(Ac), ctypes.byref(Dc), _ptr(coords), _ptr(sigma_edge), ctypes.byref(o),
                             _stream(stream), ctypes.byref(h)))
    return Handle(h.value)
