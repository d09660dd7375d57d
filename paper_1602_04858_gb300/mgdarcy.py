"""Thin ctypes binding of libmgdarcy.so (include/mgdarcy.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays may be torch tensors (CUDA or CPU) or NumPy arrays (host); FP64,
contiguous.  If the library is missing the import fails with a message that
says how to build it: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgdarcy.so")

MG_OK = 0
STATUS = {0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_OOM", 3: "MG_ERR_CUDA", 4: "MG_ERR_NOT_CONVERGED",
          5: "MG_ERR_BREAKDOWN", 6: "MG_ERR_DEVICE_TIMEOUT", 7: "MG_ERR_UNSUPPORTED"}
PREC = {"fp64": 0, "fp32": 1, "fp32_bf16inv": 2}

API = [
    "mg_setup", "mg_destroy", "mg_sizes", "mg_apply", "mg_vcycle", "mg_solve", "mg_smooth", "mg_colour_pass",
    "mg_level_load", "mg_level_store", "mg_restrict", "mg_prolong_add", "mg_coarse_solve", "mg_patch_info",
    "mg_kernel_launches", "mg_status_string", "mg_last_error", "mg_residual_norm", "mg_residual_norm_noalloc",
]


class mg_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_coarse", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("degree", ctypes.c_int), ("mu", ctypes.c_double), ("c", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("m_fine", ctypes.c_int), ("variable_cycle", ctypes.c_int),
                ("coarse_avg", ctypes.c_int), ("dense_level", ctypes.c_int)]


class mg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("initial_rel_residual", ctypes.c_double), ("removed_flux", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_1602_04858_gb300.build` "
                          "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.mg_setup.argtypes = [ctypes.POINTER(mg_problem), vp, ctypes.POINTER(vp)]
    lib.mg_destroy.argtypes = [vp]
    lib.mg_destroy.restype = None
    lib.mg_sizes.argtypes = [vp, i, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.mg_apply.argtypes = [vp, i, vp, vp]
    lib.mg_vcycle.argtypes = [vp, vp, vp]
    lib.mg_solve.argtypes = [vp, vp, vp, vp, i, d, i, i, ctypes.POINTER(mg_stats)]
    lib.mg_smooth.argtypes = [vp, i, vp, vp, i]
    lib.mg_colour_pass.argtypes = [vp, i, i]
    lib.mg_level_load.argtypes = [vp, i, vp, vp]
    lib.mg_level_store.argtypes = [vp, i, vp]
    lib.mg_restrict.argtypes = [vp, i, vp, vp]
    lib.mg_prolong_add.argtypes = [vp, i, vp, vp]
    lib.mg_coarse_solve.argtypes = [vp, vp, vp]
    lib.mg_patch_info.argtypes = [vp, i, i, ctypes.POINTER(i64), ctypes.POINTER(i)]
    lib.mg_residual_norm.argtypes = [vp, i, vp, vp, vp, vp]
    lib.mg_residual_norm_noalloc.argtypes = [i, i, i, d, vp, vp, vp, vp, vp]
    lib.mg_kernel_launches.argtypes = [vp]
    lib.mg_kernel_launches.restype = i64
    lib.mg_status_string.argtypes = [i]
    lib.mg_status_string.restype = ctypes.c_char_p
    lib.mg_last_error.argtypes = []
    lib.mg_last_error.restype = ctypes.c_char_p
    for name in API:
        if name not in ("mg_destroy", "mg_kernel_launches", "mg_status_string", "mg_last_error"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a contiguous FP64 torch tensor or NumPy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be contiguous float64")
        return a.ctypes.data
    if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    return a.data_ptr()


def _check(status):
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode())


def _stream_ptr(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def residual_norm_noalloc(dim, degree, n, mu, c, x, b, norm, stream=None):
    """mg_residual_norm_noalloc: ||b - A x||_2 into the device scalar `norm`,
    for callers that cannot allocate device memory (no handle needed)."""
    _check(load().mg_residual_norm_noalloc(int(dim), int(degree), int(n), float(mu), _ptr(c), _ptr(x), _ptr(b),
                                           _ptr(norm), ctypes.c_void_p(_stream_ptr(stream))))


class Multigrid:
    """A level hierarchy on the current CUDA device (mg_setup)."""

    def __init__(self, dim, n_coarse, n_levels, degree, mu, c, precision="fp64", m_fine=2,
                 variable_cycle=True, coarse_avg=0, dense_level=-1, stream=None):
        lib = load()
        self._keep = c if not isinstance(c, np.ndarray) else np.ascontiguousarray(c, dtype=np.float64)
        prob = mg_problem(dim, n_coarse, n_levels, degree, float(mu), _ptr(self._keep),
                          PREC[precision] if isinstance(precision, str) else int(precision), int(m_fine),
                          1 if variable_cycle else 0, int(coarse_avg), int(dense_level))
        h = ctypes.c_void_p()
        _check(lib.mg_setup(ctypes.byref(prob), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self.h = h
        self.dim, self.degree, self.n_levels = dim, degree, n_levels
        self.n_coarse = n_coarse
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            load().mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self, level=-1):
        nu, np_ = ctypes.c_int64(), ctypes.c_int64()
        _check(load().mg_sizes(self.h, level, ctypes.byref(nu), ctypes.byref(np_)))
        return nu.value, np_.value

    def ndof(self, level=-1):
        nu, np_ = self.sizes(level)
        return nu + np_

    def apply(self, x, y, level=-1):
        _check(load().mg_apply(self.h, level, _ptr(x), _ptr(y)))

    def vcycle(self, r, z):
        _check(load().mg_vcycle(self.h, _ptr(r), _ptr(z)))

    def solve(self, f, g, x, use_x0=False, tol=1e-8, maxit=200, restart=0, check=True):
        st = mg_stats()
        status = load().mg_solve(self.h, _ptr(f), _ptr(g), _ptr(x), 1 if use_x0 else 0, float(tol), int(maxit),
                                 int(restart), ctypes.byref(st))
        if check:
            _check(status)
        return st, status

    def smooth(self, level, x, b, steps=1):
        _check(load().mg_smooth(self.h, level, _ptr(x), _ptr(b), steps))

    def level_load(self, level, x, b):
        _check(load().mg_level_load(self.h, level, _ptr(x), _ptr(b)))

    def level_store(self, level, x):
        _check(load().mg_level_store(self.h, level, _ptr(x)))

    def colour_pass(self, level, colour):
        _check(load().mg_colour_pass(self.h, level, colour))

    def restrict(self, level, r_fine, b_coarse):
        _check(load().mg_restrict(self.h, level, _ptr(r_fine), _ptr(b_coarse)))

    def prolong_add(self, level, x_coarse, x_fine):
        _check(load().mg_prolong_add(self.h, level, _ptr(x_coarse), _ptr(x_fine)))

    def coarse_solve(self, b, x):
        _check(load().mg_coarse_solve(self.h, _ptr(b), _ptr(x)))

    def patch_info(self, level, colour):
        cnt, nv = ctypes.c_int64(), ctypes.c_int()
        _check(load().mg_patch_info(self.h, level, colour, ctypes.byref(cnt), ctypes.byref(nv)))
        return cnt.value, nv.value

    def residual_norm(self, x, b, r=None, level=-1):
        """||b - A x||_2 (FP64) of device tensors; also stores r = b - A x if given."""
        out = ctypes.c_double()
        _check(load().mg_residual_norm(self.h, level, _ptr(x), _ptr(b), _ptr(r), ctypes.addressof(out)))
        return out.value

    def launches(self):
        return load().mg_kernel_launches(self.h)
