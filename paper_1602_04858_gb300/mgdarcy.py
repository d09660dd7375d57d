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
    "mg_level_pass_kernel", "mg_dense_level", "mg_level_rhs_group", "mg_level_row_threads", "mg_kernel_launches", "mg_status_string", "mg_last_error", "mg_residual_norm", "mg_residual_norm_noalloc",
    "mg_setup_batch", "mg_destroy_batch", "mg_batch_layout", "mg_vcycle_batch", "mg_solve_batch",
    "mg_batch_kernel_launches", "mg_batch_level_choice", "mg_load_vector",
    "mg_cnn_create", "mg_cnn_destroy", "mg_cnn_param_count", "mg_cnn_get_params", "mg_cnn_set_params",
    "mg_cnn_set_normalisation", "mg_cnn_features", "mg_cnn_targets", "mg_cnn_forward", "mg_cnn_gradients",
    "mg_cnn_train_step", "mg_cnn_guess", "mg_pass_tables_check",
    "mg_sync", "mg_set_wait_limit", "mg_set_block_limit", "mg_set_residual_history", "mg_inject_alloc_failure", "mg_sync_batch",
    "mg_batch_set_wait_limit", "mg_patch_nnz", "mg_measure_fma_peak", "mg_measure_sync_cost", "mg_time_passes", "mg_boundary_patch_info",
]


class mg_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_coarse", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("degree", ctypes.c_int), ("mu", ctypes.c_double), ("c", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("m_fine", ctypes.c_int), ("variable_cycle", ctypes.c_int),
                ("coarse_avg", ctypes.c_int), ("dense_level", ctypes.c_int), ("pass_kernel", ctypes.c_int),
                ("additive", ctypes.c_double), ("escalate_window", ctypes.c_int), ("boundary_patches", ctypes.c_int),
                ("nrhs", ctypes.c_int)]


class mg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("initial_rel_residual", ctypes.c_double), ("removed_flux", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("escalated_at", ctypes.c_int)]


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
    lib.mg_level_pass_kernel.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.mg_level_rhs_group.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.mg_dense_level.argtypes = [vp, ctypes.POINTER(i)]
    lib.mg_level_row_threads.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.mg_residual_norm.argtypes = [vp, i, vp, vp, vp, vp]
    lib.mg_residual_norm_noalloc.argtypes = [i, i, i, d, vp, vp, vp, vp, vp]
    lib.mg_setup_batch.argtypes = [ctypes.POINTER(mg_problem), i, i, vp, ctypes.POINTER(vp)]
    lib.mg_destroy_batch.argtypes = [vp]
    lib.mg_destroy_batch.restype = None
    lib.mg_batch_layout.argtypes = [vp, i, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.mg_vcycle_batch.argtypes = [vp, vp, vp]
    lib.mg_solve_batch.argtypes = [vp, vp, vp, i, d, i, i, ctypes.POINTER(mg_stats)]
    lib.mg_batch_kernel_launches.argtypes = [vp]
    lib.mg_batch_level_choice.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.mg_batch_kernel_launches.restype = i64
    lib.mg_load_vector.argtypes = [vp, i, vp, vp, vp]
    f = ctypes.c_float
    lib.mg_cnn_create.argtypes = [i, i, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    lib.mg_cnn_destroy.argtypes = [vp]
    lib.mg_cnn_destroy.restype = None
    lib.mg_cnn_param_count.argtypes = [vp]
    lib.mg_cnn_param_count.restype = i64
    lib.mg_cnn_get_params.argtypes = [vp, vp]
    lib.mg_cnn_set_params.argtypes = [vp, vp]
    lib.mg_cnn_set_normalisation.argtypes = [vp, vp]
    lib.mg_cnn_features.argtypes = [vp, vp, vp, vp]
    lib.mg_cnn_targets.argtypes = [vp, vp, vp]
    lib.mg_cnn_forward.argtypes = [vp, vp, i, vp]
    lib.mg_cnn_gradients.argtypes = [vp, vp, vp, i, ctypes.POINTER(f), vp]
    lib.mg_cnn_train_step.argtypes = [vp, vp, vp, i, f, ctypes.POINTER(f)]
    lib.mg_cnn_guess.argtypes = [vp, vp, vp, vp]
    lib.mg_pass_tables_check.argtypes = [i, i, i, i, d, ctypes.c_char_p, i]
    lib.mg_sync.argtypes = [vp]
    lib.mg_set_wait_limit.argtypes = [vp, d]
    lib.mg_set_block_limit.argtypes = [vp, i]
    lib.mg_set_residual_history.argtypes = [vp, vp, i]
    lib.mg_inject_alloc_failure.argtypes = [i64]
    lib.mg_inject_alloc_failure.restype = None
    lib.mg_sync_batch.argtypes = [vp]
    lib.mg_batch_set_wait_limit.argtypes = [vp, d]
    lib.mg_patch_nnz.argtypes = [vp, i, ctypes.POINTER(i64)]
    lib.mg_time_passes.argtypes = [vp, i, i, ctypes.POINTER(d)]
    lib.mg_boundary_patch_info.argtypes = [vp, i, i, ctypes.POINTER(i64), ctypes.POINTER(i)]
    lib.mg_measure_fma_peak.argtypes = [i, ctypes.POINTER(d), vp]
    lib.mg_measure_sync_cost.argtypes = [i, i, ctypes.POINTER(d), vp]
    lib.mg_kernel_launches.argtypes = [vp]
    lib.mg_kernel_launches.restype = i64
    lib.mg_status_string.argtypes = [i]
    lib.mg_status_string.restype = ctypes.c_char_p
    lib.mg_last_error.argtypes = []
    lib.mg_last_error.restype = ctypes.c_char_p
    for name in API:
        if name not in ("mg_destroy", "mg_kernel_launches", "mg_status_string", "mg_last_error",
                        "mg_destroy_batch", "mg_batch_kernel_launches", "mg_cnn_destroy", "mg_cnn_param_count",
                        "mg_inject_alloc_failure"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def pass_tables_check(dim, degree, precision, n, mu):
    """mg_pass_tables_check: host check of the colour-pass tables of an n^dim
    level (no GPU).  Returns (code, message); code 0 means every check held."""
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    buf = ctypes.create_string_buffer(512)
    r = load().mg_pass_tables_check(int(dim), int(degree), prec, int(n), float(mu), buf, len(buf))
    return r, buf.value.decode()


def _ptr(a, dtype="float64"):
    """Raw pointer of a contiguous torch tensor or NumPy array of the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"arrays must be contiguous {dtype}")
        return a.ctypes.data
    if str(a.dtype) != "torch." + dtype or not a.is_contiguous():
        raise TypeError(f"tensors must be contiguous {dtype}")
    return a.data_ptr()


def _need(a, count, what):
    """The C interface takes bare pointers: refuse a buffer shorter than the
    entries the call reads or writes (None passes, for optional arguments)."""
    if a is None:
        return
    n = a.size if isinstance(a, np.ndarray) else a.numel()
    if n < count:
        raise ValueError(f"{what} has {n} entries, the call needs {count}")


def _check(status):
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode())


def _stream_ptr(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def inject_alloc_failure(after):
    """mg_inject_alloc_failure: the library's allocation after the next `after`
    ones is refused with MG_ERR_OOM (once); after < 0 cancels.  For tests."""
    load().mg_inject_alloc_failure(int(after))


def measure_fma_peak(kind, stream=None):
    """mg_measure_fma_peak: measured FMA throughput in TFLOP/s; kind "fp64", "fp32" or "fp32x2"."""
    k = {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind]
    out = ctypes.c_double()
    _check(load().mg_measure_fma_peak(k, ctypes.byref(out), ctypes.c_void_p(_stream_ptr(stream))))
    return out.value


def measure_sync_cost(kind, blocks, stream=None):
    """mg_measure_sync_cost: microseconds per grid-wide ordering point on `blocks`
    blocks; kind "grid_barrier" (one cooperative launch) or "dependent_launch"."""
    k = {"grid_barrier": 0, "dependent_launch": 1}[kind]
    out = ctypes.c_double()
    _check(load().mg_measure_sync_cost(k, int(blocks), ctypes.byref(out), ctypes.c_void_p(_stream_ptr(stream))))
    return out.value


def residual_norm_noalloc(dim, degree, n, mu, c, x, b, norm, stream=None):
    """mg_residual_norm_noalloc: ||b - A x||_2 into the device scalar `norm`,
    for callers that cannot allocate device memory (no handle needed)."""
    _check(load().mg_residual_norm_noalloc(int(dim), int(degree), int(n), float(mu), _ptr(c), _ptr(x), _ptr(b),
                                           _ptr(norm), ctypes.c_void_p(_stream_ptr(stream))))


class Multigrid:
    """A level hierarchy on the current CUDA device (mg_setup)."""

    def __init__(self, dim, n_coarse, n_levels, degree, mu, c, precision="fp64", m_fine=2,
                 variable_cycle=True, coarse_avg=0, dense_level=-1, pass_kernel=0, additive=0.0,
                 escalate_window=0, boundary_patches=False, nrhs=1, stream=None):
        lib = load()
        self._keep = c if not isinstance(c, np.ndarray) else np.ascontiguousarray(c, dtype=np.float64)
        _need(self._keep, (int(n_coarse) << (int(n_levels) - 1)) ** int(dim), "c (one value per finest cell)")
        prob = mg_problem(dim, n_coarse, n_levels, degree, float(mu), _ptr(self._keep),
                          PREC[precision] if isinstance(precision, str) else int(precision), int(m_fine),
                          1 if variable_cycle else 0, int(coarse_avg), int(dense_level), int(pass_kernel),
                          float(additive), int(escalate_window), 1 if boundary_patches else 0, int(nrhs))
        h = ctypes.c_void_p()
        _check(lib.mg_setup(ctypes.byref(prob), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self.h = h
        self.dim, self.degree, self.n_levels = dim, degree, n_levels
        self.n_coarse = n_coarse
        self.precision = precision
        self.nrhs = int(nrhs)
        self._nd = {}

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

    def _sizes(self, level):
        """mg_sizes of a level, cached (the argument checks of every call use it)."""
        if level not in self._nd:
            self._nd[level] = self.sizes(level)
        return self._nd[level]

    def _vec(self, level, *named):
        n = sum(self._sizes(level))
        for what, a in named:
            _need(a, n, what)

    def apply(self, x, y, level=-1):
        self._vec(level, ("x", x), ("y", y))
        _check(load().mg_apply(self.h, level, _ptr(x), _ptr(y)))

    def vcycle(self, r, z):
        n = sum(self._sizes(-1)) * max(1, self.nrhs)
        _need(r, n, "r")
        _need(z, n, "z")
        _check(load().mg_vcycle(self.h, _ptr(r), _ptr(z)))

    def solve(self, f, g, x, use_x0=False, tol=1e-8, maxit=200, restart=0, check=True, history=None):
        """mg_solve; history: None or a float64 NumPy array that receives the
        relative residual after each iteration (mg_set_residual_history)."""
        lib = load()
        nu, np_ = self._sizes(-1)
        _need(f, nu, "f")
        _need(g, np_, "g")
        _need(x, nu + np_, "x")
        st = mg_stats()
        if history is not None:
            _check(lib.mg_set_residual_history(self.h, _ptr(history), int(history.size)))
        try:
            status = lib.mg_solve(self.h, _ptr(f), _ptr(g), _ptr(x), 1 if use_x0 else 0, float(tol), int(maxit),
                                  int(restart), ctypes.byref(st))
        finally:
            if history is not None:
                lib.mg_set_residual_history(self.h, None, 0)
        if check:
            _check(status)
        return st, status

    def sync(self, check=True):
        """mg_sync: wait for the stream; MG_ERR_DEVICE_TIMEOUT if a device wait ran out."""
        status = load().mg_sync(self.h)
        if check:
            _check(status)
        return status

    def set_block_limit(self, blocks):
        """mg_set_block_limit: cap the grid of the persistent colour-pass kernels (0: no cap)."""
        _check(load().mg_set_block_limit(self.h, int(blocks)))

    def set_wait_limit(self, seconds):
        _check(load().mg_set_wait_limit(self.h, float(seconds)))

    def smooth(self, level, x, b, steps=1):
        self._vec(level, ("x", x), ("b", b))
        _check(load().mg_smooth(self.h, level, _ptr(x), _ptr(b), steps))

    def level_load(self, level, x, b):
        self._vec(level, ("x", x), ("b", b))
        _check(load().mg_level_load(self.h, level, _ptr(x), _ptr(b)))

    def level_store(self, level, x):
        self._vec(level, ("x", x))
        _check(load().mg_level_store(self.h, level, _ptr(x)))

    def colour_pass(self, level, colour):
        _check(load().mg_colour_pass(self.h, level, colour))

    def restrict(self, level, r_fine, b_coarse):
        self._vec(level, ("r_fine", r_fine))
        self._vec(level - 1, ("b_coarse", b_coarse))
        _check(load().mg_restrict(self.h, level, _ptr(r_fine), _ptr(b_coarse)))

    def prolong_add(self, level, x_coarse, x_fine):
        self._vec(level - 1, ("x_coarse", x_coarse))
        self._vec(level, ("x_fine", x_fine))
        _check(load().mg_prolong_add(self.h, level, _ptr(x_coarse), _ptr(x_fine)))

    def coarse_solve(self, b, x):
        self._vec(0, ("b", b), ("x", x))
        _check(load().mg_coarse_solve(self.h, _ptr(b), _ptr(x)))

    def patch_info(self, level, colour):
        cnt, nv = ctypes.c_int64(), ctypes.c_int()
        _check(load().mg_patch_info(self.h, level, colour, ctypes.byref(cnt), ctypes.byref(nv)))
        return cnt.value, nv.value

    def patch_nnz(self, level):
        """Nonzeros of the operator rows of one interior patch of a level (mg_patch_nnz)."""
        v = ctypes.c_int64()
        _check(load().mg_patch_nnz(self.h, level, ctypes.byref(v)))
        return v.value

    def boundary_patch_info(self, level, colour):
        """(count, largest size) of the boundary-vertex patches of a colour (mg_boundary_patch_info)."""
        cnt, nv = ctypes.c_int64(), ctypes.c_int()
        _check(load().mg_boundary_patch_info(self.h, level, colour, ctypes.byref(cnt), ctypes.byref(nv)))
        return cnt.value, nv.value

    def time_passes(self, level, kernel=0):
        """Microseconds per colour pass of a level (mg_time_passes); kernel 0: the level's own."""
        v = ctypes.c_double()
        _check(load().mg_time_passes(self.h, level, int(kernel), ctypes.byref(v)))
        return v.value

    def pass_kernel(self, level):
        """Colour-pass kernel of a level: 1 warp per patch, 2 block per patch, 3 persistent blocks."""
        k = ctypes.c_int()
        _check(load().mg_level_pass_kernel(self.h, level, ctypes.byref(k)))
        return k.value

    def dense_level(self):
        """Level whose sub-cycle setup folded into a dense matrix (mg_dense_level); 0: none."""
        v = ctypes.c_int()
        _check(load().mg_dense_level(self.h, ctypes.byref(v)))
        return v.value

    def row_threads(self, level):
        """Threads per patch row of the block kernel on a level (mg_level_row_threads): 4, 2 or 8."""
        t = ctypes.c_int()
        _check(load().mg_level_row_threads(self.h, level, ctypes.byref(t)))
        return t.value

    def rhs_group(self, level):
        """Right-hand sides sharing each patch-inverse load on a level (mg_level_rhs_group): 4 or 1."""
        g = ctypes.c_int()
        _check(load().mg_level_rhs_group(self.h, level, ctypes.byref(g)))
        return g.value

    def residual_norm(self, x, b, r=None, level=-1):
        """||b - A x||_2 (FP64) of device tensors; also stores r = b - A x if given."""
        self._vec(level, ("x", x), ("b", b), ("r", r))
        out = ctypes.c_double()
        _check(load().mg_residual_norm(self.h, level, _ptr(x), _ptr(b), _ptr(r), ctypes.addressof(out)))
        return out.value

    def load_vector(self, f, g, b, level=-1):
        """b = load vector of cellwise-constant f (dim x cells) and g (cells or None); device tensors."""
        cells = (int(self.n_coarse) << (level if level >= 0 else self.n_levels - 1)) ** int(self.dim)
        _need(f, self.dim * cells, "f")
        _need(g, cells, "g")
        self._vec(level, ("b", b))
        _check(load().mg_load_vector(self.h, level, _ptr(f), _ptr(g), _ptr(b)))

    def launches(self):
        return load().mg_kernel_launches(self.h)


class Batch:
    """Independent problems with nrhs right-hand sides each (mg_setup_batch).

    problems: list of dicts with keys dim, n_coarse, n_levels, degree, mu, c
    (and optionally precision, m_fine, variable_cycle, coarse_avg, dense_level, pass_kernel, additive).
    """

    def __init__(self, problems, nrhs=4, stream=None):
        lib = load()
        arr = (mg_problem * len(problems))()
        self._keep = []
        for k, p in enumerate(problems):
            c = p["c"]
            _need(c, (int(p["n_coarse"]) << (int(p["n_levels"]) - 1)) ** int(p["dim"]),
                  f"problem {k}: c (one value per finest cell)")
            self._keep.append(c)
            prec = p.get("precision", "fp32")
            arr[k] = mg_problem(p["dim"], p["n_coarse"], p["n_levels"], p["degree"], float(p["mu"]), _ptr(c),
                                PREC[prec] if isinstance(prec, str) else int(prec), int(p.get("m_fine", 2)),
                                1 if p.get("variable_cycle", True) else 0, int(p.get("coarse_avg", 0)),
                                int(p.get("dense_level", -1)), int(p.get("pass_kernel", 0)),
                                float(p.get("additive", 0.0)), int(p.get("escalate_window", 0)),
                                1 if p.get("boundary_patches", False) else 0)
        h = ctypes.c_void_p()
        _check(lib.mg_setup_batch(arr, len(problems), int(nrhs), ctypes.c_void_p(_stream_ptr(stream)),
                                  ctypes.byref(h)))
        self.h = h
        self.nprob, self.nrhs = len(problems), nrhs

    def close(self):
        if getattr(self, "h", None):
            load().mg_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self, p):
        nd, off, tot = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().mg_batch_layout(self.h, p, ctypes.byref(nd), ctypes.byref(off), ctypes.byref(tot)))
        return nd.value, off.value, tot.value

    def total(self):
        return self.layout(0)[2]

    def level_choice(self, p, level):
        """(kernel, right-hand-side grouping, threads per patch row) of problem p's
        colour passes on a level (mg_batch_level_choice)."""
        k, g, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().mg_batch_level_choice(self.h, p, level, ctypes.byref(k), ctypes.byref(g), ctypes.byref(t)))
        return k.value, g.value, t.value

    def vcycle(self, r, z):
        n = self.total()
        _need(r, n, "r")
        _need(z, n, "z")
        _check(load().mg_vcycle_batch(self.h, _ptr(r), _ptr(z)))

    def solve(self, rhs, x, use_x0=False, tol=1e-8, maxit=200, restart=20, check=True):
        n = self.total()
        _need(rhs, n, "rhs")
        _need(x, n, "x")
        st = (mg_stats * (self.nprob * self.nrhs))()
        status = load().mg_solve_batch(self.h, _ptr(rhs), _ptr(x), 1 if use_x0 else 0, float(tol), int(maxit),
                                       int(restart), st)
        if check:
            _check(status)
        return list(st), status

    def launches(self):
        return load().mg_batch_kernel_launches(self.h)

    def sync(self, check=True):
        status = load().mg_sync_batch(self.h)
        if check:
            _check(status)
        return status

    def set_wait_limit(self, seconds):
        _check(load().mg_batch_set_wait_limit(self.h, float(seconds)))


class CNN:
    """The learned-initial-guess network (mg_cnn_*); n x n RT_0 cell grids."""

    def __init__(self, n, max_batch=16, seed=0, stream=None):
        h = ctypes.c_void_p()
        _check(load().mg_cnn_create(int(n), int(max_batch), int(seed), ctypes.c_void_p(_stream_ptr(stream)),
                                    ctypes.byref(h)))
        self.h, self.n = h, n

    def close(self):
        if getattr(self, "h", None):
            load().mg_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def param_count(self):
        return load().mg_cnn_param_count(self.h)

    def get_params(self):
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(load().mg_cnn_get_params(self.h, _ptr(out, "float32")))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().mg_cnn_set_params(self.h, _ptr(p, "float32")))

    def set_normalisation(self, in_mean, in_std, out_mean, out_std):
        v = np.ascontiguousarray(np.concatenate([in_mean, in_std, out_mean, out_std]), dtype=np.float32)
        _check(load().mg_cnn_set_normalisation(self.h, _ptr(v, "float32")))

    def features(self, c, f, out):
        _check(load().mg_cnn_features(self.h, _ptr(c), _ptr(f), _ptr(out, "float32")))

    def targets(self, x, out):
        _check(load().mg_cnn_targets(self.h, _ptr(x), _ptr(out, "float32")))

    def forward(self, inp, batch, out):
        _check(load().mg_cnn_forward(self.h, _ptr(inp, "float32"), int(batch), _ptr(out, "float32")))

    def gradients(self, inp, target, batch):
        loss = ctypes.c_float()
        g = np.zeros(self.param_count(), dtype=np.float32)
        _check(load().mg_cnn_gradients(self.h, _ptr(inp, "float32"), _ptr(target, "float32"), int(batch),
                                       ctypes.byref(loss), _ptr(g, "float32")))
        return loss.value, g

    def train_step(self, inp, target, batch, lr):
        loss = ctypes.c_float()
        _check(load().mg_cnn_train_step(self.h, _ptr(inp, "float32"), _ptr(target, "float32"), int(batch),
                                        ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value

    def guess(self, c, f, x0):
        _check(load().mg_cnn_guess(self.h, _ptr(c), _ptr(f), _ptr(x0)))
