"""The C interface: the library builds, loads and exports every declared entry point.

These tests need no GPU: they check the symbols and the argument validation
that happens on the host before any device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1602_04858_gb300 import build as builder
from paper_1602_04858_gb300 import mgdarcy

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mgdarcy.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    builder.build()
    return mgdarcy.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "mg_setup" in names and "mg_solve" in names and "mg_vcycle" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert sorted(mgdarcy.API) == declared_functions()


def _setup(lib, **kw):
    c = kw.pop("c", np.ones((8, 8)))
    p = mgdarcy.mg_problem(kw.get("dim", 2), kw.get("n_coarse", 2), kw.get("n_levels", 3), kw.get("degree", 0),
                           kw.get("mu", 1.0), c.ctypes.data if c is not None else None, kw.get("precision", 0),
                           kw.get("m_fine", 2), 1, kw.get("coarse_avg", 0), kw.get("dense_level", 0),
                           kw.get("pass_kernel", 0), kw.get("additive", 0.0))
    h = ctypes.c_void_p()
    return lib.mg_setup(ctypes.byref(p), None, ctypes.byref(h))


@pytest.mark.parametrize("kw,status", [
    (dict(dim=4), 1),
    (dict(degree=3), 7),
    (dict(dim=3, degree=2, c=np.ones((8, 8, 8))), 7),
    (dict(dim=3, degree=1, c=np.ones((8, 8, 8))), 7),
    (dict(n_coarse=1), 1),
    (dict(mu=-1.0), 1),
    (dict(mu=float("nan")), 1),
    (dict(precision=5), 1),
    (dict(m_fine=0), 1),
    (dict(c=np.full((8, 8), -1.0)), 1),
    (dict(c=np.full((8, 8), np.inf)), 1),
    (dict(c=None), 1),
    (dict(dense_level=3), 1),
    (dict(dense_level=-2), 1),
    (dict(pass_kernel=11), 1),
    (dict(pass_kernel=-1), 1),
    (dict(dim=3, n_coarse=2, n_levels=10, c=np.ones((2, 2, 2))), 1),   # 4.3e9 dofs: rejected before c is read
    (dict(additive=-0.1), 1),
    (dict(additive=1.5), 1),
    (dict(additive=float("nan")), 1),
])
def test_setup_rejects_bad_arguments(lib, kw, status):
    assert _setup(lib, **kw) == status
    assert lib.mg_last_error().decode()


def test_status_strings(lib):
    for s in range(8):
        assert lib.mg_status_string(s).decode()


def test_status_entry_points_reject_null_handles(lib):
    assert lib.mg_sync(None) == 1
    assert lib.mg_sync_batch(None) == 1
    assert lib.mg_set_wait_limit(None, 1.0) == 1
    assert lib.mg_batch_set_wait_limit(None, 1.0) == 1
    assert lib.mg_set_residual_history(None, None, 0) == 1


def test_injected_allocation_failure_is_reported_as_oom(lib):
    """The failure-injection hook refuses the first device allocation of the
    next set-up before any CUDA call is made, so this runs without a GPU: the
    set-up returns MG_ERR_OOM and frees what it had; the hook is one-shot."""
    lib.mg_inject_alloc_failure(0)
    try:
        assert _setup(lib, dense_level=0) == 2
        assert "refused" in lib.mg_last_error().decode()
    finally:
        lib.mg_inject_alloc_failure(-1)
    # the next set-up reaches the device (which this machine may lack): no second refusal
    status = _setup(lib, dense_level=0)
    assert status != 2 or "refused" not in lib.mg_last_error().decode()


def test_escalate_window_is_validated(lib):
    c = np.ones((8, 8))
    p = mgdarcy.mg_problem(2, 2, 3, 0, 1.0, c.ctypes.data, 1, 2, 1, 0, 0, 0, 0.0, 1000000)
    h = ctypes.c_void_p()
    assert lib.mg_setup(ctypes.byref(p), None, ctypes.byref(h)) == 1


def test_binding_refuses_short_buffers(lib):
    """The C interface takes bare pointers, so the binding checks each
    buffer's length against what the call reads or writes before calling:
    a coefficient array with fewer values than finest cells is refused before
    any set-up runs (no GPU needed), for a single problem and in a batch."""
    with pytest.raises(ValueError, match="c "):
        mgdarcy.Multigrid(2, 2, 3, 0, 1.0, np.ones(63))
    with pytest.raises(ValueError, match="problem 1"):
        mgdarcy.Batch([dict(dim=2, n_coarse=2, n_levels=3, degree=0, mu=1.0, c=np.ones(64)),
                       dict(dim=3, n_coarse=2, n_levels=2, degree=0, mu=0.0, c=np.ones(63))])
    mgdarcy._need(np.ones(5), 5, "x")
    mgdarcy._need(None, 5, "r")
    with pytest.raises(ValueError, match="x has 4 entries"):
        mgdarcy._need(np.ones(4), 5, "x")


C_CALLER = r"""
#include "mgdarcy.h"
#include <stdio.h>
#include <string.h>
int main(void) {
  mg_problem p;
  mg_handle* h = 0;
  memset(&p, 0, sizeof p);
  p.dim = 4;
  mg_status s = mg_setup(&p, 0, &h);
  printf("%d|%s|%s\n", (int)s, mg_status_string(s), mg_last_error());
  mg_destroy(0);
  mg_destroy_batch(0);
  return (s == MG_ERR_INVALID_ARG && h == 0) ? 0 : 1;
}
"""


def test_plain_c_caller(lib, tmp_path):
    """The boundary is a C interface: the header compiles as strict C99 and a
    C program links against the library and gets an argument error back as a
    status, with no C++ runtime of its own and no GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.dirname(HEADER)
    libdir = os.path.dirname(mgdarcy.LIB_PATH)
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                    "-L", libdir, "-lmgdarcy", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    status, text, msg = out.stdout.strip().split("|")
    assert int(status) == 1 and text == "invalid argument" and "dim" in msg


def test_binding_checks_every_buffer_length(lib):
    """Every call of the binding that passes vectors checks their lengths
    against the level sizes before calling the library: a buffer one entry
    short raises ValueError, and the right lengths reach the C function (which
    here refuses the null handle with its own status).  Host only: the handle
    is a stand-in with the sizes of a 2x2 -> 8x8 RT_0 hierarchy."""
    G = object.__new__(mgdarcy.Multigrid)
    G.h = None
    G.dim, G.degree, G.n_levels, G.n_coarse, G.nrhs = 2, 0, 3, 2, 1
    G._nd = {0: (12, 4), 1: (40, 16), 2: (144, 64), -1: (144, 64)}
    ok = {j: np.zeros(sum(v)) for j, v in G._nd.items()}
    short = {j: np.zeros(sum(v) - 1) for j, v in G._nd.items()}
    f_ok, f_short = np.zeros(2 * 64), np.zeros(2 * 64 - 1)
    calls = {
        "apply": (lambda v: G.apply(v[-1], ok[-1])),
        "vcycle": (lambda v: G.vcycle(ok[-1], v[-1])),
        "solve": (lambda v: G.solve(np.zeros(144), np.zeros(64), v[-1])),
        "smooth": (lambda v: G.smooth(1, v[1], ok[1])),
        "level_load": (lambda v: G.level_load(1, ok[1], v[1])),
        "level_store": (lambda v: G.level_store(2, v[2])),
        "restrict": (lambda v: G.restrict(2, ok[2], v[1])),
        "prolong_add": (lambda v: G.prolong_add(2, v[1], ok[2])),
        "coarse_solve": (lambda v: G.coarse_solve(v[0], ok[0])),
        "residual_norm": (lambda v: G.residual_norm(ok[-1], v[-1])),
        "load_vector": (lambda v: G.load_vector(f_ok, None, v[-1])),
    }
    for name, call in calls.items():
        with pytest.raises(ValueError):
            call(short)
        with pytest.raises(mgdarcy.MGError) as e:    # the lengths pass; the library refuses the null handle
            call(ok)
        assert e.value.status == 1, name
    with pytest.raises(ValueError):
        G.load_vector(f_short, None, ok[-1])
    with pytest.raises(ValueError):
        G.solve(np.zeros(143), np.zeros(64), ok[-1])
