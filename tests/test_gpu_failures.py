"""Failure detection through the C interface, in forms that fault, trap or hang
no GPU: device-side waits made to run out by a zero wait limit (the kernels
record the timeout, let their own copies land and return early), GMRES
stopped at maxit, device allocations refused by the library's
failure-injection hook (in set-up, in a solve's workspace and in its
enlargement), host pointers and aliased buffers refused before any kernel
runs, and a zero right-hand side.  After each failure the handle (or a new
one) must work normally again.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import inputs, mgdarcy  # noqa: E402

TIMEOUT = 6
NOT_CONVERGED = 4
OOM = 2


def make(precision="fp32", n0=4, levels=4, **kw):
    c = inputs.channel_c(n0 * 2 ** (levels - 1), 4, 2)
    return mgdarcy.Multigrid(2, n0, levels, 1, 0.01, torch.as_tensor(c, device="cuda"), precision=precision, **kw)


def load(G, seed=3):
    """Load vector of a random cellwise body force (no divergence source)."""
    nu, npr = G.sizes()
    n = int(round((G.sizes()[1]) ** 0.5)) // (G.degree + 1)
    f = torch.as_tensor(np.random.default_rng(seed).standard_normal((2, n * n)), device="cuda")
    b = torch.zeros(nu + npr, dtype=torch.float64, device="cuda")
    G.load_vector(f, None, b)
    return b[:nu].contiguous(), b[nu:].contiguous()


@pytest.mark.parametrize("pass_kernel", [1, 2, 3])
def test_timeout_in_solve_is_reported_and_cleared(pass_kernel):
    G = make(pass_kernel=pass_kernel)
    f, g = load(G)
    n = G.ndof()
    G.set_wait_limit(0.0)          # every device-side wait runs out at once
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, status = G.solve(f, g, x, tol=1e-8, maxit=5, check=False)
    assert status == TIMEOUT
    torch.cuda.synchronize()       # the context is intact
    G.set_wait_limit(2.0)
    x1 = torch.zeros_like(x)
    st1, status1 = G.solve(f, g, x1, tol=1e-10, maxit=200, check=False)
    assert status1 == 0 and st1.converged
    ref = make(pass_kernel=pass_kernel)
    x2 = torch.zeros_like(x)
    st2, _ = ref.solve(f, g, x2, tol=1e-10, maxit=200)
    assert st1.iterations == st2.iterations
    assert torch.max(torch.abs(x1 - x2)).item() <= 1e-12 * torch.max(torch.abs(x2)).item()


def test_timeout_in_async_vcycle_is_reported_by_sync():
    G = make(precision="fp64")
    n = G.ndof()
    r = torch.as_tensor(np.random.default_rng(4).standard_normal(n), device="cuda")
    z0 = torch.zeros_like(r)
    G.vcycle(r, z0)
    assert G.sync(check=False) == 0
    G.set_wait_limit(0.0)
    z = torch.zeros_like(r)
    G.vcycle(r, z)
    assert G.sync(check=False) == TIMEOUT
    assert G.sync(check=False) == 0        # reading the word cleared it
    G.set_wait_limit(2.0)
    G.vcycle(r, z)
    assert G.sync(check=False) == 0
    assert torch.equal(z, z0)


def test_timeout_in_batched_solve_is_reported():
    probs = []
    for i, n in enumerate((16, 16, 32)):
        c = inputs.lognormal_c(n, 2, 1.0, 2.0, 50 + i)
        probs.append(dict(dim=2, n_coarse=4, n_levels=int(np.log2(n // 4)) + 1, degree=1, mu=0.01,
                          c=torch.as_tensor(c, device="cuda"), precision="fp32"))
    B = mgdarcy.Batch(probs, nrhs=2)
    total = B.total()
    rhs = torch.zeros(total, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    for p, pr in enumerate(probs):
        nd, off, _ = B.layout(p)
        n = pr["c"].shape[0]
        G = mgdarcy.Multigrid(2, 4, pr["n_levels"], 1, 0.01, pr["c"], precision="fp32")
        nu, _ = G.sizes()
        for rr in range(2):
            f = torch.as_tensor(rng.standard_normal((2, n * n)), device="cuda")
            b = torch.zeros(nd, dtype=torch.float64, device="cuda")
            G.load_vector(f, None, b)
            rhs[off + rr * nd: off + (rr + 1) * nd] = b
        del G
    x = torch.zeros_like(rhs)
    B.set_wait_limit(0.0)
    _, status = B.solve(rhs, x, tol=1e-8, maxit=4, restart=4, check=False)
    assert status == TIMEOUT
    B.set_wait_limit(0.0)
    B.vcycle(rhs, x)
    assert B.sync(check=False) == TIMEOUT
    B.set_wait_limit(2.0)
    x = torch.zeros_like(rhs)
    stats, status = B.solve(rhs, x, tol=1e-8, maxit=100, restart=20, check=False)
    assert status == 0 and all(s.converged for s in stats)


def test_maxit_gives_not_converged():
    G = make()
    f, g = load(G)
    x = torch.zeros(G.ndof(), dtype=torch.float64, device="cuda")
    st, status = G.solve(f, g, x, tol=1e-12, maxit=2, check=False)
    assert status == NOT_CONVERGED
    assert st.iterations == 2 and not st.converged and st.rel_residual < 1.0


def test_zero_rhs_converges_at_once():
    G = make()
    nu, npr = G.sizes()
    f = torch.zeros(nu, dtype=torch.float64, device="cuda")
    g = torch.zeros(npr, dtype=torch.float64, device="cuda")
    x = torch.full((nu + npr,), 7.0, dtype=torch.float64, device="cuda")
    st, status = G.solve(f, g, x, tol=1e-8, maxit=10)
    assert status == 0 and st.converged and st.iterations == 0
    assert torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("after", [0, 3, 17, 60])
def test_refused_allocation_gives_oom_and_frees_everything(after):
    G = make(levels=5)                          # every kernel of the set-up loaded once
    del G
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    mgdarcy.inject_alloc_failure(after)
    try:
        with pytest.raises(mgdarcy.MGError) as ei:
            make(levels=5)
        assert ei.value.status == OOM
    finally:
        mgdarcy.inject_alloc_failure(-1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= 4 << 20      # nothing of the failed set-up is left behind
    G = make(levels=5)                          # the library works normally afterwards
    f, g = load(G)
    x = torch.zeros(G.ndof(), dtype=torch.float64, device="cuda")
    st, _ = G.solve(f, g, x, tol=1e-8, maxit=100)
    assert st.converged


def test_refused_allocation_in_solve_leaves_handle_usable():
    G = make()
    f, g = load(G)
    x = torch.zeros(G.ndof(), dtype=torch.float64, device="cuda")
    mgdarcy.inject_alloc_failure(0)            # the Krylov workspace of the first solve
    try:
        st, status = G.solve(f, g, x, tol=1e-8, maxit=50, check=False)
        assert status == OOM
    finally:
        mgdarcy.inject_alloc_failure(-1)
    st, status = G.solve(f, g, x, tol=1e-8, maxit=50)
    assert status == 0 and st.converged


def test_refused_workspace_growth_keeps_no_freed_buffer():
    """A solve with a larger restart frees the Krylov workspace before it
    allocates the larger one.  If one of those allocations is refused, the
    handle must hold no freed buffer: a later solve with the old, smaller
    restart allocates again and repeats the first solve's result."""
    G = make()
    f, g = load(G)
    x0 = torch.zeros(G.ndof(), dtype=torch.float64, device="cuda")
    st0, status0 = G.solve(f, g, x0, tol=1e-8, maxit=60, restart=10, check=False)
    x = torch.zeros_like(x0)
    mgdarcy.inject_alloc_failure(1)            # the second buffer of the larger workspace
    try:
        _, status = G.solve(f, g, x, tol=1e-8, maxit=60, restart=30, check=False)
        assert status == OOM
    finally:
        mgdarcy.inject_alloc_failure(-1)
    x1 = torch.zeros_like(x0)
    st1, status1 = G.solve(f, g, x1, tol=1e-8, maxit=60, restart=10, check=False)
    assert status1 == status0 and st1.iterations == st0.iterations
    assert torch.max(torch.abs(x1 - x0)).item() <= 1e-12 * torch.max(torch.abs(x0)).item()


def test_device_only_steps_refuse_host_pointers():
    """The single-step entry points take device vectors only: a host array is
    refused with MG_ERR_INVALID_ARG before any kernel sees it, and so is
    mg_apply with x and y the same buffer.  The handle works normally
    afterwards.  Whether a NumPy buffer counts as host memory is the CUDA
    runtime's answer for the platform (where host memory is reported as device
    memory the refusals do not apply and that part is skipped); the long-standing
    check of mg_residual_norm asks it first."""
    G = make(precision="fp64")
    n1, n0, nJ = G.ndof(1), G.ndof(0), G.ndof()
    y = torch.zeros(nJ, dtype=torch.float64, device="cuda")
    with pytest.raises(mgdarcy.MGError) as e:
        G.apply(y, y)
    assert e.value.status == 1
    x = torch.as_tensor(np.random.default_rng(5).standard_normal(nJ), device="cuda")
    G.apply(x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all().item() and torch.count_nonzero(y).item() > 0
    try:
        G.residual_norm(np.zeros(nJ), np.zeros(nJ))
    except mgdarcy.MGError as ex:
        assert ex.status == 1
    else:
        pytest.skip("the CUDA runtime reports host memory as device memory here")
    hx, hc = np.zeros(n1), np.zeros(n0)
    dx = torch.zeros(n1, dtype=torch.float64, device="cuda")
    dc = torch.zeros(n0, dtype=torch.float64, device="cuda")
    calls = [lambda: G.restrict(1, hx, dc), lambda: G.restrict(1, dx, hc), lambda: G.prolong_add(1, hc, dx),
             lambda: G.coarse_solve(hc, dc), lambda: G.smooth(1, hx, dx), lambda: G.level_load(1, hx, None),
             lambda: G.level_store(1, hx)]
    for call in calls:
        with pytest.raises(mgdarcy.MGError) as e:
            call()
        assert e.value.status == 1
    G.restrict(1, dx, dc)
    torch.cuda.synchronize()
