"""Parity of the CUDA path (through the C interface) with the FP64 oracle.

Tolerances: FP64 operator 1e-13 of |A||x| per entry; FP64 single steps and
V-cycles 1e-10 relative (Sec. 3.2/3.3 quantities, conditioning-limited); the
FP32 V-cycle is compared with a bound derived from FP32 rounding (see
test_vcycle_fp32_error).  Inputs are seeded synthetic fields with the
structure of the paper's workloads (lognormal and channelised coefficients).
"""
import numpy as np
import pytest

from oracle import krylov
from oracle import multigrid as mg
from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

DEV = "cuda"


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# (name, d, k, n_coarse, n_levels, mu, coefficient factory)
CASES = [
    ("rt0_2d_lognormal_mu1", 2, 0, 2, 4, 1.0, lambda n: inputs.lognormal_c(n, 2, 1.0, 4.0, 1)),
    ("rt1_2d_channels", 2, 1, 2, 4, 0.01, lambda n: inputs.channel_c(n, 4, 2)),
    ("rt1_2d_ragged", 2, 1, 3, 3, 0.3, lambda n: inputs.lognormal_c(n, 2, 1.5, 3.0, 5)),
    ("rt0_3d_darcy", 3, 0, 2, 3, 0.0, lambda n: inputs.lognormal_c(n, 3, 3.0, 2.0, 3)),
    ("rt0_3d_brinkman", 3, 0, 3, 2, 0.05, lambda n: inputs.lognormal_c(n, 3, 1.0, 2.0, 4)),
]
# Bound on the FP32 V-cycle's relative difference from the FP64 oracle V-cycle
# (2-norm): 2e-3 for the contrast-1e6 channel field, 1e-5 for the others.  The
# oracle's V-cycle run entirely in float32 differs from its FP64 one by 1.1e-5
# and 0.8-3e-7 on these cases; test_fp32_tolerance_model.py keeps every bound
# between 3 and 1000 times that rounding-model error.
FP32_VCYCLE_TOL = {"rt1_2d_channels": 2e-3}


def physical_rhs(L, seed):
    """Random load in the velocity rows, no divergence source (g = 0), u.n = 0."""
    b = np.random.default_rng(seed).standard_normal(L.S.ndof)
    b[L.cm] = 0.0
    b[L.S.n_u:] = 0.0
    return b

_cache = {}


# colour-pass kernels: 1 one warp per patch, 2 one thread block per patch,
# 3 persistent thread blocks, 9 / 10 the block kernel with 2 / 8 threads per
# patch row
KERNELS = [1, 2, 3, 9, 10]
KERNEL_IDS = ["warp", "block", "persistent", "block_2threads", "block_8threads"]


def build(case, precision="fp64", variable=True, m_fine=2, dense_level=-1, pass_kernel=0, additive=0.0):
    name, d, k, n0, L, mu, cf = case
    nf = n0 * 2 ** (L - 1)
    c = cf(nf)
    key = (name,)
    if key not in _cache:
        _cache[key] = mg.Hierarchy(d, n0, L, k, mu, c)
    H = _cache[key]
    G = mgdarcy.Multigrid(d, n0, L, k, mu, dev(c), precision=precision, m_fine=m_fine, variable_cycle=variable,
                          dense_level=dense_level, pass_kernel=pass_kernel, additive=additive)
    return H, G


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sizes_match_layout(case):
    H, G = build(case)
    for j, L in enumerate(H.levels):
        assert G.sizes(j) == (L.S.n_u, L.S.n_p)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_apply_parity(case):
    H, G = build(case)
    rng = np.random.default_rng(1)
    for j, L in enumerate(H.levels):
        x = rng.standard_normal(L.S.ndof)
        y = torch.zeros(L.S.ndof, dtype=torch.float64, device=DEV)
        G.apply(dev(x), y, level=j)
        yo = L.A @ x
        bound = 1e-13 * (abs(L.A) @ np.abs(x)) + 1e-300
        assert np.all(np.abs(host(y) - yo) <= bound), f"level {j}: {np.max(np.abs(host(y) - yo) / bound)}"


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_transfer_parity(case):
    H, G = build(case)
    rng = np.random.default_rng(2)
    for j in range(1, len(H.levels)):
        Lf, Lc = H.levels[j], H.levels[j - 1]
        r = rng.standard_normal(Lf.S.ndof)
        bc = torch.zeros(Lc.S.ndof, dtype=torch.float64, device=DEV)
        G.restrict(j, dev(r), bc)
        rr = r.copy()
        rr[Lf.cm] = 0.0
        bo = H.P[j].T @ rr
        bo[Lc.cm] = 0.0
        assert rel_inf(host(bc), bo) < 1e-14
        xc = rng.standard_normal(Lc.S.ndof)
        xc[Lc.cm] = 0.0
        x0 = rng.standard_normal(Lf.S.ndof)
        xf = dev(x0)
        G.prolong_add(j, dev(xc), xf)
        xo = x0 + H.P[j] @ xc
        assert rel_inf(host(xf), xo) < 1e-14


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_coarse_solve_parity(case):
    H, G = build(case)
    L0 = H.levels[0]
    rng = np.random.default_rng(3)
    b = rng.standard_normal(L0.S.ndof)
    x = torch.zeros_like(dev(b))
    G.coarse_solve(dev(b), x)
    assert rel_inf(host(x), mg.coarse_solve(H, b)) < 1e-11


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_smoothing_step_parity_fp64(case, kernel):
    H, G = build(case, pass_kernel=kernel)
    rng = np.random.default_rng(4)
    for j in range(1, len(H.levels)):
        L = H.levels[j]
        x0 = rng.standard_normal(L.S.ndof)
        b = rng.standard_normal(L.S.ndof)
        x = dev(x0)
        G.smooth(j, x, dev(b), steps=1)
        xo = mg.smooth_step(L, x0, b)
        assert rel_inf(host(x), xo) < 1e-10, f"level {j}"


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("variable", [True, False])
@pytest.mark.parametrize("dense_level", [0, -1, 1], ids=["passes", "dense_auto", "dense_1"])
def test_vcycle_parity_fp64(case, variable, dense_level):
    """One V-cycle, all levels as colour passes or with the sub-cycle of the
    coarsest levels applied as its precomputed dense matrix."""
    H, G = build(case, variable=variable, m_fine=2 if variable else 1, dense_level=dense_level)
    LJ = H.levels[-1]
    rng = np.random.default_rng(5)
    r = rng.standard_normal(LJ.S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    zo = mg.vcycle(H, r, m_fine=2 if variable else 1, variable=variable)
    assert rel_inf(host(z), zo) < 1e-10


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vcycle_parity_fp64_each_kernel(case, kernel):
    """One variable V-cycle with every level's colour passes on one kernel."""
    H, G = build(case, dense_level=0, pass_kernel=kernel)
    LJ = H.levels[-1]
    r = np.random.default_rng(15).standard_normal(LJ.S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    assert rel_inf(host(z), mg.vcycle(H, r)) < 1e-10


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=[CASES[1][0], CASES[3][0]])
def test_smoothing_step_fp32_each_kernel(case, kernel):
    """A symmetric FP32 smoothing step on every level against the FP64 oracle
    step: relative error of the update within the FP32 bound FP32_VCYCLE_TOL."""
    H, G = build(case, precision="fp32", pass_kernel=kernel)
    tol = FP32_VCYCLE_TOL.get(case[0], 1e-5)
    rng = np.random.default_rng(16)
    for j in range(1, len(H.levels)):
        L = H.levels[j]
        x0 = rng.standard_normal(L.S.ndof)
        b = rng.standard_normal(L.S.ndof)
        x = dev(x0)
        G.smooth(j, x, dev(b), steps=1)
        d_gpu, d_ora = host(x) - x0, mg.smooth_step(L, x0, b) - x0
        err = np.linalg.norm(d_gpu - d_ora) / np.linalg.norm(d_ora)
        assert err < tol, f"level {j}: {err}"


@pytest.mark.parametrize("other", [2, 3, 9, 10], ids=["block", "persistent", "block_2threads", "block_8threads"])
@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16inv"])
@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=[CASES[1][0], CASES[3][0]])
def test_colour_pass_kernels_agree(case, precision, other):
    """The kernels read the same stored inverses (BF16 ones included) and
    differ only in FP32 summation order, so their smoothing steps agree within
    twice the FP32 bound FP32_VCYCLE_TOL."""
    _, Gw = build(case, precision=precision, pass_kernel=1)
    _, Gb = build(case, precision=precision, pass_kernel=other)
    tol = 2.0 * FP32_VCYCLE_TOL.get(case[0], 1e-5)
    rng = np.random.default_rng(17)
    for j in range(1, case[4]):
        nd = Gw.ndof(j)
        x0 = rng.standard_normal(nd)
        b = rng.standard_normal(nd)
        xw, xb = dev(x0), dev(x0)
        Gw.smooth(j, xw, dev(b), steps=1)
        Gb.smooth(j, xb, dev(b), steps=1)
        dw, db = host(xw) - x0, host(xb) - x0
        assert np.linalg.norm(dw - db) <= tol * np.linalg.norm(dw), f"level {j}"


def test_config1_vcycle_and_solve():
    """The 16x16 RT_0 lognormal workload (levels 2x2 -> 16x16, mu = 1, V(1,1))."""
    w = inputs.workload("small_2d")
    H = mg.Hierarchy(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], w["c"])
    G = mgdarcy.Multigrid(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], dev(w["c"]),
                          precision="fp64", m_fine=1, variable_cycle=False)
    LJ = H.levels[-1]
    rng = np.random.default_rng(6)
    b = rng.standard_normal(LJ.S.ndof)
    b[LJ.cm] = 0.0
    b[LJ.S.n_u:] -= b[LJ.S.n_u:].mean()
    z = torch.zeros_like(dev(b))
    G.vcycle(dev(b), z)
    assert rel_inf(host(z), mg.vcycle(H, b, 1, False)) < 1e-10
    xo, its_o, _ = krylov.fgmres(lambda v: LJ.A @ v, lambda v: mg.vcycle(H, v, 1, False), b, tol=1e-8)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:LJ.S.n_u]), dev(b[LJ.S.n_u:]), x, tol=1e-8, maxit=100)
    assert st.converged == 1 and st.rel_residual <= 1e-8
    assert abs(st.iterations - its_o) <= 1
    xg = host(x)
    assert np.linalg.norm(LJ.A @ xg - b) <= 1e-8 * np.linalg.norm(b) * 1.01


def direct_solution(L, b):
    """Sparse direct solve of A x = b on the free dofs with zero pressure mean (bordered, SciPy LU)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    fr = L.free
    w = L.w[fr]
    Af = L.A[fr][:, fr]
    M = sp.bmat([[Af, sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]]).tocsc()
    y = spl.splu(M).solve(np.concatenate([b[fr], [0.0]]))
    x = b.copy()
    x[fr] = y[:-1]
    return x


# relative distance of the 1e-10 GMRES solution from the direct solution
SOLVE_TOL = {"rt1_2d_channels": 1e-5}


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_solve_fp64_matches_oracle(case):
    """Iteration counts agree with the oracle's FGMRES at 1e-8; the 1e-10 solution matches a direct solve."""
    H, G = build(case)
    LJ = H.levels[-1]
    S = LJ.S
    b = physical_rhs(LJ, 7)
    _, its_o, _ = krylov.fgmres(lambda v: LJ.A @ v, lambda v: mg.vcycle(H, v), b, tol=1e-8, maxit=300)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-8, maxit=300)
    assert st.converged == 1
    assert abs(st.iterations - its_o) <= 2, (st.iterations, its_o)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-10, maxit=400)
    xg = host(x)
    assert np.linalg.norm(LJ.A @ xg - b) <= 1.01e-10 * np.linalg.norm(b)
    xd = direct_solution(LJ, b)
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) < SOLVE_TOL.get(case[0], 1e-8)


@pytest.mark.parametrize("kernel", [0, 4], ids=["rule", "timed"])
@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16inv"])
@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_mixed_precision_solve_reaches_1e8(case, precision, kernel):
    """FP32 / BF16-inverse V-cycle inside FP64 flexible GMRES reaches 1e-8 (FP64 residual)."""
    H, G = build(case, precision=precision, pass_kernel=kernel)
    LJ = H.levels[-1]
    S = LJ.S
    b = physical_rhs(LJ, 8)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-8, maxit=300)
    xg = host(x)
    assert st.converged == 1
    assert np.linalg.norm(LJ.A @ xg - b) <= 1.01e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_vcycle_fp32_error(case, kernel):
    """FP32 V-cycle vs the FP64 oracle V-cycle, bound FP32_VCYCLE_TOL."""
    H, G = build(case, precision="fp32", pass_kernel=kernel)
    LJ = H.levels[-1]
    rng = np.random.default_rng(9)
    r = rng.standard_normal(LJ.S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    zo = mg.vcycle(H, r)
    err = np.linalg.norm(host(z) - zo) / np.linalg.norm(zo)
    assert err < FP32_VCYCLE_TOL.get(case[0], 1e-5), err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_persistent_blocks_walk_many_patches(precision, tol):
    """On a 128^2 RT_1 level (1,800 patches per colour, more than the resident
    blocks) each persistent block updates several patches in turn: its
    smoothing step agrees with the warp kernel's to rounding."""
    c = inputs.lognormal_c(128, 2, 2.0, 8.0, 21)
    Gs = [mgdarcy.Multigrid(2, 4, 6, 1, 0.01, dev(c), precision=precision, dense_level=0, pass_kernel=pk)
          for pk in (1, 3)]
    rng = np.random.default_rng(22)
    for j in (5, 4):
        nd = Gs[0].ndof(j)
        x0, b = rng.standard_normal(nd), rng.standard_normal(nd)
        d = []
        for G in Gs:
            x = dev(x0)
            G.smooth(j, x, dev(b), steps=1)
            d.append(host(x) - x0)
        assert np.linalg.norm(d[1] - d[0]) <= tol * np.linalg.norm(d[0]), j


@pytest.mark.parametrize("dense_level", [0, -1], ids=["passes", "dense_auto"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_additive_vcycle_parity_fp64(case, dense_level):
    """The additive Schwarz variant (omega = 0.25, not the paper's smoother):
    one V-cycle against the oracle's."""
    H, G = build(case, dense_level=dense_level, additive=0.25)
    LJ = H.levels[-1]
    r = np.random.default_rng(23).standard_normal(LJ.S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    assert rel_inf(host(z), mg.vcycle(H, r, additive=0.25)) < 1e-10


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_additive_solve_reaches_1e8(case):
    H, G = build(case, precision="fp32", additive=0.25)
    LJ = H.levels[-1]
    S = LJ.S
    b = physical_rhs(LJ, 24)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-8, maxit=400)
    assert st.converged == 1
    assert np.linalg.norm(LJ.A @ host(x) - b) <= 1.01e-8 * np.linalg.norm(b)


def test_pass_kernel_choice():
    """Explicit choices are kept; the fixed rule (pass_kernel 5) takes the
    block kernel where a level's largest colour holds at most 10,000 inverse
    entries per SM; the default timed trial picks, per level, a kernel whose
    measured pass time is within the timing noise of the fastest."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    case = CASES[1]
    for pk, want in ((1, 1), (2, 2), (3, 3)):
        _, G = build(case, pass_kernel=pk)
        assert all(G.pass_kernel(j) == want for j in range(1, case[4]))
    _, G = build(case, pass_kernel=5)
    for j in range(1, case[4]):
        mx, nv = max(G.patch_info(j, c) for c in range(9))
        assert G.pass_kernel(j) == (2 if mx * nv * nv <= 10000 * nsm else 1)
    for precision in ("fp32", "fp64"):
        _, G = build(case, precision=precision)
        for j in range(1, case[4]):
            t = [G.time_passes(j, k) for k in (1, 2, 3)]
            assert G.pass_kernel(j) in (1, 2, 3)
            assert t[G.pass_kernel(j) - 1] <= 1.25 * min(t) + 0.3, (precision, j, t, G.pass_kernel(j))
    with pytest.raises(mgdarcy.MGError):
        G.pass_kernel(0)


def test_host_pointers_give_the_same_vcycle():
    case = CASES[1]
    H, G = build(case)
    n = H.levels[-1].S.ndof
    r = np.random.default_rng(10).standard_normal(n)
    z_host = np.zeros(n)
    G.vcycle(r, z_host)
    z_dev = torch.zeros(n, dtype=torch.float64, device=DEV)
    G.vcycle(dev(r), z_dev)
    assert np.array_equal(z_host, host(z_dev))


def test_single_level_is_the_coarse_solve():
    d, k, n0, mu = 2, 1, 4, 0.2
    c = inputs.lognormal_c(n0, 2, 1.0, 2.0, 11)
    H = mg.Hierarchy(d, n0, 1, k, mu, c)
    G = mgdarcy.Multigrid(d, n0, 1, k, mu, dev(c))
    r = np.random.default_rng(12).standard_normal(H.levels[0].S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    assert rel_inf(host(z), mg.vcycle(H, r)) < 1e-11


def test_setup_rejects_bad_coefficient_on_device():
    c = np.ones((8, 8))
    c[3, 4] = -1.0
    with pytest.raises(mgdarcy.MGError) as e:
        mgdarcy.Multigrid(2, 2, 3, 0, 1.0, dev(c))
    assert e.value.status == 1


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_residual_norm_parity(case):
    H, G = build(case)
    LJ = H.levels[-1]
    rng = np.random.default_rng(13)
    x = rng.standard_normal(LJ.S.ndof)
    b = rng.standard_normal(LJ.S.ndof)
    r = torch.zeros_like(dev(x))
    nrm = G.residual_norm(dev(x), dev(b), r)
    ro = b - LJ.A @ x
    bound = 1e-13 * (abs(LJ.A) @ np.abs(x) + np.abs(b))
    assert np.all(np.abs(host(r) - ro) <= bound)
    assert abs(nrm - np.linalg.norm(ro)) <= 1e-12 * np.linalg.norm(ro)


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]], ids=[CASES[0][0], CASES[1][0], CASES[3][0]])
def test_load_vector_parity(case):
    """Cellwise-constant f and g: GPU load vector against the oracle's quadrature (eq. BCh)."""
    from oracle import fem
    name, d, k, n0, L, mu, cf = case
    n = n0 * 2 ** (L - 1)
    H, G = build(case)
    S = H.levels[-1].S
    rng = np.random.default_rng(14)
    fc = rng.standard_normal((d,) + (n,) * d)
    gc = rng.standard_normal((n,) * d)
    h = 1.0 / n

    def cell_of(X):
        idx = np.minimum((X / h).astype(int), n - 1)
        return tuple(idx[:, e] for e in reversed(range(d)))

    f = lambda X, c: np.stack([fc[i][cell_of(X)] for i in range(d)], 1)
    g = lambda X: gc[cell_of(X)]
    bo = fem.load_vector(S, mu, H.levels[-1].c, f=f, div_source=g)
    b = torch.zeros(S.ndof, dtype=torch.float64, device=DEV)
    G.load_vector(dev(fc.reshape(d, -1)), dev(gc.reshape(-1)), b)
    assert rel_inf(host(b), bo) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", [0, 2, 7], ids=["timed", "block", "block_rhs1"])
def test_vcycle_with_several_right_hand_sides(precision, kernel):
    """A single problem set up with nrhs = 5 (a group of four sharing each
    patch-inverse load and one on its own): every vector of one mg_vcycle call
    against the oracle's V-cycle of that vector (FP64 1e-10, FP32 the bound
    FP32_VCYCLE_TOL of the case); mg_solve refuses the handle."""
    case = CASES[1]
    name, d, k, n0, L, mu, cf = case
    tol = 1e-10 if precision == "fp64" else FP32_VCYCLE_TOL.get(name, 1e-5)
    c = cf(n0 * 2 ** (L - 1))
    H, _ = build(case)
    G = mgdarcy.Multigrid(d, n0, L, k, mu, dev(c), precision=precision, pass_kernel=kernel, nrhs=5)
    nd = H.levels[-1].S.ndof
    r = np.random.default_rng(33).standard_normal(5 * nd)
    z = torch.zeros(5 * nd, dtype=torch.float64, device=DEV)
    G.vcycle(dev(r), z)
    zh = host(z)
    for q in range(5):
        zo = mg.vcycle(H, r[q * nd:(q + 1) * nd])
        assert np.linalg.norm(zh[q * nd:(q + 1) * nd] - zo) <= tol * np.linalg.norm(zo), q
    nu, npr = G.sizes()
    with pytest.raises(mgdarcy.MGError) as e:
        G.solve(dev(np.zeros(nu)), dev(np.zeros(npr)), torch.zeros(nd, dtype=torch.float64, device=DEV))
    assert e.value.status == 7
