"""RT_2 x Q_2 (Sec. 2.3 defines RT_k x Q_k for every k) on the GPU against the
FP64 oracle.

Patches of RT_2 hold 96 dofs in 2-D; their colour passes run the block
kernels (one block per patch, or persistent blocks walking the patches), with
the inverses staged in dynamic shared memory (37 KB FP32, 74 KB FP64).
The bounds are those of the RT_0/RT_1 parity tests: FP64 operator 1e-13 of
|A||x| per entry, transfers 1e-14, coarse solve 1e-11, single smoothing steps
and V-cycles 1e-10 relative; FP32 V-cycles 1e-5 relative on lognormal fields
(FP32 rounding, u = 6e-8, amplified by the conditioning of the patch
inverses); mixed-precision solves reach an FP64-evaluated 1e-8.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import krylov
from oracle import multigrid as mg
from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

DEV = "cuda"

# (name, n_coarse, n_levels, mu, coefficient factory)
CASES = [
    ("rt2_lognormal_brinkman", 2, 4, 0.01, lambda n: inputs.lognormal_c(n, 2, 1.5, 4.0, 41)),
    ("rt2_ragged_darcy", 3, 3, 0.0, lambda n: inputs.lognormal_c(n, 2, 2.0, 3.0, 42)),
    ("rt2_channels_stokeslike", 2, 3, 1.0, lambda n: inputs.channel_c(n, 2, 43)),
]
IDS = [c[0] for c in CASES]
_cache = {}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def build(case, boundary_patches=False, **kw):
    name, n0, L, mu, cf = case
    c = cf(n0 * 2 ** (L - 1))
    key = (name, boundary_patches)
    if key not in _cache:
        _cache[key] = mg.Hierarchy(2, n0, L, 2, mu, c, boundary_patches=boundary_patches)
    G = mgdarcy.Multigrid(2, n0, L, 2, mu, dev(c), boundary_patches=boundary_patches, **kw)
    return _cache[key], G


def physical_rhs(L, seed):
    b = np.random.default_rng(seed).standard_normal(L.S.ndof)
    b[L.cm] = 0.0
    b[L.S.n_u:] = 0.0
    return b


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_sizes_and_patches(case):
    H, G = build(case)
    for j, L in enumerate(H.levels):
        assert G.sizes(j) == (L.S.n_u, L.S.n_p)
    LJ = H.levels[-1]
    total = 0
    for col in range(9):
        cnt, nv = G.patch_info(len(H.levels) - 1, col)
        assert nv == 96
        total += cnt
    assert total == (LJ.S.n - 1) ** 2


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_and_residual_parity(case):
    H, G = build(case)
    rng = np.random.default_rng(1)
    for j, L in enumerate(H.levels):
        x = rng.standard_normal(L.S.ndof)
        y = torch.zeros(L.S.ndof, dtype=torch.float64, device=DEV)
        G.apply(dev(x), y, level=j)
        bound = 1e-13 * (abs(L.A) @ np.abs(x)) + 1e-300
        assert np.all(np.abs(host(y) - L.A @ x) <= bound), j
    LJ = H.levels[-1]
    x, b = rng.standard_normal(LJ.S.ndof), rng.standard_normal(LJ.S.ndof)
    r = torch.zeros_like(dev(x))
    nrm = G.residual_norm(dev(x), dev(b), r)
    ro = b - LJ.A @ x
    assert np.all(np.abs(host(r) - ro) <= 1e-13 * (abs(LJ.A) @ np.abs(x) + np.abs(b)))
    assert abs(nrm - np.linalg.norm(ro)) <= 1e-12 * np.linalg.norm(ro)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_transfer_and_coarse_parity(case):
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
        assert rel_inf(host(xf), x0 + H.P[j] @ xc) < 1e-14
    b = rng.standard_normal(H.levels[0].S.ndof)
    x = torch.zeros_like(dev(b))
    G.coarse_solve(dev(b), x)
    assert rel_inf(host(x), mg.coarse_solve(H, b)) < 1e-11


KERNELS = [2, 3, 9, 10]
KERNEL_IDS = ["block", "persistent", "block_2threads", "block_8threads"]


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_smoothing_step_parity_fp64(case, kernel):
    H, G = build(case, pass_kernel=kernel)
    rng = np.random.default_rng(4)
    for j in range(1, len(H.levels)):
        L = H.levels[j]
        x0, b = rng.standard_normal(L.S.ndof), rng.standard_normal(L.S.ndof)
        x = dev(x0)
        G.smooth(j, x, dev(b), steps=1)
        assert rel_inf(host(x), mg.smooth_step(L, x0, b)) < 1e-10, j


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("variable", [True, False])
@pytest.mark.parametrize("dense_level", [0, -1], ids=["passes", "dense_auto"])
def test_vcycle_parity_fp64(case, variable, dense_level):
    H, G = build(case, variable_cycle=variable, m_fine=2 if variable else 1, dense_level=dense_level)
    r = np.random.default_rng(5).standard_normal(H.levels[-1].S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    zo = mg.vcycle(H, r, m_fine=2 if variable else 1, variable=variable)
    assert rel_inf(host(z), zo) < 1e-10


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_vcycle_fp32_error(case, kernel):
    H, G = build(case, precision="fp32", pass_kernel=kernel)
    r = np.random.default_rng(9).standard_normal(H.levels[-1].S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    zo = mg.vcycle(H, r)
    assert np.linalg.norm(host(z) - zo) / np.linalg.norm(zo) < 1e-5


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_additive_vcycle_parity_fp64(case):
    H, G = build(case, additive=0.25, dense_level=0)
    r = np.random.default_rng(23).standard_normal(H.levels[-1].S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    assert rel_inf(host(z), mg.vcycle(H, r, additive=0.25)) < 1e-10


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_boundary_patches_vcycle_parity_fp64(case):
    """Patches of every vertex (Sec. 3.3): the boundary ones (at most 45 dofs
    for RT_2) through the listed-patch pass after each colour's interior pass."""
    H, G = build(case, boundary_patches=True, dense_level=0)
    r = np.random.default_rng(25).standard_normal(H.levels[-1].S.ndof)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    assert rel_inf(host(z), mg.vcycle(H, r)) < 1e-10
    cnt, mx = G.boundary_patch_info(len(H.levels) - 1, 0)
    assert cnt > 0 and 0 < mx <= 96


def direct_solution(L, b):
    fr = L.free
    w = L.w[fr]
    M = sp.bmat([[L.A[fr][:, fr], sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]]).tocsc()
    y = spl.splu(M).solve(np.concatenate([b[fr], [0.0]]))
    x = b.copy()
    x[fr] = y[:-1]
    return x


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_solve_fp64_matches_oracle(case):
    H, G = build(case)
    LJ = H.levels[-1]
    S = LJ.S
    b = physical_rhs(LJ, 7)
    _, its_o, _ = krylov.fgmres(lambda v: LJ.A @ v, lambda v: mg.vcycle(H, v), b, tol=1e-8, maxit=300)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-8, maxit=300)
    assert st.converged == 1 and abs(st.iterations - its_o) <= 2, (st.iterations, its_o)
    x = torch.zeros_like(dev(b))
    G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-10, maxit=400)
    xg = host(x)
    assert np.linalg.norm(LJ.A @ xg - b) <= 1.01e-10 * np.linalg.norm(b)
    xd = direct_solution(LJ, b)
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) < 1e-8


@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16inv"])
@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_mixed_precision_solve_reaches_1e8(case, precision):
    H, G = build(case, precision=precision)
    LJ = H.levels[-1]
    S = LJ.S
    b = physical_rhs(LJ, 8)
    x = torch.zeros_like(dev(b))
    st, _ = G.solve(dev(b[:S.n_u]), dev(b[S.n_u:]), x, tol=1e-8, maxit=300)
    assert st.converged == 1
    assert np.linalg.norm(LJ.A @ host(x) - b) <= 1.01e-8 * np.linalg.norm(b)


@pytest.fixture(scope="module")
def big():
    """64^2 RT_2 Brinkman (mu = 0.01), lognormal c: 3,969 patches of 96 dofs on
    the finest level, 441 per colour."""
    c = inputs.lognormal_c(64, 2, 2.0, 8.0, 44)
    H = mg.Hierarchy(2, 4, 5, 2, 0.01, c)
    r = np.random.default_rng(45).standard_normal(H.levels[-1].S.ndof)
    return c, H, r, mg.vcycle(H, r)


@pytest.mark.parametrize("kernel", [0, 2, 3], ids=["timed", "block", "persistent"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_vcycle_64(big, precision, tol, kernel):
    """FP64 at the parity bound, FP32 at the FP32 bound of the small cases;
    the persistent blocks walk several patches each on the finest level."""
    c, H, r, zo = big
    G = mgdarcy.Multigrid(2, 4, 5, 2, 0.01, dev(c), precision=precision, pass_kernel=kernel)
    z = torch.zeros_like(dev(r))
    G.vcycle(dev(r), z)
    err = np.linalg.norm(host(z) - zo) / np.linalg.norm(zo)
    assert err < tol, err


def test_batches_reject_degree_2():
    c = dev(inputs.lognormal_c(8, 2, 1.0, 2.0, 1))
    with pytest.raises(mgdarcy.MGError) as e:
        mgdarcy.Batch([dict(dim=2, n_coarse=2, n_levels=3, degree=2, mu=0.0, c=c)], nrhs=1)
    assert e.value.status == 7   # MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("kernel", [0, 2, 3], ids=["timed", "block", "persistent"])
def test_vcycle_with_four_right_hand_sides(kernel):
    """RT_2 with nrhs = 4 in one handle: the block kernels' four-right-hand-side
    path (each S_v load shared by the four) against the oracle per vector."""
    case = CASES[0]
    name, n0, L, mu, cf = case
    H, _ = build(case)
    c = cf(n0 * 2 ** (L - 1))
    G = mgdarcy.Multigrid(2, n0, L, 2, mu, dev(c), pass_kernel=kernel, nrhs=4)
    nd = H.levels[-1].S.ndof
    r = np.random.default_rng(71).standard_normal(4 * nd)
    z = torch.zeros(4 * nd, dtype=torch.float64, device=DEV)
    G.vcycle(dev(r), z)
    zh = host(z)
    for q in range(4):
        zo = mg.vcycle(H, r[q * nd:(q + 1) * nd])
        assert rel_inf(zh[q * nd:(q + 1) * nd], zo) < 1e-10, q
