"""The smoother with the patches of every vertex (Sec. 3.3), boundary
vertices included (mg_problem.boundary_patches), against the FP64 oracle with
the same option: patch counts, one V-cycle in FP64 (1e-10) for every
colour-pass kernel and both cycles, the FP32 V-cycle within the FP32 bound of
the other parity tests, and a mixed-precision solve to an FP64-evaluated 1e-8.
"""
import numpy as np
import pytest

from oracle import multigrid as mg
from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

# (name, d, k, n_coarse, n_levels, mu, coefficient factory)
CASES = [
    ("rt0_2d_lognormal", 2, 0, 2, 4, 1.0, lambda n: inputs.lognormal_c(n, 2, 1.0, 4.0, 1)),
    ("rt1_2d_channels", 2, 1, 2, 4, 0.01, lambda n: inputs.channel_c(n, 4, 2)),
    ("rt1_2d_ragged", 2, 1, 3, 3, 0.3, lambda n: inputs.lognormal_c(n, 2, 1.5, 3.0, 5)),
    ("rt0_3d_brinkman", 3, 0, 2, 3, 0.05, lambda n: inputs.lognormal_c(n, 3, 1.0, 2.0, 4)),
]
IDS = [c[0] for c in CASES]
FP32_TOL = {"rt1_2d_channels": 2e-3}
_cache = {}


def oracle(case):
    name, d, k, n0, L, mu, cf = case
    if name not in _cache:
        c = cf(n0 * 2 ** (L - 1))
        _cache[name] = (c, mg.Hierarchy(d, n0, L, k, mu, c, boundary_patches=True))
    return _cache[name]


def gpu(case, c, **kw):
    name, d, k, n0, L, mu, _ = case
    return mgdarcy.Multigrid(d, n0, L, k, mu, torch.as_tensor(c, device="cuda"), boundary_patches=True, **kw)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_boundary_patch_counts(case):
    c, H = oracle(case)
    G = gpu(case, c, precision="fp64")
    for j in range(1, H.J + 1):
        Lj = H.levels[j]
        nmax = 0
        for col in range(len(Lj.colours)):
            want = sum(g[0].shape[0] for g in Lj.bcolours[col])
            nmax = max([nmax] + [g[0].shape[1] for g in Lj.bcolours[col]])
            cnt, nv = G.boundary_patch_info(j, col)
            assert cnt == want, (j, col, cnt, want)
        assert G.boundary_patch_info(j, 0)[1] == nmax


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["warp", "block", "persistent"])
@pytest.mark.parametrize("variable", [True, False], ids=["variable", "standard"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_boundary_patch_vcycle_fp64(case, variable, kernel):
    c, H = oracle(case)
    G = gpu(case, c, precision="fp64", variable_cycle=variable, pass_kernel=kernel)
    LJ = H.levels[-1]
    r = np.random.default_rng(31).standard_normal(LJ.S.ndof)
    z = torch.zeros(LJ.S.ndof, dtype=torch.float64, device="cuda")
    G.vcycle(torch.as_tensor(r, device="cuda"), z)
    zo = mg.vcycle(H, r, m_fine=2, variable=variable)
    assert np.max(np.abs(z.cpu().numpy() - zo)) < 1e-10 * np.max(np.abs(zo))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_boundary_patch_smoothing_step_fp64(case):
    c, H = oracle(case)
    G = gpu(case, c, precision="fp64")
    j = H.J
    Lj = H.levels[j]
    rng = np.random.default_rng(32)
    x0 = rng.standard_normal(Lj.S.ndof)
    b = rng.standard_normal(Lj.S.ndof)
    x = torch.as_tensor(x0, device="cuda")
    G.smooth(j, x, torch.as_tensor(b, device="cuda"), steps=1)
    xo = mg.smooth_step(Lj, x0, b)
    assert np.max(np.abs(x.cpu().numpy() - xo)) < 1e-10 * np.max(np.abs(xo))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_boundary_patch_vcycle_fp32(case):
    c, H = oracle(case)
    G = gpu(case, c, precision="fp32")
    LJ = H.levels[-1]
    r = np.random.default_rng(33).standard_normal(LJ.S.ndof)
    z = torch.zeros(LJ.S.ndof, dtype=torch.float64, device="cuda")
    G.vcycle(torch.as_tensor(r, device="cuda"), z)
    zo = mg.vcycle(H, r)
    assert np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo) < FP32_TOL.get(case[0], 1e-5)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_boundary_patch_solve_fp32(case):
    c, H = oracle(case)
    G = gpu(case, c, precision="fp32")
    LJ = H.levels[-1]
    b = np.random.default_rng(34).standard_normal(LJ.S.ndof)
    b[LJ.cm] = 0.0
    b[LJ.S.n_u:] = 0.0
    x = torch.zeros(LJ.S.ndof, dtype=torch.float64, device="cuda")
    st, _ = G.solve(torch.as_tensor(b[:LJ.S.n_u], device="cuda"), torch.as_tensor(b[LJ.S.n_u:], device="cuda"), x,
                    tol=1e-8, maxit=200)
    assert st.converged == 1
    assert np.linalg.norm(LJ.A @ x.cpu().numpy() - b) <= 1.01e-8 * np.linalg.norm(b)


def test_boundary_patches_rejected_where_unsupported():
    case = CASES[0]
    c, _ = oracle(case)
    with pytest.raises(mgdarcy.MGError) as ei:
        gpu(case, c, additive=0.25)
    assert ei.value.status == 7
    probs = [dict(dim=2, n_coarse=2, n_levels=3, degree=0, mu=1.0, c=torch.as_tensor(c[::2, ::2].copy(), device="cuda"),
                  boundary_patches=True)]
    with pytest.raises(mgdarcy.MGError) as ei:
        mgdarcy.Batch(probs, nrhs=1)
    assert ei.value.status == 7
