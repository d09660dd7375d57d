"""Batched problems of uneven sizes with four right-hand sides each.

The batch runs every problem's V-cycle as a branch of one CUDA graph and the
four right-hand sides of a problem share each patch-inverse load; FGMRES runs
over all systems in lockstep.  Each system is checked against the FP64
oracle: the V-cycle to 1e-10 (FP64) or the FP32 bound of the single-problem
tests, the solve by its FP64 residual.
"""
import numpy as np
import pytest

from oracle import multigrid as mg
from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

NRHS = 4
# (n_coarse, n_levels, degree, mu, sigma, seed): uneven sizes 8^2, 16^2, 32^2 and a 3-D one
SPECS = [(4, 2, 1, 0.01, 1.0, 11), (4, 3, 1, 0.01, 2.0, 12), (4, 4, 1, 0.01, 3.0, 13)]


def _problems(precision, pass_kernel=0):
    probs, hier = [], []
    for n0, L, k, mu, sig, seed in SPECS:
        n = n0 * 2 ** (L - 1)
        c = inputs.lognormal_c(n, 2, sig, n / 8, seed)
        probs.append(dict(dim=2, n_coarse=n0, n_levels=L, degree=k, mu=mu, c=torch.as_tensor(c, device="cuda"),
                          precision=precision, pass_kernel=pass_kernel))
        hier.append(mg.Hierarchy(2, n0, L, k, mu, c))
    return probs, hier


@pytest.fixture(scope="module")
def oracle_hierarchies():
    return _problems("fp64")[1]


@pytest.mark.parametrize("kernel", [0, 5, 1, 2, 3, 6, 7, 8],
                         ids=["timed", "rule", "warp", "block", "persistent", "warp_rhs1", "block_rhs1",
                              "persistent_rhs1"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_batched_vcycle_matches_oracle(precision, tol, kernel, oracle_hierarchies):
    probs, _ = _problems(precision, kernel)
    B = mgdarcy.Batch(probs, nrhs=NRHS)
    total = B.total()
    rng = np.random.default_rng(4)
    r = rng.standard_normal(total)
    z = torch.zeros(total, dtype=torch.float64, device="cuda")
    B.vcycle(torch.as_tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    for p, H in enumerate(oracle_hierarchies):
        nd, off, _ = B.layout(p)
        for rr in range(NRHS):
            seg = slice(off + rr * nd, off + (rr + 1) * nd)
            zo = mg.vcycle(H, r[seg])
            err = np.linalg.norm(zh[seg] - zo) / np.linalg.norm(zo)
            assert err < tol, (p, rr, err)


def test_batched_solve_converges_every_system(oracle_hierarchies):
    probs, _ = _problems("fp32")
    B = mgdarcy.Batch(probs, nrhs=NRHS)
    total = B.total()
    rng = np.random.default_rng(5)
    b = np.zeros(total)
    for p, H in enumerate(oracle_hierarchies):
        nd, off, _ = B.layout(p)
        LJ = H.levels[-1]
        for rr in range(NRHS):
            seg = b[off + rr * nd: off + (rr + 1) * nd]
            seg[:] = rng.standard_normal(nd)
            seg[LJ.cm] = 0.0
            seg[LJ.S.n_u:] = 0.0
    x = torch.zeros(total, dtype=torch.float64, device="cuda")
    stats, status = B.solve(torch.as_tensor(b, device="cuda"), x, tol=1e-8, maxit=300, restart=20)
    assert status == 0
    xh = x.cpu().numpy()
    for p, H in enumerate(oracle_hierarchies):
        nd, off, _ = B.layout(p)
        A = H.levels[-1].A
        for rr in range(NRHS):
            seg = slice(off + rr * nd, off + (rr + 1) * nd)
            s = stats[p * NRHS + rr]
            assert s.converged == 1
            res = np.linalg.norm(A @ xh[seg] - b[seg]) / np.linalg.norm(b[seg])
            assert res <= 1.01e-8, (p, rr, res)


# Problems of one shape run as one group (storage one after another, one
# launch per kernel for the whole group); two shapes, in contiguous or
# interleaved order, with 1, 2 or 4 right-hand sides per problem.
GROUP_SHAPES = {"a": (4, 3, 1, 0.01), "b": (2, 4, 0, 1.0)}   # (n_coarse, n_levels, degree, mu)


def _group_problems(order, precision):
    probs, hier = [], []
    for i, key in enumerate(order):
        n0, L, k, mu = GROUP_SHAPES[key]
        n = n0 * 2 ** (L - 1)
        c = inputs.lognormal_c(n, 2, 1.0 + 0.5 * i, n / 4, 40 + i)
        probs.append(dict(dim=2, n_coarse=n0, n_levels=L, degree=k, mu=mu, c=torch.as_tensor(c, device="cuda"),
                          precision=precision))
        hier.append(mg.Hierarchy(2, n0, L, k, mu, c))
    return probs, hier


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("order", ["aaabb", "ababa"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_grouped_batch_matches_oracle(precision, tol, order, nrhs):
    probs, hier = _group_problems(order, precision)
    B = mgdarcy.Batch(probs, nrhs=nrhs)
    total = B.total()
    r = np.random.default_rng(6).standard_normal(total)
    z = torch.zeros(total, dtype=torch.float64, device="cuda")
    B.vcycle(torch.as_tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    for p, H in enumerate(hier):
        nd, off, _ = B.layout(p)
        for rr in range(nrhs):
            seg = slice(off + rr * nd, off + (rr + 1) * nd)
            zo = mg.vcycle(H, r[seg])
            err = np.linalg.norm(zh[seg] - zo) / np.linalg.norm(zo)
            assert err < tol, (p, rr, err)


def test_group_launches_once_per_kernel():
    """A V-cycle of three problems of one shape launches as many kernels as
    one problem's."""
    def per_vcycle(order):
        probs, _ = _group_problems(order, "fp32")
        B = mgdarcy.Batch(probs, nrhs=4)
        r = torch.zeros(B.total(), dtype=torch.float64, device="cuda")
        z = torch.zeros_like(r)
        B.vcycle(r, z)
        l0 = B.launches()
        B.vcycle(r, z)
        return B.launches() - l0
    assert per_vcycle("aaa") == per_vcycle("a")


def test_persistent_blocks_in_a_large_group():
    """Sixteen 32^2 RT_1 problems with four right-hand sides: the persistent
    blocks of each right-hand-side group walk several patches; the FP64
    batched V-cycle agrees with the warp kernel's to rounding."""
    probs_w, probs_p = [], []
    for i in range(16):
        c = torch.as_tensor(inputs.lognormal_c(32, 2, 1.5, 4.0, 60 + i), device="cuda")
        for lst, pk in ((probs_w, 1), (probs_p, 3)):
            lst.append(dict(dim=2, n_coarse=4, n_levels=4, degree=1, mu=0.01, c=c, precision="fp64", pass_kernel=pk))
    Bw, Bp = mgdarcy.Batch(probs_w, nrhs=4), mgdarcy.Batch(probs_p, nrhs=4)
    r = torch.as_tensor(np.random.default_rng(8).standard_normal(Bw.total()), device="cuda")
    zw, zp = torch.zeros_like(r), torch.zeros_like(r)
    Bw.vcycle(r, zw)
    Bp.vcycle(r, zp)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(zp - zw) / torch.linalg.norm(zw)).item() < 1e-11


def test_timed_choice_covers_rhs_grouping():
    """With four right-hand sides the timed choice picks, per level, a kernel
    and a grouping (four sharing each inverse load, or one each); forced modes
    report what they force."""
    probs, _ = _problems("fp32", 0)
    B = mgdarcy.Batch(probs, nrhs=NRHS)
    for p, (n0, L, *_rest) in enumerate(SPECS):
        for j in range(1, L):
            k, g, t = B.level_choice(p, j)
            assert k in (1, 2, 3) and g in (1, 4) and t in (2, 4, 8)
    probs, _ = _problems("fp32", 7)
    B = mgdarcy.Batch(probs, nrhs=NRHS)
    assert all(B.level_choice(p, j) == (2, 1, 4) for p, (n0, L, *_r) in enumerate(SPECS) for j in range(1, L))
    probs, _ = _problems("fp32", 2)
    B = mgdarcy.Batch(probs, nrhs=NRHS)
    assert all(B.level_choice(p, j) == (2, 4, 4) for p, (n0, L, *_r) in enumerate(SPECS) for j in range(1, L))
