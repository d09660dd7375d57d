"""Parity at the benchmarked size: 256x256 RT_1, 7 levels, channel field (contrast 1e6).

The launch configuration is the one bench.py times (variable V-cycle,
m(J) = 2, FP32 and FP64 V-cycles).  The FP64 oracle (assembled, plain) runs
the same V-cycle on the same seeded vector: FP64 must agree to 1e-10
relative, FP32 to the channel-field bound of the small-case tests; the FP64
operator agrees entry-wise with the assembled matrix to 1e-13 of |A||x|.
"""
import numpy as np
import pytest

from oracle import multigrid as mg
from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402


@pytest.fixture(scope="module")
def workload():
    w = inputs.workload("channels_256")
    H = mg.Hierarchy(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"], w["c"])
    return w, H


def _gpu(w, prec):
    return mgdarcy.Multigrid(w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"],
                             torch.as_tensor(w["c"], device="cuda"), precision=prec, m_fine=2,
                             variable_cycle=True)


def test_fullsize_apply(workload):
    w, H = workload
    LJ = H.levels[-1]
    G = _gpu(w, "fp64")
    x = np.random.default_rng(1).standard_normal(LJ.S.ndof)
    y = torch.zeros(LJ.S.ndof, dtype=torch.float64, device="cuda")
    G.apply(torch.as_tensor(x, device="cuda"), y)
    yo = LJ.A @ x
    bound = 1e-13 * (abs(LJ.A) @ np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - yo) <= bound)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-3)])
def test_fullsize_vcycle(workload, prec, tol):
    w, H = workload
    LJ = H.levels[-1]
    G = _gpu(w, prec)
    r = np.random.default_rng(2).standard_normal(LJ.S.ndof)
    z = torch.zeros(LJ.S.ndof, dtype=torch.float64, device="cuda")
    G.vcycle(torch.as_tensor(r, device="cuda"), z)
    zo = mg.vcycle(H, r, m_fine=2, variable=True)
    err = np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo)
    assert err < tol, err
