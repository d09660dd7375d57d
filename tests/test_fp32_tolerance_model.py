"""The FP32 tolerances of the GPU parity tests, tied to a rounding model.

test_gpu_parity.py compares the FP32 V-cycle of the CUDA path with the FP64
oracle V-cycle within FP32_VCYCLE_TOL: 2e-3 on the contrast-1e6 channel case,
1e-5 on the others.  Here the oracle's V-cycle runs on the same cases and the
same vector with every operator, patch inverse, transfer, coarse inverse and
vector in single precision (NumPy float32): its difference from the FP64
V-cycle is the error that FP32 arithmetic itself makes on these problems.
Each tolerance must lie between 3 and 1000 times that model error: above it,
with room for the GPU's other summation order and fused multiply-adds, and
not so far above that a mistake well below O(1) could pass.  (Measured on
these cases: 1.1e-5 on the channel field, 0.8-3e-7 on the others.)
"""
import numpy as np
import pytest

import test_gpu_parity as parity
from oracle import multigrid as mg


def single_precision(H):
    """The hierarchy's operators, inverses, transfers and coarse inverse in float32."""
    for L in H.levels:
        L.A = L.A.astype(np.float32)
        L.colours = [None if e is None else (e[0], e[1].astype(np.float32), e[2].astype(np.float32))
                     for e in L.colours]
    H.P = [None] + [P.astype(np.float32) for P in H.P[1:]]
    H.coarse_inv = H.coarse_inv.astype(np.float32)


@pytest.mark.parametrize("case", parity.CASES, ids=[c[0] for c in parity.CASES])
def test_fp32_tolerance_is_a_rounding_bound(case):
    name, d, k, n0, L, mu, cf = case
    H = mg.Hierarchy(d, n0, L, k, mu, cf(n0 * 2 ** (L - 1)))
    r = np.random.default_rng(9).standard_normal(H.levels[-1].S.ndof)
    z = mg.vcycle(H, r)
    single_precision(H)
    z32 = mg.vcycle(H, r.astype(np.float32))
    assert z32.dtype == np.float32
    model = np.linalg.norm(z32 - z) / np.linalg.norm(z)
    tol = parity.FP32_VCYCLE_TOL.get(name, 1e-5)
    assert 3.0 * model <= tol <= 1000.0 * model, (name, model, tol)
