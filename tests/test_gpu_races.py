"""Race detection for the colour passes (Sec. 3.3: the patches of one colour
are disjoint and do not couple, so their updates commute).

The persistent kernels walk every patch of a colour whatever their grid, and a
patch's arithmetic does not depend on which block or warp takes it.  So a
smoothing step or a V-cycle computed with one block walking each colour patch
by patch must equal, to the last bit, the one computed with the full grid in
which patches run concurrently: any read of x that raced with a concurrent
write of the same colour, any shared-memory reuse between patches of one
block, or any lost update would change bits.  Checked in FP64 and FP32, on
RT_0, RT_1 and RT_2 levels, for the warp-per-patch and the persistent-block
kernels.  The host-side counterpart (no two patches of one colour couple) is
pinned in tests/test_oracle_pins.py.
"""
import numpy as np
import pytest

from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

# (d, k, n_coarse, n_levels, mu, kernels)
CASES = [(2, 1, 4, 6, 0.01, (1, 3)), (2, 0, 4, 7, 1.0, (1, 3)), (3, 0, 2, 5, 0.0, (1, 3)), (2, 2, 4, 5, 0.01, (3,))]
IDS = ["rt1_128", "rt0_256", "rt0_3d_32", "rt2_64"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_one_block_per_colour_is_bit_identical(case, precision):
    d, k, n0, L, mu, kernels = case
    n = n0 * 2 ** (L - 1)
    c = torch.as_tensor(inputs.lognormal_c(n, d, 2.0, n / 8, 81), device="cuda")
    for kernel in kernels:
        G = mgdarcy.Multigrid(d, n0, L, k, mu, c, precision=precision, pass_kernel=kernel, dense_level=0)
        nd = G.ndof()
        rng = np.random.default_rng(82)
        x0 = torch.as_tensor(rng.standard_normal(nd), device="cuda")
        b = torch.as_tensor(rng.standard_normal(nd), device="cuda")
        r = torch.as_tensor(rng.standard_normal(nd), device="cuda")
        out = []
        for blocks in (0, 1):
            G.set_block_limit(blocks)
            x = x0.clone()
            G.smooth(L - 1, x, b, steps=1)
            z = torch.zeros_like(r)
            G.vcycle(r, z)
            torch.cuda.synchronize()
            out.append((x.clone(), z.clone()))
        assert torch.equal(out[0][0], out[1][0]), (kernel, "smoothing step")
        assert torch.equal(out[0][1], out[1][1]), (kernel, "V-cycle")
        assert not torch.equal(out[0][0], x0)
        del G
