"""mg_residual_norm_noalloc: the residual norm for callers that cannot allocate.

Callers whose allocator owns the device, or that may not call cudaMalloc at
all (and so have no mg_handle), get ||b - A x||_2 from an entry point whose
scratch is a static device array.  It must give the value of the handle-based
mg_residual_norm (same FP64 arithmetic, tolerance 1e-12 relative as in the
parity tests), on two calls in a row that share the static array.  This file
is collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_1602_04858_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402

CASES = [
    ("rt1_2d_channels", 2, 1, 4, 4, 0.01, lambda n: inputs.channel_c(n, 4, 2)),
    ("rt0_2d_lognormal", 2, 0, 2, 5, 1.0, lambda n: inputs.lognormal_c(n, 2, 1.0, 4.0, 1)),
    ("rt0_3d_darcy", 3, 0, 2, 3, 0.0, lambda n: inputs.lognormal_c(n, 3, 3.0, 2.0, 3)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_handle_entry_point_twice(case):
    name, d, k, n0, L, mu, cf = case
    n = n0 * 2 ** (L - 1)
    c = torch.as_tensor(cf(n), device="cuda")
    G = mgdarcy.Multigrid(d, n0, L, k, mu, c, precision="fp64")
    ndof = G.ndof()
    rng = np.random.default_rng(3)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        x = torch.as_tensor(rng.standard_normal(ndof), device="cuda")
        b = torch.as_tensor(rng.standard_normal(ndof), device="cuda")
        expect = G.residual_norm(x, b)
        mgdarcy.residual_norm_noalloc(d, k, n, mu, c, x, b, out[call:call + 1])
        torch.cuda.synchronize()
        got = float(out[call].item())
        assert abs(got - expect) <= 1e-12 * expect, (call, got, expect)


def test_noalloc_rejects_levels_beyond_the_static_scratch():
    c = torch.ones(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 3000^2 cells of RT_1 is ~4.5e7 dofs, above the 16,777,216-dof limit
    with pytest.raises(mgdarcy.MGError) as e:
        mgdarcy.residual_norm_noalloc(2, 1, 3000, 0.1, c, x, x, x)
    assert e.value.status == 1
    assert "static scratch" in str(e.value)
