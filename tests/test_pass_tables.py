"""Host construction of the colour-pass tables (Sec. 3.3), without a GPU.

The colour pass evaluates the rows of A on a patch from a sparse lane plan per
patch type (vertex next to the lower boundary, interior, next to the upper
boundary, or both, per direction) and gathers x, b and the cell coefficients
by contiguous segments.  mg_pass_tables_check builds these tables exactly as
mg_setup does and checks on the host that

* every row of every patch type is reproduced exactly (same columns, same
  coefficients) by the pieces its row map names, mass entries included;
* the plan evaluated on a random window and random cell coefficients agrees
  with the operator's row visitor evaluated directly (FP64: 1e-12, FP32
  tables: 1e-5 of the sum of the magnitudes of the terms);
* every segment entry gathers the window column, patch row or cell it stands
  for, zero outside the domain, and the patch-row segments name the window
  column of each row;
* the same for the tables of the block-per-patch pass: its four-thread row
  plans reproduce the row visitor, and its per-entry gather descriptors
  address every window column, patch row and cell exactly once;
* the operator row plans (one per class of rows, used by the apply and the
  residual kernels) evaluated for every free row of the level, as the kernels
  evaluate them, agree with the row visitor to 1e-13 of the row's sum of
  |terms| on random x and cell coefficients spanning e^-6 .. e^6, and address
  only entries and cells of the level.

Levels with n = 2 (one patch touching every side), n = 3 (only boundary
types) and n >= 4 (all types) are covered for every supported (d, k) (RT_2:
block-pass tables only; it has no warp pass), every
storage precision of the inverses and mu = 0 (Darcy) and mu > 0 (Brinkman).
"""
import pytest

from paper_1602_04858_gb300 import build as builder
from paper_1602_04858_gb300 import mgdarcy


@pytest.fixture(scope="module", autouse=True)
def lib():
    builder.build()
    return mgdarcy.load()


@pytest.mark.parametrize("dim,degree", [(2, 0), (2, 1), (2, 2), (3, 0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_bf16inv"])
@pytest.mark.parametrize("n", [2, 3, 4, 7, 16])
@pytest.mark.parametrize("mu", [0.0, 0.01, 1.0])
def test_tables_reproduce_the_operator(dim, degree, precision, n, mu):
    code, msg = mgdarcy.pass_tables_check(dim, degree, precision, n, mu)
    assert code == 0, msg


@pytest.mark.parametrize("args", [(4, 0, 1, 8, 0.0), (3, 1, 1, 8, 0.0), (2, 0, 7, 8, 0.0), (2, 0, 1, 1, 0.0),
                                  (2, 0, 1, 8, -1.0)])
def test_unsupported_arguments(args):
    code, _ = mgdarcy.pass_tables_check(*args)
    assert code == 2
