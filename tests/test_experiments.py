"""The driven-flow experiments of Sec. 4.1 (boundary velocity g = (1, 0), f = 0).

experiments.py solves them as u = u_g + u_0: u_g = g everywhere and u_0 with
homogeneous boundary values and body force -c g.  The CPU test checks that
identity on the oracle (its own load vector with the boundary data of
eq. (BCh), lifted, against the homogeneous problem plus the constant field),
which pins the reformulation independently of the CUDA path; the GPU test
checks the CUDA solve of u_0 plus the lift against the oracle's direct solve
of the driven problem.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import fem
from oracle import multigrid as mg
from paper_1602_04858_gb300 import experiments, inputs


def direct(L, b):
    """A x = b on the free dofs with zero weighted pressure mean (bordered LU)."""
    fr = L.free
    w = L.w[fr]
    M = sp.bmat([[L.A[fr][:, fr], sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]]).tocsc()
    y = spl.splu(M).solve(np.concatenate([b[fr], [0.0]]))
    x = b.copy()
    x[fr] = y[:-1]
    return x


def small_field(n, seed):
    m = inputs.inclusions_mask(n, seed, fraction=0.2)
    return np.where(m, 1.0e3, 1.0)


def test_constant_lift_reproduces_the_driven_problem_3d():
    n = 4
    c = np.exp(np.random.default_rng(5).standard_normal((n, n, n)))
    L = mg.Level(fem.Space(3, n, 0), 0.01, c, with_patches=False)
    g = np.array([0.0, 1.0, 0.0])
    x_drv = direct(L, fem.load_vector(L.S, 0.01, c, g=lambda X: np.tile(g, (X.shape[0], 1))))
    x_0 = direct(L, fem.load_vector(L.S, 0.01, c, f=lambda X, cv: np.tile(-cv * g, (X.shape[0], 1))))
    x = experiments.add_lift(x_0, n, 0, tuple(g))
    assert np.max(np.abs(x - x_drv)) <= 1e-10 * np.max(np.abs(x_drv))


@pytest.mark.parametrize("degree", [0, 1, 2])
@pytest.mark.parametrize("mu", [0.0, 0.01, 1.0])
def test_constant_lift_reproduces_the_driven_problem(mu, degree):
    n = 8
    c = small_field(n, 3)
    L = mg.Level(fem.Space(2, n, degree), mu, c, with_patches=False)
    g = np.array([1.0, 0.0])
    b_drv = fem.load_vector(L.S, mu, c, g=lambda X: np.tile(g, (X.shape[0], 1)))
    x_drv = direct(L, b_drv)
    b_0 = fem.load_vector(L.S, mu, c, f=lambda X, cv: np.tile(-cv * g, (X.shape[0], 1)))
    x_0 = direct(L, b_0)
    x = experiments.add_lift(x_0, n, degree, g)
    assert np.max(np.abs(x - x_drv)) <= 1e-10 * np.max(np.abs(x_drv))
    # the driven velocity carries the boundary flux: u.n = 1 on the left and right walls
    N = n * (degree + 1)
    ux = x[:(N + 1) * N].reshape(N, N + 1)
    assert np.allclose(ux[:, 0], 1.0) and np.allclose(ux[:, -1], 1.0)


def test_case_coefficients():
    ca = experiments.coefficient("inclusions", "a", 1e4, 256)
    cb = experiments.coefficient("inclusions", "b", 1e4, 256)
    assert ca.shape == (256, 256)
    assert set(np.unique(ca)) == {1.0, 1e4} and np.array_equal(ca * cb, np.full_like(ca, 1e4))
    # refinement keeps the geometry: the 256^2 field is the 128^2 one with cells split 2 x 2
    c128 = experiments.coefficient("connected", "a", 1e5, 128)
    assert np.array_equal(experiments.coefficient("connected", "a", 1e5, 256)[::2, ::2], c128)


@pytest.mark.gpu
@pytest.mark.parametrize("mu", [0.0, 0.01])
@pytest.mark.parametrize("geometry", ["foam", "connected"])
def test_driven_solve_matches_oracle(geometry, mu):
    torch = pytest.importorskip("torch")
    n = 16
    c = experiments.coefficient(geometry, "a", 1e4, n, n0=16)
    st, x, _ = experiments.driven_solve(torch, c, mu, tol=1e-11, precision="fp64", n_coarse=2)
    assert st.converged == 1
    xg = experiments.add_lift(x.cpu().numpy(), n)
    L = mg.Level(fem.Space(2, n, 0), mu, c, with_patches=False)
    x_drv = direct(L, fem.load_vector(L.S, mu, c, g=lambda X: np.tile([1.0, 0.0], (X.shape[0], 1))))
    assert np.linalg.norm(xg - x_drv) <= 1e-6 * np.linalg.norm(x_drv)
