"""The seeded input generators hold to their stated recipe (no GPU).

The synthetic fields stand in for the paper's figure-only binary fields and
for SPE10, so their structure is what the workloads claim: channels that are
two cells wide, continuous across the domain and at contrast 1e6; isolated
rectangular inclusions of the stated sizes, one cell apart, to 15 % cover;
a foam of many disconnected islands; Gaussian random fields with the stated
variance and squared-exponential correlation; refinement that keeps the
geometry.  The generators hold no arithmetic of the method.
"""
import numpy as np
import pytest
from scipy import ndimage

from paper_1602_04858_gb300 import inputs


def test_channels_are_two_cells_wide_and_cross_the_domain():
    n = 256
    m = inputs.channel_mask(n, 20, 2)
    up = np.zeros_like(m)
    up[1:] = m[:-1]
    down = np.zeros_like(m)
    down[:-1] = m[1:]
    assert np.all(~m | up | down)                       # every channel cell has a vertical partner
    assert m.sum(axis=0).min() >= 2                     # every column is crossed
    lab, nc = ndimage.label(m)                          # 4-connected pieces
    for comp in range(1, nc + 1):
        assert (lab[:, 0] == comp).any() and (lab[:, -1] == comp).any()
    c = inputs.channel_c(n, 20, 2)
    assert set(np.unique(c)) == {1.0, 1.0e6}
    assert np.array_equal(c == 1.0, m)


@pytest.mark.parametrize("n", [128, 256])
def test_inclusions_are_separated_rectangles(n):
    m = inputs.inclusions_mask(n, 11)
    assert 0.15 <= m.mean() < 0.17
    lab, nc = ndimage.label(m, structure=np.ones((3, 3)))   # touching diagonally counts as touching
    assert nc > 20
    for sl in ndimage.find_objects(lab):
        block = m[sl]
        assert block.all()                              # each piece is one filled rectangle
        assert max(2, n // 32) <= min(block.shape) and max(block.shape) <= max(3, n // 16)


@pytest.mark.parametrize("seed", [3, 11])
def test_foam_is_many_disconnected_islands(seed):
    m = inputs.foam_mask(128, seed)
    assert 0.05 < m.mean() < 0.2
    lab, nc = ndimage.label(m)
    assert nc > 30
    assert np.bincount(lab.ravel())[1:].max() < 0.2 * m.sum()   # no island dominates


def test_grf_variance_and_correlation():
    """Squared-exponential covariance sigma^2 exp(-r^2 / (2 ell^2)): the sample
    variance near sigma^2 and the correlation at lags ell and 2 ell near
    exp(-1/2) and exp(-2) (one seeded 512^2 field; finite-sample bounds)."""
    sigma, ell = 2.0, 8.0
    g = inputs.grf(512, 2, sigma, ell, 7)
    assert abs(g.mean()) < 0.1 * sigma
    assert 0.75 * sigma ** 2 < g.var() < 1.25 * sigma ** 2
    for lag, expect in ((int(ell), np.exp(-0.5)), (int(2 * ell), np.exp(-2.0))):
        rho = np.mean(g[:, :-lag] * g[:, lag:]) / g.var()
        assert abs(rho - expect) < 0.06, (lag, rho, expect)
    assert np.array_equal(inputs.lognormal_c(64, 2, sigma, ell, 7), np.exp(inputs.grf(64, 2, sigma, ell, 7)))


def test_refinement_keeps_the_geometry():
    a = inputs.channel_mask(32, 3, 5)
    r = inputs.refine_cells(a.astype(np.int8), 4)
    assert r.shape == (128, 128)
    for dy in range(4):
        for dx in range(4):
            assert np.array_equal(r[dy::4, dx::4], a)


def test_workloads_are_the_stated_problems():
    w = inputs.workload("channels_256")
    assert (w["d"], w["n_coarse"], w["n_levels"], w["degree"], w["mu"]) == (2, 4, 7, 1, 0.01)
    assert w["c"].shape == (256, 256) and w["c"].max() / w["c"].min() == 1.0e6
    w3 = inputs.workload("lognormal_3d_64")
    assert (w3["d"], w3["n_coarse"], w3["n_levels"], w3["degree"], w3["mu"]) == (3, 2, 6, 0, 0.0)
    assert w3["c"].shape == (64, 64, 64) and w3["c"].max() / w3["c"].min() > 1.0e5
    # the same seed gives the same field, another seed another one
    assert np.array_equal(inputs.channel_c(64, 4, 9), inputs.channel_c(64, 4, 9))
    assert not np.array_equal(inputs.channel_c(64, 4, 9), inputs.channel_c(64, 4, 10))
