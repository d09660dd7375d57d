"""The library's own measurements behind its rooflines and design choices:
the CUDA-core FMA rates (the FP64 mode's ALU roofline) and the cost of one
ordering point between dependent colour passes, as a software grid barrier in
one cooperative launch and as a dependent launch in a CUDA graph."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_04858_gb300 import mgdarcy  # noqa: E402


@pytest.mark.parametrize("kind,lo,hi", [("fp64", 0.1, 20.0), ("fp32", 1.0, 500.0), ("fp32x2", 1.0, 500.0)])
def test_fma_peak_is_plausible(kind, lo, hi):
    v = mgdarcy.measure_fma_peak(kind)
    assert math.isfinite(v) and lo < v < hi, v


def test_fma_peaks_order():
    """FP32 CUDA cores run many times the FP64 rate on this part."""
    assert mgdarcy.measure_fma_peak("fp32") > 10 * mgdarcy.measure_fma_peak("fp64")


@pytest.mark.parametrize("kind", ["grid_barrier", "dependent_launch"])
def test_sync_cost_is_measured(kind):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for nb in (nsm, 2 * nsm):
        v = mgdarcy.measure_sync_cost(kind, nb)
        assert math.isfinite(v) and 0.05 < v < 100.0, (kind, nb, v)


def test_grid_barrier_rejects_blocks_that_cannot_be_resident():
    with pytest.raises(mgdarcy.MGError) as e:
        mgdarcy.measure_sync_cost("grid_barrier", 65535)
    assert e.value.status == 1   # MG_ERR_INVALID_ARG
    # the device stays usable
    assert mgdarcy.measure_sync_cost("dependent_launch", 152) > 0
