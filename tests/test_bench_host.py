"""Host-side pieces of bench.py (no GPU): the algorithmic byte count behind
the roofline figure and the batched workload recipe."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_colour_pass_bytes_of_the_finest_pass():
    # 7,225 patches of n_v = 40: the 40 x 40 FP32 inverse once, b_v and x_v read, x_v written
    assert bench.colour_pass_bytes(7225, 40, 4, 4) == 7225 * (1600 * 4 + 3 * 40 * 4) == 49_708_000


def test_traffic_figure_is_close_to_the_algorithmic_bytes():
    algo = bench.colour_pass_bytes(7225, 40, 4, 4)
    assert algo <= bench.FINEST_PASS_DRAM_BYTES <= 1.05 * algo


def test_batched_workload_recipe():
    probs = bench.batched_workload(per_size=2)
    assert [p["c"].shape[0] for p in probs] == [64, 64, 128, 128, 256, 256, 512, 512]
    assert all(p["n_levels"] == int(np.log2(p["c"].shape[0] // 4)) + 1 for p in probs)
    # a subset of the sizes keeps the same problems (seeds count all sizes)
    sub = bench.batched_workload(per_size=2, sizes=(128, 512), pass_kernel=2)
    assert [p["c"].shape[0] for p in sub] == [128, 128, 512, 512]
    assert np.array_equal(sub[0]["c"], probs[2]["c"]) and np.array_equal(sub[3]["c"], probs[7]["c"])
    assert all(p["pass_kernel"] == 2 for p in sub)
    # lognormal fields with sigma in [1, 3]: positive, finite, not constant
    for p in probs:
        assert np.all(p["c"] > 0) and np.all(np.isfinite(p["c"])) and p["c"].std() > 0
