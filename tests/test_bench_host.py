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


def test_vcycle_model_by_hand():
    """Two levels (J = 2), variable cycle with m(J) = 2: m(2) = 2, m(1) = 4;
    2-D, C = 9 colours, so a sweep count of 2 m (2C - 1)/C = 68/9 on the finest
    level and 136/9 on level 1."""
    lv = [(50, 1, 8, 30), (200, 9, 8, 40)]   # (dofs, patches, n_v, nnz)
    big = 1 << 40
    b, f = bench.vcycle_model(lv, 2, "fp32", big)
    s1, s2 = 136 / 9, 68 / 9
    expect_b = (1 * 64 * 4 + s1 * 3 * 50 * 4 + 6 * 50 * 4) + (9 * 64 * 4 + s2 * 3 * 200 * 4 + 6 * 200 * 4)
    expect_f = s1 * 1 * (2 * 64 + 60) + s2 * 9 * (2 * 64 + 80)
    assert abs(b - expect_b) < 1e-9 * expect_b and abs(f - expect_f) < 1e-9 * expect_f
    # an L2 smaller than the finest inverses: those are streamed once per sweep
    b_small, _ = bench.vcycle_model(lv, 2, "fp32", 1000)
    assert abs(b_small - (expect_b + (s2 - 1) * 9 * 64 * 4)) < 1e-9 * b_small
    # FP64 doubles every byte; BF16 inverses halve the finest level's inverse bytes only
    assert abs(bench.vcycle_model(lv, 2, "fp64", big)[0] - 2 * expect_b) < 1e-9 * expect_b
    b_bf, _ = bench.vcycle_model(lv, 2, "fp32_bf16inv", big)
    assert abs(b_bf - (expect_b - 9 * 64 * 2)) < 1e-9 * expect_b
    # the standard cycle: m = 2 on both levels
    b_std, _ = bench.vcycle_model(lv, 2, "fp32", big, variable=False)
    assert abs(b_std - (expect_b - (s1 - s2) * 3 * 50 * 4)) < 1e-9 * expect_b


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


def test_workload_configs_name_their_degree():
    """The default and the RT_2 workload describe themselves; the traffic
    figures are keyed by workload and the finest level's kernel."""
    assert bench.workload_config()["degree"] == 1
    old = bench.WORKLOAD
    try:
        bench.WORKLOAD = "channels_256_rt2"
        assert bench.workload_config()["degree"] == 2
    finally:
        bench.WORKLOAD = old
    assert set(bench.FINEST_PASS_DRAM_BYTES) <= {("channels_256", "warp"), ("channels_256_rt2", "persistent blocks"),
                                                 ("lognormal_3d_64", "warp")}
    # each traffic figure lies within 25 % above its algorithmic bytes
    # (7,225 patches of 40 or 96 dofs; 9,261 of 20 in 3-D)
    for (wl, _), t in bench.FINEST_PASS_DRAM_BYTES.items():
        npat, nv = {"channels_256": (7225, 40), "channels_256_rt2": (7225, 96), "lognormal_3d_64": (9261, 20)}[wl]
        alg = bench.colour_pass_bytes(npat, nv, 4, 4)
        assert alg <= t <= 1.25 * alg


def test_traffic_figures_are_the_committed_captures():
    """Each traffic figure bench.py reports is the DRAM read + write of one
    launch in the committed ncu summary of that workload's finest pass."""
    import re
    prof = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    files = {"channels_256": "colour_pass_channels256_fp32.md",
             "channels_256_rt2": "colour_pass_channels256_rt2_fp32.md",
             "lognormal_3d_64": "colour_pass_lognormal64_3d_fp32.md"}
    for (wl, _), t in bench.FINEST_PASS_DRAM_BYTES.items():
        with open(os.path.join(prof, files[wl])) as f:
            m = re.search(r"DRAM traffic: ([0-9.]+) MB per launch", f.read())
        assert m, files[wl]
        assert abs(t / 1e6 - float(m.group(1))) < 0.006


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """bench.py --impl reference: one JSON line with the keys of the benchmark
    contract, the reference arm's own cpu_baseline and e2e objects, and the
    metric, unit and direction of the GPU arm (here on the 16^2 workload so
    that the oracle finishes at once; the real run uses the 256^2 one)."""
    import json
    import types
    monkeypatch.setattr(bench, "WORKLOAD", "small_2d")
    bench.reference_arm(types.SimpleNamespace(gpus=1, steps=2, warmup=1), 0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
    # other ranks print nothing
    bench.reference_arm(types.SimpleNamespace(gpus=2, steps=1, warmup=0), 1)
    assert capsys.readouterr().out.strip() == ""
