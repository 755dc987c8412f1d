"""Host logic of bench.py (CPU): the algorithmic work model behind
roofline.achieved, the parsing of nvidia-smi clock samples, and the reference
arm's JSON line (the FP64 oracle on a bounded sample of the 64-primitive
workload)."""
import argparse

import pytest


def test_work_model_counts():
    import bench
    fwd, bwd = bench.fma_per_unit(16, 32)
    mlp = (3 + 8) * 32 + 32 * 32 + 3 * 32          # first layer, hidden layer, output layer
    assert mlp == 1472
    assert fwd == {"cand": 21, "hit": 12 + 12 * 16, "comp": 10 + mlp}
    assert bwd["comp"] == 10 + 3 * mlp + 24 * 16 + 80 and bwd["hit"] == fwd["hit"]
    f0, _ = bench.fma_per_unit(8, 0)
    assert f0["comp"] == 10                          # no colour network
    counts = {"cand": 1000, "hit": 400, "comp": 100}
    assert bench.flops(counts, fwd) == 2.0 * (1000 * 21 + 400 * 204 + 100 * 1482)


def test_clock_summary_median_and_reasons():
    import bench
    c = bench.ClockSampler()
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler().summary() is None


def test_reference_arm_json_line():
    import bench
    args = argparse.Namespace(workload="tiny64_128px", steps=1, warmup=0, ref_tiles=2)
    res = bench.run_reference(args, rank=0, world=1)
    assert res["impl"] == "reference" and res["unit"] == "Mpixel/s" and res["value"] > 0
    assert res["cpu_baseline"]["kind"] == "oracle" and res["cpu_baseline"]["cores"] >= 1
    assert res["e2e"]["h2d_bytes_per_step"] == 0 and res["e2e"]["value"] == res["value"]
    assert bench.run_reference(args, rank=1, world=2) is None   # other ranks do no work
