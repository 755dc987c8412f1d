"""Host logic of bench.py (CPU): the executed-work model behind
roofline.achieved (per pipe), the validity rule of the committed DRAM traffic,
the parsing of nvidia-smi clock samples, and the reference arm's JSON line (the
FP64 oracle on a bounded sample of the 64-primitive workload)."""
import argparse

import pytest


def test_work_model_counts():
    import bench
    ns, nc = 16, 32
    fwd, bwd = bench.work_per_unit(ns, nc, colour_store=True)
    # (FP32 lane-ops, tensor multiply-adds, MUFU ops) per unit
    assert fwd["cand"] == (28, 0, 0)
    assert fwd["hit"] == (29 + 15 * ns, 0, 2 + 3 * ns)
    assert fwd["comp"] == (10 + 6 * nc + 3, nc * nc, 8)      # the hidden layer is tensor-core work
    # the backward tests no candidates and, with the colour store, replays no alpha_hat
    assert bwd["cand"] == (0, 0, 0) and bwd["hit"] == (0, 0, 0)
    assert bwd["comp"] == (177 + 40 * ns + 14 * nc, 3 * nc * nc, 3 + 5 * ns)
    _, bwd_replay = bench.work_per_unit(ns, nc, colour_store=False)
    assert bwd_replay["comp"][0] == bwd["comp"][0] + 28 + 29 + 15 * ns + 6 * nc + 3
    assert bwd_replay["comp"][1] == 4 * nc * nc
    f0, b0 = bench.work_per_unit(8, 0, colour_store=True)   # no colour network: alpha_hat store
    assert f0["comp"] == (10, 0, 2) and b0["comp"] == (177 + 40 * 8, 0, 3 + 5 * 8)
    _, b0r = bench.work_per_unit(8, 0, colour_store=False)  # alpha_hat replayed
    assert b0r["comp"][0] == 177 + 40 * 8 + 28 + 29 + 15 * 8
    counts = {"cand": 1000, "hit": 400, "comp": 100}
    fp32, tensor, mufu = bench.kernel_work(counts, fwd)
    assert fp32 == 2.0 * (1000 * 28 + 400 * (29 + 15 * ns) + 100 * (10 + 6 * nc + 3))
    assert tensor == 2.0 * 100 * nc * nc and mufu == 400 * (2 + 3 * ns) + 100 * 8
    peaks = {"fp32_tflops": 80.0, "tensor_tflops": 1700.0, "mufu_tops": 5.0, "hbm_gbs": 6800.0}
    roof = bench.pipe_roofline((80e9, 17e9, 5e9), 10.0, 6.8e9, peaks)   # 10 ms
    assert roof["fp32"]["frac"] == 0.1 and roof["tensor"]["frac"] == 0.001
    assert roof["mufu"]["frac"] == 0.1 and roof["hbm"]["frac"] == 0.1


def test_traffic_is_dropped_when_the_kernels_change(tmp_path, monkeypatch):
    import json
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"workload": "w", "sources": bench.raster_sources_digest(),
                                                    "k_raster_bwd": {"bytes_per_launch": 7}}))
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "raster_sources_digest", lambda: json.loads((prof / "traffic.json").read_text())["sources"])
    assert bench.raster_traffic("w") == {"k_raster_bwd": 7}
    assert bench.raster_traffic("other") == {}
    monkeypatch.setattr(bench, "raster_sources_digest", lambda: "changed")
    assert bench.raster_traffic("w") == {}
    monkeypatch.setattr(bench, "ROOT", real_root)


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
