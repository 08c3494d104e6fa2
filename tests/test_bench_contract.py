"""The JSON line of bench.py's reference arm (the FP64 oracle timed on the host cores):
the keys and values the benchmark contract asks for, with the oracle's rate stubbed so
that the check takes no CPU time (no GPU)."""

import argparse

import numpy as np

import bench


def _fake_rate(workload, budget_s, processes=None, eps=None):
    _fake_rate.calls.append((workload, budget_s))
    _fake_rate.eps = eps
    return {"value": 2.0e6, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
            "sample": f"stub of {workload}"}


def test_reference_line_keeps_the_contract(monkeypatch):
    _fake_rate.calls = []
    monkeypatch.setattr(bench, "cpu_oracle_rate", _fake_rate)
    args = argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, steps=2, warmup=3, gpus=1)
    line = bench.run_reference(args)
    assert len(_fake_rate.calls) == 5                        # warm-up samples are taken, not counted
    assert all(b >= 2.0 for _, b in _fake_rate.calls)        # each step a bounded sample
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT == "poses/s"
    assert line["value"] == 2.0e6 and line["higher_is_better"] is True
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["scaling"] == "weak" and line["vs_baseline"] is None and line["data"] == "synthetic"
    assert line["dtype"] == "f64"
    assert "8192 images x 4096 templates" in line["config"]["workload"]
    poses = 8192 * 4096 * 384 * 797
    assert abs(line["ms_per_step"] - poses / 2.0e6 * 1e3) < 1e-6 * line["ms_per_step"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] == 16 and cb["sample"]
    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_line_follows_an_overridden_precision_target(monkeypatch):
    # config 3 names eps = 1e-3 and 1e-4: with --eps the oracle legs build their plan at it
    _fake_rate.calls = []
    monkeypatch.setattr(bench, "cpu_oracle_rate", _fake_rate)
    line = bench.run_reference(argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, steps=1, warmup=0, gpus=1,
                                                  eps=1e-4))
    assert _fake_rate.eps == 1e-4
    assert "eps=0.0001" in line["config"]["workload"]


def test_reference_line_for_the_uneven_groups_samples_its_first_group(monkeypatch):
    _fake_rate.calls = []
    monkeypatch.setattr(bench, "cpu_oracle_rate", _fake_rate)
    from workloads import BATCH_GROUPS
    line = bench.run_reference(argparse.Namespace(workload="batch4", steps=1, warmup=0, gpus=1))
    assert {w for w, _ in _fake_rate.calls} == {BATCH_GROUPS[0]}
    assert line["value"] == 2.0e6


def test_roofline_work_per_kernel_counts_the_algorithmic_terms():
    # Step 3 (and the fused Steps 2-3): 4 N H 2Q flops per pair with H the rank over all
    # orders; Step 1: 8 H M 2Q; "executed" counts the H' terms of orders l >= 0 instead
    class P:
        N, two_Q, M, H, H_half = 441, 192, 32, 82, 44

    class W:
        images = np.zeros((3, 1, 1))
        templates = np.zeros((5, 1, 1))

    for k in ("step3_tc", "step23_tc", "step23c_tc", "step3_simt"):
        assert bench.kernel_work(k, P, W) == ("flops", 15 * 4 * 441 * 82 * 192)
        assert bench.kernel_work(k, P, W, terms="executed") == ("flops", 15 * 4 * 441 * 44 * 192)
    assert bench.kernel_work("step1_tc", P, W) == ("flops", 15 * 8 * 82 * 32 * 192)
    assert bench.kernel_work("fft_pack", P, W) == ("bytes", 15 * 44 * 192 * 16)
    assert bench.kernel_work("no_such_kernel", P, W) == (None, None)


def test_ncu_traffic_is_dropped_once_the_kernel_source_changed(monkeypatch, tmp_path):
    import json
    import os
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1905_12317_gb300" / "csrc").mkdir(parents=True)
    src = tmp_path / "paper_1905_12317_gb300" / "csrc" / "k_step23_tc.cu"
    src.write_text("// kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.src_hash("step23_tc")
    g64 = {"n": 64, "two_Q": 192, "N": 441}
    g128 = {"n": 128, "two_Q": 384, "N": 797}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"step23_tc": [
        {"grid": g64, "dram_bytes_per_pair": 100.0, "src_sha": sha},
        {"grid": g128, "dram_bytes_per_pair": 300.0, "src_sha": sha}]}))
    assert bench.ncu_traffic("step23_tc", 7, g64) == 700.0
    assert bench.ncu_traffic("step23_tc", 7, g128) == 2100.0
    assert bench.ncu_traffic("step23_tc", 7, {"n": 32, "two_Q": 96, "N": 9}) is None  # no capture on this grid
    src.write_text("// kernel v2\n")                 # changed since the counters were taken
    assert bench.ncu_traffic("step23_tc", 7, g64) is None
    assert bench.ncu_traffic("step1_tc", 7, g64) is None   # no entry
    os.remove(tmp_path / "profiles" / "ncu_traffic.json")
    assert bench.ncu_traffic("step23_tc", 7, g64) is None  # no table
