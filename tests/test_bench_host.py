"""Host-side logic of bench.py (CPU): the DRAM-traffic figure is reported
only while the committed ncu summary was taken on the current kernel
sources, and is scaled to the grid by the cells a launch processes."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_tree(tmp_path, source_text):
    csrc = tmp_path / "paper_1907_07774_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_text(source_text)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    root = _fake_tree(tmp_path, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic("op_axis01", 256) is None          # no summary yet
    h = bench.csrc_hash()
    summary = {"csrc_hash": h, "classes": {"op_axis01": {"bytes_per_launch": 2.0e8, "cells": 256 ** 3}}}
    (root / "profiles" / "ncu_traffic.json").write_text(json.dumps(summary))
    assert bench.ncu_traffic("op_axis01", 256) == 2.0e8
    # scaled by the cells of the launch (a smaller capture stands for a full launch)
    summary["classes"]["op_axis01"]["cells"] = 128 ** 3
    (root / "profiles" / "ncu_traffic.json").write_text(json.dumps(summary))
    assert bench.ncu_traffic("op_axis01", 256) == 2.0e8 * 8
    assert bench.ncu_traffic("pcg_opx", 256) is None            # class not captured
    # any change of the kernel sources withdraws the figure
    (root / "paper_1907_07774_gb300" / "csrc" / "k.cuh").write_text("kernel v2")
    assert bench.csrc_hash() != h
    assert bench.ncu_traffic("op_axis01", 256) is None


def test_committed_summary_names_a_captured_kernel_class():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    assert len(d["csrc_hash"]) == 16
    for ent in d["classes"].values():
        assert ent["bytes_per_launch"] > 0 and ent["cells"] > 0 and ent["kernel"]


def test_oracle_work_comes_from_the_stored_oracle_run(tmp_path, monkeypatch):
    """The CPU baseline scales its per-iteration sample by the oracle's own PCG
    work, read from the stored full oracle run; without one there is none."""
    monkeypatch.setattr(bench, "GOLDEN", str(tmp_path))
    assert bench.oracle_work(256, 32) is None
    run = {"pcg_iters_forward": [3, 4, 5], "pcg_iters_adjoint": [20, 21, 22], "seconds_gradient": 9.0}
    (tmp_path / "oracle_full_work256_nt32_rtol1e-6.json").write_text(json.dumps(run))
    w = bench.oracle_work(256, 32)
    assert w["iters"] == 75 and w["solves"] == 6
    v, t = bench.cpu_cells_per_s(256, 32, 2.0, 0.5, w["iters"], w["solves"])
    assert t == 75 * 2.5 + 6 * 2.5 + 32 * 0.75 * 2.0
    assert v == 256 ** 3 * 32 / t


def test_reference_arm_without_stored_work_prints_unavailable(tmp_path, monkeypatch, capsys):
    import argparse
    monkeypatch.setattr(bench, "GOLDEN", str(tmp_path))
    args = argparse.Namespace(n=256, nt=32, warmup=1, steps=1, gpus=1)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_reference_arm_measures_the_same_config_as_ours(monkeypatch, capsys):
    """Both arms time the same workload: the reference line carries the very
    config dict of our arm (the oracle's arithmetic goes in its own keys).
    The oracle sample is replaced by fixed times so that nothing heavy runs."""
    import argparse
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda n, nt, k_f: (2.5, 0.75))
    args = argparse.Namespace(n=256, nt=32, warmup=0, steps=1, gpus=1, ckpt_stride=0)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == bench.gradient_config(256, 32, bench.GRADIENT_GAUSSIANS, 0, 1)
    assert line["e2e"]["value"] == line["value"] == line["cpu_baseline"]["value"]


def test_cpu_model_is_a_string():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
