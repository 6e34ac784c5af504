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
