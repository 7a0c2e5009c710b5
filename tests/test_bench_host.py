"""Host logic of bench.py that needs no GPU: the DRAM traffic figure of the roofline entry is reported
only while the ncu capture it comes from still describes the timed kernel (same source text) and the
timed workload (same number of unknowns and band applications per unknown)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record():
    return json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["kernels"]["pass_f64"]


def test_traffic_reported_on_the_captured_shape():
    rec = _record()
    assert bench.traffic_for("pass_f64", rec["shape"]) == rec["dram_bytes_per_launch"]
    assert rec["dram_bytes_per_launch"] == sum(rec["per_launch_bytes"]) / len(rec["per_launch_bytes"])


def test_traffic_void_on_another_workload():
    shape = dict(_record()["shape"])
    shape["band_apps_per_dof"] -= 5
    assert bench.traffic_for("pass_f64", shape) is None
    shape = dict(_record()["shape"])
    shape["n_dof"] *= 8
    assert bench.traffic_for("pass_f64", shape) is None


def test_traffic_void_once_the_kernel_source_changes(monkeypatch):
    rec = _record()
    monkeypatch.setattr(bench, "source_hash", lambda span: "0" * 16)
    assert bench.traffic_for("pass_f64", rec["shape"]) is None


def test_traffic_void_for_a_kernel_without_a_capture():
    assert bench.traffic_for("modeprod2d_f32", _record()["shape"]) is None
