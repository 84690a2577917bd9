"""Host-side pieces of bench.py's reporting contract (no GPU): the DRAM traffic figure is
reported only while the measured kernel's source is the one the counters were taken from; the
whole-job throughput and the max-over-ranks time follow their definitions."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    # the committed figure matches the committed kernel source
    assert isinstance(bench.traffic_for("csr_spmm_f64_n64"), int)
    assert bench.traffic_for("no_such_kernel") is None
    # a copy of the tree whose kernel source differs by one byte: no traffic figure
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["csr_spmm_f64_n64"]
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    src = tmp_path / d["source"]
    src.parent.mkdir(parents=True)
    src.write_bytes(open(os.path.join(ROOT, d["source"]), "rb").read() + b"\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("csr_spmm_f64_n64") is None
    src.write_bytes(open(os.path.join(ROOT, d["source"]), "rb").read())
    assert bench.traffic_for("csr_spmm_f64_n64") == d["dram_bytes_per_launch"]


def test_whole_job_throughput_and_slowest_rank():
    # every rank processes its own replica: world x work / the step time
    assert bench.whole_job_gflops(2e9, 4, 1.0) == pytest.approx(8000.0)
    torch = pytest.importorskip("torch")
    assert bench.max_over_ranks(torch, 3.5, 1, "cpu") == 3.5
