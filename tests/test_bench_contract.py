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
    # the committed figures match the committed kernel sources
    d_all = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key in d_all:
        assert isinstance(bench.traffic_for(key), int), key
    assert bench.traffic_for("no_such_kernel") is None
    # a copy of the tree in which one of the captured sources differs by one byte: no figure
    key = sorted(d_all)[0]
    d = d_all[key]
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    srcs = list(d["sources"])
    for src in srcs:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, src), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for(key) == d["dram_bytes_per_launch"]
    last = tmp_path / srcs[-1]
    last.write_bytes(open(os.path.join(ROOT, srcs[-1]), "rb").read() + b"\n")
    assert bench.traffic_for(key) is None
    last.write_bytes(open(os.path.join(ROOT, srcs[-1]), "rb").read())
    assert bench.traffic_for(key) == d["dram_bytes_per_launch"]


def test_whole_job_throughput_and_slowest_rank():
    # every rank processes its own replica: world x work / the step time
    assert bench.whole_job_gflops(2e9, 4, 1.0) == pytest.approx(8000.0)
    torch = pytest.importorskip("torch")
    assert bench.max_over_ranks(torch, 3.5, 1, "cpu") == 3.5
