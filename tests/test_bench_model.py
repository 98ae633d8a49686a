"""Host arithmetic of the benchmark's roofline object: the algorithmic bytes of
each kernel class (the hot-path scope table's per-particle figures) and the
lookup of the ncu DRAM traffic, which must be withheld once the kernels differ
from the ones the counters were taken on."""
from __future__ import annotations

import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_algorithmic_bytes_match_the_scope_table():
    # k = 29 list entries and no window particles: 428 B per particle-step for the
    # count, chain and force passes with the BAOAB update (rebuilds amortised apart)
    b = bench.class_bytes_per_particle(29.0, 0.0)
    assert b["chain"] == 0.0
    assert b["count"] + b["chain"] + b["force"] == pytest.approx(428.0)
    # the chain-rule pre-pass walks the window fraction only
    assert bench.class_bytes_per_particle(29.0, 0.25)["chain"] == pytest.approx(0.25 * (4 * 29 + 32))
    assert b["rebuild"] == pytest.approx(4 * 29 + 48)


def test_traffic_only_for_the_profiled_kernels(tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic("count", 1000) is None  # no summary
    f.write_text(json.dumps({"kernel_sources_sha256_16": bench.kernel_hash(),
                             "dram_bytes_per_particle": {"count": 99.5}}))
    assert bench.ncu_traffic("count", 1000) == pytest.approx(99_500.0)
    assert bench.ncu_traffic("force", 1000) is None  # a class that was not captured
    f.write_text(json.dumps({"kernel_sources_sha256_16": "0" * 16,
                             "dram_bytes_per_particle": {"count": 99.5}}))
    assert bench.ncu_traffic("count", 1000) is None  # kernels changed since the capture


def test_committed_summary_names_its_command_and_kernels():
    with open(bench.TRAFFIC_FILE) as fh:
        t = json.load(fh)
    assert t["command"].startswith("ncu ") and "--clock-control none" in t["command"]
    assert set(t["dram_bytes_per_particle"]) == {"count", "chain", "force", "rebuild"}
    assert len(t["kernel_sources_sha256_16"]) == 16
