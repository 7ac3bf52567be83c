"""The DRAM traffic the benchmark reports comes from committed ncu records
keyed by a hash of the kernel and BVH-builder sources: every record must be
consistent in itself, the benchmark uses a record only while it belongs to
the current sources, and a record of other sources is ignored (reported as
null) rather than used."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_records_are_consistent():
    for name in ("trace_kernel_traffic.json", "trace_kernel_building_traffic.json"):
        d = json.load(open(os.path.join(ROOT, "profiles", name)))
        assert len(d["kernel_source_sha256_16"]) == 16, name
        assert d["passes"] == 1 and "--clock-control none" in d["command"]
        for k in ("trace_kernel_forward", "trace_kernel_adjoint"):
            r = d[k]
            per = (r["dram_read_bytes"] + r["dram_write_bytes"]) / r["segments"]
            assert abs(per - r["dram_bytes_per_segment"]) <= 1e-4 * per + 1e-4, (name, k)


def test_a_record_of_other_sources_is_ignored(monkeypatch):
    d = json.load(open(bench.TRAFFIC_FILE))
    monkeypatch.setattr(bench, "kernel_hash", lambda: d["kernel_source_sha256_16"])
    assert bench.stored_traffic("trace_kernel_adjoint") == d["trace_kernel_adjoint"]["dram_bytes_per_segment"]
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.stored_traffic("trace_kernel_adjoint") is None
