"""Host-side checks of the benchmark's roofline bookkeeping (no GPU): the
walk profile's machine-readable record, and the rule that its DRAM traffic is
reported only for the kernel sources it was captured on."""

import pytest

import bench


def _profile_record():
    rec_text = open(bench.WALK_PROFILE).read()
    import json
    import re
    m = re.search(r"<!-- traffic (\{.*?\}) -->", rec_text)
    assert m, "the walk profile has no machine-readable traffic record"
    return json.loads(m.group(1))


def test_profile_record_is_complete():
    rec = _profile_record()
    for key in ("kernel", "field", "receivers", "dram_read_bytes", "dram_write_bytes",
                "duration_ms", "l2_hit_pct", "lanes_active", "issue_active_pct",
                "sources_sha256"):
        assert key in rec, key
    assert rec["kernel"] == "k_walk"
    assert rec["receivers"] > 0 and rec["duration_ms"] > 0
    assert rec["dram_read_bytes"] > 0 and rec["dram_write_bytes"] > 0
    assert 0 < rec["lanes_active"] <= 32 and 0 < rec["issue_active_pct"] <= 100
    assert len(rec["sources_sha256"]) == 64


def test_sources_hash_covers_every_walk_source():
    """Changing any file the walk kernel is compiled from changes the hash."""
    import hashlib
    import os
    h = hashlib.sha256()
    csrc = os.path.join(bench.ROOT, "paper_2310_15235_gb300", "csrc")
    for name in ("walk.cu", "walk.cuh", "healpix.cuh", "internal.cuh"):
        h.update(open(os.path.join(csrc, name), "rb").read())
    h.update(open(os.path.join(bench.ROOT, "include", "trevr2.h"), "rb").read())
    assert bench.kernel_sources_sha256() == h.hexdigest()


def test_traffic_only_for_the_captured_sources(monkeypatch):
    rec = _profile_record()
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: rec["sources_sha256"])
    per = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / rec["receivers"]
    traffic, note = bench._walk_traffic(2 * rec["receivers"])
    assert traffic == pytest.approx(2 * per * rec["receivers"])
    assert "scaled by receivers" in note
    c = bench._walk_counters(6672.2)
    assert c["warp_execution_efficiency"] == pytest.approx(rec["lanes_active"] / 32)
    gbs = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / (rec["duration_ms"] * 1e-3) / 1e9
    assert c["dram_gbs"] == pytest.approx(gbs)

    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "0" * 64)
    traffic, note = bench._walk_traffic(rec["receivers"])
    assert traffic is None and "capture it again" in note
    assert bench._walk_counters(6672.2) is None
