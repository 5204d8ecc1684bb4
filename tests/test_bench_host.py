"""Host-side logic of bench.py: the lookup of the committed DRAM-traffic
record (exact workload and velocity width, or scaled by particles from a
record of the same velocity width; nothing once the kernels changed) and the
end-to-end step-interval summary."""
import json
import os

import bench


def _record(tmp_path, entries):
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": entries}))


def test_recorded_traffic_lookup(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda kind=None: "d1")
    _record(tmp_path, [
        {"kind": "ikd_count", "workload": "w256", "vel_bits": 8, "particles": 100, "scale": "particles",
         "bytes_per_launch": 1000, "csrc": "d1"},
        {"kind": "ikd_count", "workload": "w256", "vel_bits": 16, "particles": 100, "scale": "particles",
         "bytes_per_launch": 1500, "csrc": "d1"},
        {"kind": "fft_a_tiles", "workload": "w256", "vel_bits": 8, "particles": 100,
         "bytes_per_launch": 7, "csrc": "d1"},
        {"kind": "deposit", "workload": "w256", "vel_bits": 8, "particles": 100, "scale": "particles",
         "bytes_per_launch": 9, "csrc": "old"},
    ])
    # exact workload: the entry of the same velocity width
    assert bench.recorded_traffic("ikd_count", "w256", 100, 8) == {"bytes": 1000, "captured_on": "w256",
                                                                   "scaled": False}
    assert bench.recorded_traffic("ikd_count", "w256", 100, 16)["bytes"] == 1500
    # another workload: scaled by the particles, only from the same velocity width
    r = bench.recorded_traffic("ikd_count", "big", 4000, 16)
    assert r == {"bytes": 60000, "captured_on": "w256", "scaled": True}
    # kinds whose traffic does not scale with particles, and stale records, give nothing
    assert bench.recorded_traffic("fft_a_tiles", "big", 4000, 8) is None
    assert bench.recorded_traffic("deposit", "w256", 100, 8) is None


def test_gap_summary():
    s = bench.gap_summary([600.0, 380.0, 390.0, 370.0, 400.0])
    assert s == {"first_step_ms": 600.0, "steady_ms_per_step": 390.0}
    assert bench.gap_summary([5.0]) == {"first_step_ms": 5.0, "steady_ms_per_step": None}


def test_kind_digests_cover_their_sources():
    # every kernel kind of the traffic record has its own digest, and kinds
    # built from the same sources share it
    assert bench.csrc_digest("ikd_count") == bench.csrc_digest("deposit")
    assert bench.csrc_digest("fft_a_tiles") == bench.csrc_digest("fft_c_tiles")
    assert bench.csrc_digest("ikd_count") != bench.csrc_digest("fft_a_tiles")
    assert bench.csrc_digest() not in (bench.csrc_digest("ikd_count"), bench.csrc_digest("fft_a_tiles"))
