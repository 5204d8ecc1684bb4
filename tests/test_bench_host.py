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


def test_byte_models_give_the_documented_figures():
    """The algorithmic bytes per launch and the whole-step model that the
    rooflines divide, for the 256^3 workload (64 tiles of 64^3 + 16, 128^3
    CDM + 256^3 nu, 8-bit codes, compression = coarse ratio 4) and the 1536^3
    one (13,824 tiles in launches of 256, 768^3 + 1536^3 particles, 16-bit
    codes), worked out here from the per-unit figures: 3 B position codes +
    1 B count byte per compression cell and species read and 4 B per fine and
    coarse cell written (deposit); 3 (1 + vb) B of codes + 12 B per fine and
    coarse force cell read (count pass); 3 (1 + vb) B written (scatter);
    T^3 4 + T^2 (T/2 + 1) 8 (pass A), T^2 (T/2 + 1) 8 + 3 t T (T/2 + 1) 8
    (pass B), 3 t T (T/2 + 1) 8 + 3 t^3 4 (pass C) per tile."""
    cfg = dict(n_fine=256, coarse_ratio=4, cmp_ratio=4, tile=64, buffer=16, tile_batch=64)
    counts = (128 ** 3, 256 ** 3)
    a = bench.algorithmic_bytes(cfg, counts, 8)
    n = 128 ** 3 + 256 ** 3
    assert a["deposit"] == 3 * n + 2 * 64 ** 3 + 4 * (256 ** 3 + 64 ** 3) == 125_304_832
    assert a["ikd_count"] == 6 * n + 12 * (256 ** 3 + 64 ** 3) == 317_718_528
    assert a["ikd_scatter"] == 6 * n == 113_246_208
    assert a["fft_a_tiles"] == 64 * (96 ** 3 * 4 + 96 * 96 * 49 * 8)
    assert a["fft_b_tiles"] == 64 * (96 * 96 * 49 * 8 + 3 * 64 * 96 * 49 * 8)
    assert a["fft_c_tiles"] == 64 * (3 * 64 * 96 * 49 * 8 + 3 * 64 ** 3 * 4)
    # the whole step: 15 B per particle, 40 B per tile cell and coarse cell, the kernels once
    assert bench.step_model_bytes(cfg, counts, 8) == (15 * n + 40 * (64 * 96 ** 3 + 64 ** 3)
                                                      + 2 * 64 ** 3 + 12 * 96 * 96 * 49) == 2_564_468_736

    big = dict(n_fine=1536, coarse_ratio=4, cmp_ratio=4, tile=64, buffer=16, tile_batch=256)
    nb = 768 ** 3 + 1536 ** 3
    b = bench.algorithmic_bytes(big, (768 ** 3, 1536 ** 3), 16)
    assert b["ikd_count"] == 9 * nb + 12 * (1536 ** 3 + 384 ** 3) == 80_857_792_512
    assert b["ikd_scatter"] == 9 * nb
    assert b["fft_c_tiles"] == 256 * (3 * 64 * 96 * 49 * 8 + 3 * 64 ** 3 * 4)
    assert bench.step_model_bytes(big, (768 ** 3, 1536 ** 3), 16) == 577_221_341_184
