"""Pins for the oracle codec (Sec. 2.4): hand-derived byte streams, exact
round trips, the quantisation error bounds implied by the bin definitions,
the 255 escape, and the ~9 B/particle footprint."""
import numpy as np
import pytest

from oracle import codec
from tests.golden_codec import load_cases


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_golden_stream(case):
    c = codec.compress(case["x"], case["v"], case["n_fine"], case["n_cmp"], case["vel_bits"])
    assert codec.serialize(c) == case["hex"]
    back = codec.deserialize(case["hex"])
    np.testing.assert_array_equal(back.pos, c.pos)
    np.testing.assert_array_equal(back.vel, c.vel)
    np.testing.assert_array_equal(back.cnt, c.cnt)
    assert back.vmax == c.vmax


def _random_state(rng, n, n_fine):
    x = (rng.random((n, 3)) * n_fine).astype(np.float32)
    x[x >= n_fine] = 0
    v = (rng.standard_normal((n, 3)) * 3).astype(np.float32)
    return x, v


@pytest.mark.parametrize("vel_bits", [16, 8])
def test_error_bounds(vel_bits):
    rng = np.random.default_rng(11)
    n_fine, n_cmp = 64, 16
    x, v = _random_state(rng, 20000, n_fine)
    c = codec.compress(x, v, n_fine, n_cmp, vel_bits)
    xd, vd = codec.decompress(c, n_fine)
    # match particles: compress is stable by cell, so recover the permutation
    cx = np.floor(x / 4).astype(np.int64)
    perm = np.argsort(cx[:, 0] + 16 * (cx[:, 1] + 16 * cx[:, 2]), kind="stable")
    r = n_fine // n_cmp
    assert np.max(np.abs(xd - x[perm])) <= r / 512 * (1 + 1e-6)
    vmax = np.max(np.abs(v))
    half_bin = vmax / 2 ** vel_bits
    assert np.max(np.abs(vd - v[perm])) <= half_bin * (1 + 1e-4) + 1e-7 * vmax


@pytest.mark.parametrize("vel_bits", [16, 8])
@pytest.mark.parametrize("order", ["stable", "canonical"])
def test_round_trip_bit_exact(vel_bits, order):
    rng = np.random.default_rng(12)
    x, v = _random_state(rng, 5000, 32)
    c = codec.compress(x, v, 32, 8, vel_bits, order=order)
    xd, vd = codec.decompress(c, 32)
    c2 = codec.compress(xd, vd, 32, 8, vel_bits, vmax=c.vmax, order=order)
    for f in ("cnt", "esc_cell", "esc_count", "pos", "vel"):
        np.testing.assert_array_equal(getattr(c2, f), getattr(c, f))
    assert codec.deserialize(codec.serialize(c)).pos.tobytes() == c.pos.tobytes()


def test_escape_path_and_counts():
    rng = np.random.default_rng(13)
    x = np.concatenate([np.full((300, 3), 1.5, np.float32), (rng.random((50, 3)) * 8).astype(np.float32)])
    v = rng.standard_normal((350, 3)).astype(np.float32)
    c = codec.compress(x, v, 8, 2, 16)
    assert c.cnt[0] == 255 and c.esc_cell.tolist() == [0] and c.esc_count[0] >= 300
    assert c.counts().sum() == 350
    back = codec.deserialize(codec.serialize(c))
    np.testing.assert_array_equal(back.esc_count, c.esc_count)
    bad = codec.Codes(c.n_cmp, c.vel_bits, c.cnt, c.esc_cell[:0], c.esc_count[:0], c.pos, c.vel, c.vmax)
    with pytest.raises(ValueError):
        codec.decompress(bad, 8)


def test_footprint_roughly_nine_bytes():
    # Sec. 2.4: 24 B per particle -> roughly 9 B (3 B position + 6 B velocity + amortised count).
    rng = np.random.default_rng(14)
    x, v = _random_state(rng, 64 * 4096, 64)     # 64 particles per cell on 16^3 cells
    s = codec.serialize(codec.compress(x, v, 64, 16, 16))
    per = (len(s) - codec.HEADER_SIZE) / x.shape[0]
    assert 9.0 < per < 9.05


def test_vmax_zero_and_clamp():
    x = np.array([[0.1, 0.2, 0.3]] * 4, np.float32)
    c0 = codec.compress(x, np.zeros((4, 3), np.float32), 4, 1, 16)
    assert np.all(c0.vel == 32768)
    _, v0 = codec.decompress(c0, 4)
    assert np.all(v0 == 0)
    v = np.array([[1, -1, 0.5]] * 4, np.float32)
    c1 = codec.compress(x, v, 4, 1, 16)
    assert c1.vel[0].tolist() == [65535, 0, 49152]


def test_rejects_out_of_range_positions():
    with pytest.raises(ValueError):
        codec.compress(np.array([[8.0, 0, 0]], np.float32), np.zeros((1, 3), np.float32), 8, 2)
