"""GPU parity of the Sec. 2.4 codec: compress / decompress through the C ABI
against the oracle, bit-exact; corrupt streams are reported, not decoded."""
import numpy as np
import pytest
import torch

from oracle import codec
from synth import make_workload
from tests.helpers import lib_codes_from_oracle, oracle_codes_from_lib, records

pytestmark = pytest.mark.gpu


def _pm(cfg):
    from paper_1611_01545_gb300 import PM
    return PM(cfg)


def _cfg(n_fine=64, vel_bits=16, **kw):
    c = dict(n_fine=n_fine, coarse_ratio=1, tile=n_fine, buffer=0, cmp_ratio=4, vel_bits=vel_bits,
             G=1 / (4 * np.pi), mass=(8.0, 0.04), count=(0, 0))
    c.update(kw)
    return c


@pytest.mark.parametrize("vel_bits", [16, 8])
@pytest.mark.parametrize("name,n_cdm,n_nu", [("single64", 16, 32), ("two_level128_t96", 24, 61)])
def test_compress_parity(vel_bits, name, n_cdm, n_nu):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    pm = _pm(_cfg(w.n_fine, vel_bits))
    for s in range(2):
        got = pm.compress(s, torch.from_numpy(w.x[s]).cuda(), torch.from_numpy(w.v[s]).cuda())
        pm.check()
        ref = codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, vel_bits)
        g = oracle_codes_from_lib(got, w.n_fine // 4, vel_bits)
        np.testing.assert_array_equal(g.cnt, ref.cnt)
        np.testing.assert_array_equal(g.esc_cell, ref.esc_cell)
        np.testing.assert_array_equal(g.esc_count, ref.esc_count)
        assert g.vmax == ref.vmax
        np.testing.assert_array_equal(records(g), records(ref))


@pytest.mark.parametrize("vel_bits", [16, 8])
def test_decompress_parity_and_round_trip(vel_bits):
    w = make_workload("two_level128_t96", n_cdm=20, n_nu=50)
    pm = _pm(_cfg(w.n_fine, vel_bits))
    for s in range(2):
        ref = codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, vel_bits)
        dc = lib_codes_from_oracle(ref)
        x, v = pm.decompress(s, dc)
        pm.check()
        xr, vr = codec.decompress(ref, w.n_fine)
        np.testing.assert_array_equal(x.cpu().numpy(), xr)
        np.testing.assert_array_equal(v.cpu().numpy(), vr)
        again = pm.compress(s, x, v, vmax=dc.vmax)
        pm.check()
        np.testing.assert_array_equal(records(oracle_codes_from_lib(again, w.n_fine // 4, vel_bits)), records(ref))


def test_escape_path_and_ragged_sizes():
    rng = np.random.default_rng(41)
    x = (rng.random((1237, 3)) * 32).astype(np.float32)
    x[:600] = np.float32(5.5)        # 600 particles in one cell -> escape
    x[600:900] = np.float32(17.25)   # 300 in another
    v = rng.standard_normal((1237, 3)).astype(np.float32)
    pm = _pm(_cfg(32))
    got = pm.compress(0, torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda())
    pm.check()
    ref = codec.compress(x, v, 32, 8, 16)
    g = oracle_codes_from_lib(got, 8, 16)
    assert g.esc_cell.tolist() == ref.esc_cell.tolist() and len(ref.esc_cell) == 2
    np.testing.assert_array_equal(records(g), records(ref))
    xd, vd = pm.decompress(0, got)
    pm.check()
    xr, vr = codec.decompress(g, 32)
    np.testing.assert_array_equal(xd.cpu().numpy(), xr)
    np.testing.assert_array_equal(vd.cpu().numpy(), vr)


def test_empty_species_and_zero_vmax():
    pm = _pm(_cfg(16))
    x = torch.zeros((0, 3), device="cuda")
    c = pm.compress(1, x, x)
    pm.check()
    assert int(c.cnt.sum()) == 0 and float(c.vmax) == 0.0
    xs = torch.full((5, 3), 3.0, device="cuda")
    c = pm.compress(0, xs, torch.zeros_like(xs))
    pm.check()
    assert torch.all(c.vel_u16() == 32768)
    _, v = pm.decompress(0, c)
    pm.check()
    assert torch.all(v == 0)


def _corrupt(kind):
    rng = np.random.default_rng(42)
    x = (rng.random((700, 3)) * 16).astype(np.float32)
    x[:300] = np.float32(1.0)
    ref = codec.compress(x, rng.standard_normal((700, 3)).astype(np.float32), 16, 4, 16)
    dc = lib_codes_from_oracle(ref)
    if kind == "missing_escape":
        dc.n_esc.zero_()
    elif kind == "count_mismatch":
        cnt = dc.cnt.clone()
        j = int(torch.nonzero(cnt < 200)[0])
        cnt[j] += 1
        dc.cnt.copy_(cnt)
    elif kind == "small_escape":
        dc.esc[0, 1] = 100
    elif kind == "nan_vmax":
        dc.vmax.fill_(float("nan"))
    return dc


@pytest.mark.parametrize("kind", ["missing_escape", "count_mismatch", "small_escape", "nan_vmax"])
def test_corrupt_streams_are_reported(kind):
    from paper_1611_01545_gb300 import PMError
    pm = _pm(_cfg(16))
    dc = _corrupt(kind)
    pm.decompress(0, dc)
    with pytest.raises(PMError) as e:
        pm.check()
    assert e.value.code == 4
    pm.check()   # status is cleared after being reported


def test_escape_overflow_reported():
    from paper_1611_01545_gb300 import PMError
    pm = _pm(_cfg(16))
    x = torch.full((600, 3), 1.0, device="cuda")
    x[300:] = 9.0
    out = pm.empty_codes(600, esc_cap=1)
    pm.compress(0, x, torch.zeros_like(x), out=out)
    with pytest.raises(PMError) as e:
        pm.check()
    assert e.value.code == 5


def test_out_of_range_position_reported():
    from paper_1611_01545_gb300 import PMError
    pm = _pm(_cfg(16))
    x = torch.rand((100, 3), device="cuda") * 16
    x[7, 1] = 16.0
    pm.compress(0, x, torch.zeros_like(x))
    with pytest.raises(PMError) as e:
        pm.check()
    assert e.value.code == 6


def test_compress_parity_large_mesh():
    # 128^3 compression cells: the count scan needs more than 992 partial sums,
    # so the single-block scan of the partials runs all 32 of its warps.
    rng = np.random.default_rng(43)
    x = (rng.random((300000, 3)) * 512).astype(np.float32)
    x[x >= 512] = 0
    x[-1000:] = np.float32(511.5)              # the last cell, escaped
    v = rng.standard_normal((300000, 3)).astype(np.float32)
    pm = _pm(_cfg(512, coarse_ratio=4, tile=64, buffer=16, r_cut=14.0, r_split=14.0 / 4.5))
    got = pm.compress(0, torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda())
    pm.check()
    ref = codec.compress(x, v, 512, 128, 16)
    g = oracle_codes_from_lib(got, 128, 16)
    np.testing.assert_array_equal(g.cnt, ref.cnt)
    np.testing.assert_array_equal(g.esc_count, ref.esc_count)
    np.testing.assert_array_equal(records(g), records(ref))
    xd, _ = pm.decompress(0, got)
    pm.check()
    np.testing.assert_array_equal(xd.cpu().numpy(), codec.decompress(g, 512)[0])
