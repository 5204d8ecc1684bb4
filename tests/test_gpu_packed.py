"""Packed codes (record bytes without padding): pack gives exactly the
oracle codec's position and velocity bytes, unpack restores the padded
words, for particle counts that do and do not fill whole groups of four and
for both velocity widths; pm_step_packed gives the same step as pm_step."""
import numpy as np
import pytest
import torch

from oracle import codec
from synth import make_workload
from tests.helpers import cfg_of, lib_codes_from_oracle, oracle_codes_from_lib, records

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("vel_bits", [8, 16])
@pytest.mark.parametrize("n", [0, 1, 3, 4, 7, 1001])
def test_pack_matches_oracle_record_bytes(vel_bits, n):
    from paper_1611_01545_gb300 import PM
    rng = np.random.default_rng(n + vel_bits)
    nf = 32
    x = (rng.random((n, 3)) * nf).astype(np.float32)
    v = rng.standard_normal((n, 3)).astype(np.float32)
    cfg = dict(n_fine=nf, coarse_ratio=1, tile=nf, buffer=0, cmp_ratio=4, vel_bits=vel_bits,
               G=1.0 / (4 * np.pi), mass=(8.0, 0.04), count=(n, n))
    pm = PM(cfg)
    oc = codec.compress(x, v, nf, nf // 4, vel_bits)
    dev = lib_codes_from_oracle(oc, esc_cap=8)
    packed = pm.pack(dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(packed.pos.cpu().numpy(), oc.pos.reshape(n, 3))
    pv = packed.vel.cpu().numpy()
    if vel_bits == 16:
        pv = pv.view(np.uint16)
    np.testing.assert_array_equal(pv, oc.vel.reshape(n, 3))
    back = pm.unpack(packed)
    torch.cuda.synchronize()
    assert torch.equal(back.pos, dev.pos) and torch.equal(back.vel, dev.vel)
    assert torch.equal(back.cnt, dev.cnt) and torch.equal(back.vmax, dev.vmax)


def test_step_packed_equals_step():
    from paper_1611_01545_gb300 import PM
    w = make_workload("two_level64", n_cdm=16, n_nu=40)
    cfg = cfg_of(w, deposit_mode=1)
    nc = w.n_fine // 4
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, nc, w.vel_bits) for s in range(2)]
    pm = PM(cfg)
    din = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    hin = [pm.pack(c).to("cpu", pin=True) for c in din]
    hout = [pm.pack(c).to("cpu", pin=True) for c in dout]
    for c in hout:
        c.pos.zero_()
        c.vel.zero_()
    # direct launches, then captured into a graph and replayed (velocity bytes
    # arrive on a second stream while the deposit and the solve run)
    for graphs in (False, True, True):
        pm.set_graphs(graphs)
        for c in hout:
            c.pos.zero_()
            c.vel.zero_()
        pm.step_packed(hin, hout, 1.0, 1.0)
        for s in range(2):
            got = oracle_codes_from_lib(pm.unpack(hout[s].to("cuda")), nc, w.vel_bits)
            ref = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
            assert got.vmax == ref.vmax
            np.testing.assert_array_equal(got.cnt, ref.cnt)
            np.testing.assert_array_equal(records(got), records(ref))
    pm.set_graphs(False)


@pytest.mark.parametrize("vel_bits,shared_output", [(8, False), (16, False), (16, True)])
def test_step_packed_async_overlapping_calls_equal_step(vel_bits, shared_output):
    """pm_step_packed_async: three calls queued back to back from one packed
    host input into three host outputs (each call's copies overlapping the
    neighbouring calls' compute), then one pm_check: every output is the
    step pm_step gives (fixed-point deposits, so bit for bit up to the order
    within a cell), and a following synchronous pm_step_packed agrees too.
    shared_output: the device is filled until the library has no room for a
    packed output buffer of its own, so the packed output shares the step
    scratch and each count pass waits for the previous output copies (the
    path the 1536^3 workload takes)."""
    from paper_1611_01545_gb300 import PM
    w = make_workload("two_level64", n_cdm=16, n_nu=40)
    cfg = cfg_of(w, deposit_mode=1, vel_bits=vel_bits)
    nc = w.n_fine // 4
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, nc, vel_bits) for s in range(2)]
    pm = PM(cfg)
    din = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    ref = [oracle_codes_from_lib(dout[s], nc, vel_bits) for s in range(2)]
    hin = [pm.pack(c).to("cpu", pin=True) for c in din]
    houts = [[pm.pack(c).to("cpu", pin=True) for c in dout] for _ in range(3)]
    for h in houts:
        for c in h:
            c.pos.zero_()
            c.vel.zero_()
    filler = None
    if shared_output:
        torch.cuda.synchronize()
        free, _ = torch.cuda.mem_get_info()
        filler = torch.empty(free - (1 << 30), dtype=torch.uint8, device="cuda")   # 1 GiB left free
    for h in houts:
        pm.step_packed_async(hin, h, 1.0, 1.0)
    pm.check()
    del filler
    torch.cuda.empty_cache()
    sync_out = [pm.pack(c).to("cpu", pin=True) for c in dout]
    pm.step_packed(hin, sync_out, 1.0, 1.0)
    for h in houts + [sync_out]:
        for s in range(2):
            got = oracle_codes_from_lib(pm.unpack(h[s].to("cuda")), nc, vel_bits)
            assert got.vmax == ref[s].vmax
            np.testing.assert_array_equal(got.cnt, ref[s].cnt)
            np.testing.assert_array_equal(records(got), records(ref[s]))
