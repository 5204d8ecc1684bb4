"""Asynchronous checkpoint: the codes copied to pinned host memory while the
state keeps stepping are those of the checkpointed step, the fence keeps a
later step from overwriting them before the copy, the serialized
checkpoint restores the state bit for bit, its byte stream is the oracle's
serialisation of the same codes, and the checkpointed state matches the
oracle's own step."""
import numpy as np
import pytest
import torch

from oracle import codec, step
from synth import make_workload
from tests.helpers import assert_codes_match, cfg_of, lib_codes_from_oracle, oracle_codes_from_lib, records

pytestmark = pytest.mark.gpu


def test_async_checkpoint_while_stepping():
    from paper_1611_01545_gb300 import PM
    from paper_1611_01545_gb300.pm import deserialize, serialize
    w = make_workload("two_level64", n_cdm=16, n_nu=40)
    cfg = cfg_of(w, deposit_mode=1)
    nc = w.n_fine // 4
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, nc, w.vel_bits) for s in range(2)]
    pm = PM(cfg)
    a = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    b = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(a, b, 0.5, 0.5)                        # state S1 in b
    host = [pm.empty_codes(c.n, esc_cap=64).to("cpu", pin=True) for c in codes]
    pm.checkpoint_begin(b, host)                   # copy S1 while stepping on
    pm.step(b, a, 0.5, 0.5)                        # S2 in a (reads b only)
    pm.checkpoint_fence()                          # the next step overwrites b
    pm.step(a, b, 0.5, 0.5)                        # S3 in b
    pm.checkpoint_wait()
    pm.check()
    # S1 recomputed from the initial state by a fresh handle
    pm2 = PM(cfg)
    a2 = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    b2 = [pm2.empty_codes(c.n, esc_cap=64) for c in codes]
    pm2.step(a2, b2, 0.5, 0.5)
    pm2.check()
    oracle_s1, _ = step.step(codes, cfg, 0.5, 0.5)
    for s in range(2):
        got = oracle_codes_from_lib(host[s], nc, w.vel_bits)
        ref = oracle_codes_from_lib(b2[s], nc, w.vel_bits)
        assert got.vmax == ref.vmax
        np.testing.assert_array_equal(got.cnt, ref.cnt)
        np.testing.assert_array_equal(records(got), records(ref))
        # the byte stream of the checkpoint restores the same codes
        blob = serialize(host[s], nc, w.vel_bits)
        # ... and is the oracle's Sec. 2.4 stream of those codes, byte for byte
        assert blob == codec.serialize(got)
        # the checkpointed state against the oracle's own step from the same codes:
        # the oracle's deserializer reads the library's stream, and every record
        # equals the oracle's or sits one quantisation step from it
        assert_codes_match(codec.deserialize(blob), oracle_s1[s], f"checkpoint species {s}")
        back = deserialize(blob, host[s].n, nc, w.vel_bits, esc_cap=64)
        assert torch.equal(back.pos[:, :3], host[s].pos[:, :3]) and torch.equal(back.cnt, host[s].cnt)
        assert torch.equal(back.vel[:, :3], host[s].vel[:, :3]) and torch.equal(back.vmax, host[s].vmax)
    with pytest.raises(Exception):
        pm.checkpoint_begin(b, host)
        pm.checkpoint_begin(b, host)               # a second pending checkpoint is refused
    pm.checkpoint_wait()
