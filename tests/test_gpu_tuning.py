"""Launch tunings (cell-block shapes, persistent launches, new-cell window,
tile batch) and the autotuner: every tuning gives the same step result, the
autotuner leaves the input codes untouched and keeps parity, and unusable
tunings are refused."""
import numpy as np
import pytest
import torch

from oracle import codec
from synth import make_workload
from tests.helpers import cfg_of, lib_codes_from_oracle, oracle_codes_from_lib, records

pytestmark = pytest.mark.gpu


def _setup(name, n_cdm, n_nu):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    cfg = cfg_of(w, deposit_mode=1)
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, w.vel_bits) for s in range(2)]
    return w, cfg, codes


def _step(pm, w, codes, tuning=None):
    if tuning:
        pm.set_tuning(tuning)
    din = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    return [oracle_codes_from_lib(dout[s], w.n_fine // 4, w.vel_bits) for s in range(2)]


def _same(a, b):
    for s in range(2):
        assert a[s].vmax == b[s].vmax
        np.testing.assert_array_equal(a[s].cnt, b[s].cnt)
        np.testing.assert_array_equal(records(a[s]), records(b[s]))


@pytest.mark.parametrize("name,n_cdm,n_nu", [("two_level64", 16, 40), ("two_level128_t96", 24, 48)])
def test_every_tuning_gives_the_same_step(name, n_cdm, n_nu):
    from paper_1611_01545_gb300 import PM
    w, cfg, codes = _setup(name, n_cdm, n_nu)
    pm = PM(cfg)
    base = pm.get_tuning()
    ref = _step(pm, w, codes)
    n = w.n_fine // 4
    tunings = [
        {"deposit_persistent": 1},
        {"deposit_block": (n // 2, 2, 1), "deposit_persistent": 0},
        {"deposit_block": (n // 4, 2, 2), "deposit_persistent": 1},
        {"kick_persistent": 1},
        {"kick_block": (n // 2, 2, 1), "kick_window": 1, "kick_persistent": 1},
        {"kick_block": (n // 4, 1, 2), "kick_window": 3, "kick_persistent": 0},
        {"tile_batch": 1},
    ]
    for t in tunings:
        pm.set_tuning(dict(base, **t))
        _same(_step(pm, w, codes), ref)


def test_autotune_keeps_input_and_parity():
    from paper_1611_01545_gb300 import PM
    w, cfg, codes = _setup("two_level64", 16, 40)
    pm = PM(cfg)
    ref = _step(pm, w, codes)
    din = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    before = [(c.pos.clone(), c.vel.clone(), c.cnt.clone(), c.vmax.clone()) for c in din]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    chosen = pm.autotune(din, dout, 1.0, 1.0, reps=1)
    torch.cuda.synchronize()
    assert chosen == pm.get_tuning()
    for c, (p, v, k, m) in zip(din, before):
        assert torch.equal(c.pos, p) and torch.equal(c.vel, v) and torch.equal(c.cnt, k) and torch.equal(c.vmax, m)
    _same(_step(pm, w, codes), ref)


def test_unusable_tunings_are_refused():
    from paper_1611_01545_gb300 import PM
    from paper_1611_01545_gb300.pm import PMError
    w, cfg, codes = _setup("two_level64", 16, 40)
    pm = PM(cfg)
    base = pm.get_tuning()
    n = w.n_fine // 4
    for bad in ({"deposit_block": (n - 1, 1, 1)}, {"kick_block": (n, n, n)}, {"kick_window": 0},
                {"tile_batch": 0}, {"tile_batch": base["tile_batch"] + 1}, {"kick_persistent": 2}):
        with pytest.raises(PMError):
            pm.set_tuning(dict(base, **bad))
    assert pm.get_tuning() == base
    _step(pm, w, codes)
