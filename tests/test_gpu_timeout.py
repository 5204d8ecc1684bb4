"""Bounded device waits (the mbarrier waits of the TMA-staged tile solve): a
wait that runs out -- an mbarrier phase that no copy completes -- gives up
after its limit, records a timeout that pm_check reports as PM_ERR_TIMEOUT,
and leaves the handle and the context usable: codes compressed afterwards
are still bit-exact against the oracle."""
import numpy as np
import pytest
import torch

from oracle import codec
from synth import make_workload
from tests.helpers import oracle_codes_from_lib, records

pytestmark = pytest.mark.gpu


def _compress_matches_oracle(pm, w, vel_bits):
    for s in range(2):
        got = pm.compress(s, torch.from_numpy(w.x[s]).cuda(), torch.from_numpy(w.v[s]).cuda())
        pm.check()
        ref = codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, vel_bits)
        g = oracle_codes_from_lib(got, w.n_fine // 4, vel_bits)
        np.testing.assert_array_equal(g.cnt, ref.cnt)
        np.testing.assert_array_equal(records(g), records(ref))


def test_wait_that_runs_out_reports_timeout_and_handle_stays_usable():
    from paper_1611_01545_gb300 import PM, _lib
    from paper_1611_01545_gb300.pm import PMError

    w = make_workload("single64", n_cdm=16, n_nu=32)
    pm = PM(dict(n_fine=w.n_fine, coarse_ratio=1, tile=w.n_fine, buffer=0, cmp_ratio=4, vel_bits=16,
                 G=1 / (4 * np.pi), mass=(8.0, 0.04), count=(0, 0)))
    _compress_matches_oracle(pm, w, 16)

    # the wait gives up after ~2e5 SM cycles (about 0.1 ms), not after the
    # library's one-second limit, and the status word says so
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    pm.wait_probe(200_000)
    e1.record(st)
    with pytest.raises(PMError) as err:
        pm.check()
    assert err.value.code == _lib.PM_ERR_TIMEOUT
    assert e0.elapsed_time(e1) < 50.0
    pm.check()   # reported once, then cleared

    # limits outside [1e3, 2e9] are refused on the host, nothing is launched
    for bad in (10, 3_000_000_000):
        with pytest.raises(PMError) as err:
            pm.wait_probe(bad)
        assert err.value.code == _lib.PM_ERR_ARG
    pm.check()

    # the context and the handle still work
    _compress_matches_oracle(pm, w, 16)
