"""GPU parity of force interpolation, kick-drift and the fused compressed step
against the oracle, and bit-exact agreement of the fused step with the
plain (one call per stage) path in fixed-point mode."""
import numpy as np
import pytest
import torch

from oracle import codec, step
from synth import make_workload
from tests.helpers import (assert_codes_match, cfg_of, lib_codes_from_oracle, oracle_codes_from_lib, records,
                           rel_rms)

pytestmark = pytest.mark.gpu

ACC_TOL = 1e-4       # per-particle accelerations, float32 vs float64, relative RMS


def _pm(cfg):
    from paper_1611_01545_gb300 import PM
    return PM(cfg)


CASES = [("single64", 16, 32), ("two_level64", 16, 40), ("two_level128_t96", 24, 48)]


def _setup(name, n_cdm, n_nu, **kw):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    cfg = cfg_of(w, **kw)
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, w.vel_bits) for s in range(2)]
    xv = [codec.decompress(c, w.n_fine) for c in codes]
    return w, cfg, codes, xv


def _plain_accel(pm, xv, fixed=False):
    rc, rf = pm.zeros_meshes(fixed=fixed)
    xs = [torch.from_numpy(p[0]).cuda() for p in xv]
    for s in range(2):
        (pm.deposit_fixed if fixed else pm.deposit)(s, xs[s], rc, rf)
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    return xs, ac, af


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_interpolated_acceleration_parity(name, n_cdm, n_nu):
    w, cfg, codes, xv = _setup(name, n_cdm, n_nu)
    pm = _pm(cfg)
    xs, ac, af = _plain_accel(pm, xv)
    got = [pm.interpolate(xs[s], ac, af).cpu().numpy() for s in range(2)]
    pm.check()
    ref = step.accel([p[0] for p in xv], cfg)
    for s in range(2):
        assert rel_rms(got[s], ref[s]) < ACC_TOL, (s, rel_rms(got[s], ref[s]))


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES[:2])
def test_kick_drift_parity(name, n_cdm, n_nu):
    w, cfg, codes, xv = _setup(name, n_cdm, n_nu)
    pm = _pm(cfg)
    xs, ac, af = _plain_accel(pm, xv)
    ref_a = step.accel([p[0] for p in xv], cfg)
    for s in range(2):
        x = xs[s].clone()
        v = torch.from_numpy(xv[s][1]).cuda()
        pm.kick_drift(x, v, ac, af, 0.5, 1.5)
        pm.check()
        x1, v1 = step.kick_drift(xv[s][0], xv[s][1], ref_a[s], 0.5, 1.5, w.n_fine)
        dv = v.cpu().numpy() - v1
        assert np.sqrt(np.mean(dv ** 2)) < ACC_TOL * 0.5 * np.sqrt(np.mean(ref_a[s] ** 2)) + 1e-6
        dx = x.cpu().numpy() - x1
        dx -= w.n_fine * np.round(dx / w.n_fine)
        assert np.max(np.abs(dx)) < 1e-3


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_fused_step_matches_oracle_codes(name, n_cdm, n_nu):
    w, cfg, codes, xv = _setup(name, n_cdm, n_nu)
    pm = _pm(cfg)
    din = [lib_codes_from_oracle(c) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    ref, states = step.step(codes, cfg, 1.0, 1.0)
    nc = w.n_fine // 4
    for s in range(2):
        g = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
        assert g.counts().sum() == ref[s].n
        assert abs(float(g.vmax) - float(ref[s].vmax)) <= 1e-5 * float(ref[s].vmax)
        # identical except for records straddling a bin edge in float32 vs float64
        assert_codes_match(g, ref[s], f"{name} species {s}")


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_fused_step_equals_plain_path_fixed_point(name, n_cdm, n_nu):
    w, cfg, codes, xv = _setup(name, n_cdm, n_nu, deposit_mode=1)
    pm = _pm(cfg)
    din = [lib_codes_from_oracle(c) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    xs, ac, af = _plain_accel(pm, xv, fixed=True)
    nc = w.n_fine // 4
    for s in range(2):
        x = xs[s].clone()
        v = torch.from_numpy(xv[s][1]).cuda()
        pm.kick_drift(x, v, ac, af, 1.0, 1.0)
        plain = pm.compress(s, x, v)
        pm.check()
        a = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
        b = oracle_codes_from_lib(plain, nc, w.vel_bits)
        assert a.vmax == b.vmax
        np.testing.assert_array_equal(a.cnt, b.cnt)
        np.testing.assert_array_equal(records(a), records(b))


def test_step_host_matches_device_step():
    w, cfg, codes, xv = _setup("two_level64", 16, 40, deposit_mode=1)
    pm = _pm(cfg)
    din = [lib_codes_from_oracle(c) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    hin = [lib_codes_from_oracle(c, device="cpu", esc_cap=64) for c in codes]
    hin = [c.to("cpu", pin=True) for c in hin]
    hout = [pm.empty_codes(c.n, esc_cap=64).to("cpu", pin=True) for c in codes]
    pm.step_host(hin, hout, 1.0, 1.0)
    for s in range(2):
        a = oracle_codes_from_lib(dout[s], w.n_fine // 4, w.vel_bits)
        b = oracle_codes_from_lib(hout[s], w.n_fine // 4, w.vel_bits)
        np.testing.assert_array_equal(records(a), records(b))
        assert a.vmax == b.vmax


def test_multi_step_invariants():
    w, cfg, codes, xv = _setup("two_level64", 16, 40, deposit_mode=1)
    pm = _pm(cfg)
    a = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
    b = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    for _ in range(4):
        pm.step(a, b, 0.5, 0.5)
        pm.check()
        a, b = b, a
    for s in range(2):
        g = oracle_codes_from_lib(a[s], w.n_fine // 4, w.vel_bits)
        assert g.counts().sum() == codes[s].n
        x, v = codec.decompress(g, w.n_fine)
        assert np.all((x >= 0) & (x < w.n_fine))


def test_graph_replay_equals_direct_launches():
    """pm_set_graphs: four ping-pong steps replayed from captured graphs give
    the same codes as four directly launched steps (fixed-point deposits, so
    both runs are deterministic up to the order within a cell), and the launch counter advances by the
    captured kernels on every replay."""
    from paper_1611_01545_gb300 import _lib
    w, cfg, codes, xv = _setup("two_level64", 16, 40, deposit_mode=1)
    lib = _lib.load()
    results = []
    for graphs in (False, True):
        pm = _pm(cfg)
        pm.set_graphs(graphs)
        a = [lib_codes_from_oracle(c, esc_cap=64) for c in codes]
        b = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
        per_step = []
        for _ in range(4):
            n0 = lib.pm_launch_count()
            pm.step(a, b, 0.5, 0.5)
            torch.cuda.synchronize()
            per_step.append(lib.pm_launch_count() - n0)
            pm.check()
            a, b = b, a
        assert len(set(per_step)) == 1 and per_step[0] > 0, per_step
        results.append(([oracle_codes_from_lib(a[s], w.n_fine // 4, w.vel_bits) for s in range(2)], per_step[0]))
        pm.set_graphs(False)
    (direct, n_direct), (replayed, n_graph) = results
    assert n_direct == n_graph
    for s in range(2):
        assert direct[s].vmax == replayed[s].vmax
        np.testing.assert_array_equal(direct[s].cnt, replayed[s].cnt)
        np.testing.assert_array_equal(records(direct[s]), records(replayed[s]))


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_fused_step_vmax_bound_mode(name, n_cdm, n_nu):
    """vmax_mode 1: v_max' is the rounded-up bound from the mesh maxima (GPU
    float32 meshes vs the oracle's float64 ones: relative 1e-4), it covers
    every kicked velocity, and the codes are the oracle codec's with that
    v_max (up to records straddling a bin edge)."""
    w, cfg, codes, xv = _setup(name, n_cdm, n_nu, vmax_mode=1)
    pm = _pm(cfg)
    din = [lib_codes_from_oracle(c) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, 1.0, 1.0)
    pm.check()
    ref, states = step.step(codes, cfg, 1.0, 1.0, vmax_mode=1)
    n, nc = w.n_fine, w.n_fine // 4
    for s in range(2):
        g = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
        assert abs(float(g.vmax) - float(ref[s].vmax)) <= 1e-4 * float(ref[s].vmax)
        x1, v1 = states[s]
        assert float(g.vmax) >= np.max(np.abs(v1)) * (1 - 1e-5)
        mine = codec.compress(step.to_f32_positions(x1, n), v1.astype(np.float32), n, nc, w.vel_bits, vmax=g.vmax)
        assert_codes_match(g, mine, f"{name} bound mode species {s}")


@pytest.mark.parametrize("case", ["empty_cdm", "zero_step"])
def test_fused_step_degenerate_cases(case):
    """The fused step's degenerate cases against the oracle: a species with no
    particles (the CDM; every pass must skip it and still scan, place and
    count the neutrinos), and a step with c_kick = c_drift = 0 (nothing moves,
    the velocities are re-quantised with the new, smaller v_max')."""
    w = make_workload("two_level64", n_cdm=16, n_nu=40)
    nc = w.n_fine // 4
    if case == "empty_cdm":
        w.x[0] = np.zeros((0, 3), np.float32)
        w.v[0] = np.zeros((0, 3), np.float32)
        ck = cd = 1.0
    else:
        ck = cd = 0.0
    cfg = cfg_of(w)
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, nc, w.vel_bits) for s in range(2)]
    pm = _pm(cfg)
    din = [lib_codes_from_oracle(c) for c in codes]
    dout = [pm.empty_codes(c.n, esc_cap=64) for c in codes]
    pm.step(din, dout, ck, cd)
    pm.check()
    ref, _ = step.step(codes, cfg, ck, cd)
    for s in range(2):
        g = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
        assert g.n == ref[s].n
        assert g.counts().sum() == ref[s].n
        assert abs(float(g.vmax) - float(ref[s].vmax)) <= 1e-5 * float(ref[s].vmax)
        assert_codes_match(g, ref[s], f"{case} species {s}")
