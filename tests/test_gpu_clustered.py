"""The batched launch forms on clustered input against the oracle.

Lognormal-clustered CDM (sigma_ln rho = 1.5, P(k) ~ k^-2, per-tile counts
spanning more than 30x) plus hot neutrinos go through the fused step in the
forms the batched workload is timed in: launch tuning picked by the
autotuner, persistent cell-block launches, and the step replayed from a
captured CUDA graph.

* clustered64 (64^3 mesh, 64 tiles, 32^3 + 64^3 particles): the whole step
  against the oracle: every post-step record equal to the oracle's or one
  quantisation step from it, v_max' and counts; accelerations interpolated
  from the GPU meshes against the oracle's per-particle acceleration.
* batched512 (512^3 mesh, 512 tiles of 96^3, 256^3 + 512^3 particles, tile
  counts 4270 .. 150905): sampled outputs the oracle computes one by one (a
  density sub-box inside the densest tile, the densest and the sparsest tile
  solves, sampled interpolations), exact fixed-point mass, and the fused
  step equal bit for bit to the plain per-stage path in fixed point.
"""
import numpy as np
import pytest
import torch

from oracle import codec, mesh, solve, step
from synth import make_workload
from tests.helpers import (assert_codes_match, cfg_of, device_records_equal, lib_codes_from_oracle,
                           oracle_codes_from_lib, rel_rms)

pytestmark = pytest.mark.gpu

ACC_TOL = 1e-4    # per-particle accelerations, float32 vs float64, relative RMS
RHO_TOL = 1e-5    # mesh density and forces, relative RMS


def _pm(cfg):
    from paper_1611_01545_gb300 import PM
    return PM(cfg)


@pytest.fixture(scope="module")
def small():
    w = make_workload("clustered64")
    assert w.notes["tile_count_max"] >= 30 * w.notes["tile_count_min"], w.notes
    cfg = cfg_of(w)
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, w.vel_bits) for s in range(2)]
    ref, states = step.step(codes, cfg, 1.0, 1.0)
    return w, cfg, codes, ref


def test_clustered_tuned_persistent_graph_step_matches_oracle(small):
    w, cfg, codes, ref = small
    pm = _pm(cfg)
    cap = [max(64, c.n // 255 + 1) for c in codes]
    din = [lib_codes_from_oracle(c, esc_cap=k) for c, k in zip(codes, cap)]
    dout = [pm.empty_codes(c.n, esc_cap=k) for c, k in zip(codes, cap)]
    tuned = pm.autotune(din, dout, 1.0, 1.0, reps=1)
    forms = [tuned, dict(tuned, deposit_persistent=1, kick_persistent=1)]
    nc = w.n_fine // 4
    for form in forms:
        pm.set_tuning(form)
        pm.set_graphs(True)
        for _ in range(2):                 # the first call captures the graph, the second replays it
            pm.step(din, dout, 1.0, 1.0)
        pm.check()
        pm.set_graphs(False)
        for s in range(2):
            g = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
            assert abs(float(g.vmax) - float(ref[s].vmax)) <= 1e-5 * float(ref[s].vmax)
            assert (g.esc_cell.size > 0) == (ref[s].esc_cell.size > 0)
            assert_codes_match(g, ref[s], f"clustered64 {form} species {s}")
    # the output takes the escape path (clusters of more than 254 particles per cell)
    assert sum(int(c.esc_cell.size) for c in ref) > 0


def test_clustered_bound_mode_step_matches_oracle(small):
    """vmax_mode 1 on the clustered set: v_max' is the oracle's rounded-up
    bound (float32 meshes: relative 1e-4), it covers every kicked velocity,
    and the codes, escapes included, are the oracle codec's with that v_max
    (the scatter copies the 12-byte coded records of 16-bit codes), in the
    one-CTA-per-block and the persistent launch forms."""
    w, _, codes, _ = small
    cfg = cfg_of(w, vmax_mode=1)
    ref, states = step.step(codes, cfg, 1.0, 1.0, vmax_mode=1)
    pm = _pm(cfg)
    cap = [max(64, c.n // 255 + 1) for c in codes]
    din = [lib_codes_from_oracle(c, esc_cap=k) for c, k in zip(codes, cap)]
    dout = [pm.empty_codes(c.n, esc_cap=k) for c, k in zip(codes, cap)]
    n, nc = w.n_fine, w.n_fine // 4
    base = pm.get_tuning()
    for form in (dict(base, kick_persistent=0), dict(base, deposit_persistent=1, kick_persistent=1)):
        pm.set_tuning(form)
        pm.step(din, dout, 1.0, 1.0)
        pm.check()
        for s in range(2):
            g = oracle_codes_from_lib(dout[s], nc, w.vel_bits)
            assert abs(float(g.vmax) - float(ref[s].vmax)) <= 1e-4 * float(ref[s].vmax)
            x1, v1 = states[s]
            assert float(g.vmax) >= np.max(np.abs(v1)) * (1 - 1e-5)
            mine = codec.compress(step.to_f32_positions(x1, n), v1.astype(np.float32), n, nc, w.vel_bits,
                                  vmax=g.vmax)
            assert (g.esc_cell.size > 0) == (mine.esc_cell.size > 0)
            assert_codes_match(g, mine, f"clustered64 bound mode {form} species {s}")


def test_clustered_interpolated_acceleration_matches_oracle(small):
    w, cfg, codes, ref = small
    pm = _pm(cfg)
    xv = [codec.decompress(c, w.n_fine) for c in codes]
    xs = [torch.from_numpy(p[0]).cuda() for p in xv]
    rc, rf = pm.zeros_meshes()
    for s in range(2):
        pm.deposit(s, xs[s], rc, rf)
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    got = [pm.interpolate(xs[s], ac, af).cpu().numpy() for s in range(2)]
    pm.check()
    want = step.accel([p[0] for p in xv], cfg)
    for s in range(2):
        assert rel_rms(got[s], want[s]) < ACC_TOL, (s, rel_rms(got[s], want[s]))


# ---------------------------------------------------------------- 512^3 --

BATCHED_TUNING = {"deposit_block": [32, 2, 1], "deposit_persistent": 1, "kick_block": [64, 1, 1],
                  "kick_window": 1, "kick_persistent": 1, "tile_batch": 256}


@pytest.fixture(scope="module")
def big():
    w = make_workload("batched512")
    assert w.notes["tile_count_max"] >= 30 * w.notes["tile_count_min"], w.notes
    out = {"w": w}
    for mode in (0, 1):
        pm = _pm(dict(w.config(), deposit_mode=mode))
        pm.set_tuning(BATCHED_TUNING)
        codes = []
        for s in range(2):
            x = torch.from_numpy(w.x[s]).cuda()
            v = torch.from_numpy(w.v[s]).cuda()
            codes.append(pm.compress(s, x, v, out=pm.empty_codes(x.shape[0], esc_cap=x.shape[0] // 255 + 1)))
            del x, v
        pm.check()
        out[mode] = (pm, codes)
    t = w.tile
    nt = w.n_fine // t
    tid = (w.x[0] // t).astype(np.int64)
    cnt = np.bincount(tid[:, 0] + nt * (tid[:, 1] + nt * tid[:, 2]), minlength=nt ** 3)
    out["dense"], out["sparse"] = int(np.argmax(cnt)), int(np.argmin(cnt))
    return out


def _tile_xyz(tile, nt):
    return tile % nt, (tile // nt) % nt, tile // (nt * nt)


def test_batched512_density_and_tile_solves_match_oracle(big):
    w = big["w"]
    pm, codes = big[0]
    n, t, b = w.n_fine, w.tile, w.buffer
    T, nt = t + 2 * b, n // t
    rc, rf = pm.zeros_meshes()
    pm.deposit_codes(codes, rc, rf)          # the fused deposit (persistent cell blocks)
    xs = [pm.decompress(s, codes[s])[0] for s in range(2)]
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    pm.check()
    rho_f = rf.cpu().numpy().astype(np.float64)
    # a 16^3 sub-box at the centre of the densest tile, from the particles around it
    ix, iy, iz = _tile_xyz(big["dense"], nt)
    lo = np.array([ix * t + 24, iy * t + 24, iz * t + 24])
    hi = lo + 16
    sub = np.zeros((18, 18, 18))
    lo_t = torch.tensor(lo - 1, dtype=torch.float32, device="cuda")
    hi_t = torch.tensor(hi + 1, dtype=torch.float32, device="cuda")
    for s in range(2):
        near = xs[s][((xs[s] >= lo_t) & (xs[s] < hi_t)).all(dim=1)]     # the particles around the sub-box
        x = near.cpu().numpy().astype(np.float64)
        sub += mesh.cic_deposit(x - (lo - 1), w.mass[s], 64)[:18, :18, :18]
    got = rho_f[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    assert rel_rms(got, sub[1:17, 1:17, 1:17]) < RHO_TOL
    # the densest and the sparsest tile solved by the oracle from the GPU's fine density
    K = solve.fine_kernel(T, w.G, w.r_split, w.r_cut)
    idx = np.arange(T)
    afc = af.cpu().numpy()
    acc_c = ac.cpu().numpy()
    for tile in (big["dense"], big["sparse"]):
        ix, iy, iz = _tile_xyz(tile, nt)
        org = np.array([ix * t - b, iy * t - b, iz * t - b])
        win = rho_f[np.ix_((org[2] + idx) % n, (org[1] + idx) % n, (org[0] + idx) % n)]
        want = solve.accel_tile(win, K)[:, b:b + t, b:b + t, b:b + t]
        got = afc[:, iz * t:(iz + 1) * t, iy * t:(iy + 1) * t, ix * t:(ix + 1) * t]
        assert rel_rms(got, want) < RHO_TOL, tile
    # sampled interpolations from the GPU's meshes
    rng = np.random.default_rng(3)
    for s in range(2):
        sel = rng.choice(xs[s].shape[0], 20000, replace=False)
        xsel = xs[s][torch.from_numpy(sel).cuda()].contiguous()
        a = pm.interpolate(xsel, ac, af).cpu().numpy()
        xp = xsel.cpu().numpy().astype(np.float64)
        want = mesh.cic_interp(acc_c, xp / w.coarse_ratio, n // w.coarse_ratio) + mesh.cic_interp(afc, xp, n)
        assert rel_rms(a, want) < 1e-6


def test_batched512_fixed_mass_and_fused_step_equals_plain(big):
    w = big["w"]
    pm, codes = big[1]
    rc, rf = pm.zeros_meshes(fixed=True)
    pm.deposit_codes(codes, rc, rf)
    pm.check()
    total = sum(w.counts[s] * mesh.fixed_mass(w.mass[s]) for s in range(2))
    assert int(rf.sum().item()) == total and int(rc.sum().item()) == total
    del rc, rf
    out = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in codes]
    pm.set_graphs(True)
    for _ in range(2):
        pm.step(codes, out, 1.0, 1.0)
    pm.check()
    pm.set_graphs(False)
    xs, vs = zip(*[pm.decompress(s, codes[s]) for s in range(2)])
    rc, rf = pm.density(list(xs), fixed=True)
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    nc = w.n_fine // 4
    for s in range(2):
        x, v = xs[s].clone(), vs[s].clone()
        pm.kick_drift(x, v, ac, af, 1.0, 1.0)
        plain = pm.compress(s, x, v, out=pm.empty_codes(x.shape[0], esc_cap=out[s].esc.shape[0]))
        pm.check()
        assert torch.equal(out[s].vmax, plain.vmax)
        assert device_records_equal(out[s], plain, nc)
        del x, v, plain
