"""Parity at the benchmark's full size (256^3 fine mesh, 64 tiles of 96^3,
2.10M CDM + 16.78M neutrinos, 8-bit velocities), in the launch configuration
bench.py times: sampled outputs the oracle can compute one by one (a density
sub-box, the coarse solve, two tile solves, sampled interpolations) and
properties that hold at any size (exact fixed-point mass, momentum balance,
particle conservation, fused step == plain path bit for bit)."""
import numpy as np
import pytest
import torch

from oracle import mesh, solve
from synth import make_workload
from tests.helpers import oracle_codes_from_lib, records, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_1611_01545_gb300 import PM
    w = make_workload("two_level256")
    cfg = w.config()
    out = {"w": w, "cfg": cfg}
    for mode in (0, 1):
        pm = PM(dict(cfg, deposit_mode=mode))
        codes = []
        for s in range(2):
            x = torch.from_numpy(w.x[s]).cuda()
            v = torch.from_numpy(w.v[s]).cuda()
            codes.append(pm.compress(s, x, v, out=pm.empty_codes(x.shape[0], esc_cap=x.shape[0] // 255 + 1)))
        pm.check()
        out[mode] = (pm, codes)
    return out


def test_density_coarse_and_tiles_match_oracle(full):
    w, cfg = full["w"], full["cfg"]
    pm, codes = full[0]
    xs = [pm.decompress(s, codes[s])[0] for s in range(2)]
    rc, rf = pm.zeros_meshes()
    for s in range(2):
        pm.deposit(s, xs[s], rc, rf)
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    pm.check()
    rho_f = rf.cpu().numpy().astype(np.float64)
    rho_c = rc.cpu().numpy().astype(np.float64)
    n = w.n_fine
    # density of a 16^3 sub-box from the particles around it
    lo, hi = np.array([100, 40, 200]), np.array([116, 56, 216])
    sub = np.zeros((18, 18, 18))
    for s in range(2):
        x = xs[s].cpu().numpy().astype(np.float64)
        sel = np.all((x >= lo - 1) & (x < hi + 1), axis=1)
        sub += mesh.cic_deposit(x[sel] - (lo - 1), w.mass[s], 64)[:18, :18, :18]
    got = rho_f[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    assert rel_rms(got, sub[1:17, 1:17, 1:17]) < 1e-5
    # coarse long-range solve on the GPU's own coarse density
    ref_c = solve.accel_periodic(rho_c, float(w.coarse_ratio), w.G, w.r_split)
    assert rel_rms(ac.cpu().numpy(), ref_c) < 1e-5
    # two sampled tile solves on the GPU's fine density
    t, b = w.tile, w.buffer
    T = t + 2 * b
    K = solve.fine_kernel(T, w.G, w.r_split, w.r_cut)
    idx = np.arange(T)
    afc = af.cpu().numpy()
    for (ix, iy, iz) in [(0, 0, 0), (3, 1, 2)]:
        org = np.array([ix * t - b, iy * t - b, iz * t - b])
        win = rho_f[np.ix_((org[2] + idx) % n, (org[1] + idx) % n, (org[0] + idx) % n)]
        a_t = solve.accel_tile(win, K)[:, b:b + t, b:b + t, b:b + t]
        got = afc[:, iz * t:(iz + 1) * t, iy * t:(iy + 1) * t, ix * t:(ix + 1) * t]
        assert rel_rms(got, a_t) < 1e-5
    # sampled interpolations from the GPU's meshes
    rng = np.random.default_rng(1)
    for s in range(2):
        sel = rng.choice(xs[s].shape[0], 20000, replace=False)
        xsel = xs[s][torch.from_numpy(sel).cuda()].contiguous()
        a = pm.interpolate(xsel, ac, af).cpu().numpy()
        xp = xsel.cpu().numpy().astype(np.float64)
        ref = mesh.cic_interp(ac.cpu().numpy(), xp / w.coarse_ratio, n // w.coarse_ratio) + mesh.cic_interp(afc, xp, n)
        assert rel_rms(a, ref) < 1e-6
        # momentum balance over all particles (pair forces are antisymmetric)
    mom, scale = np.zeros(3), 0.0
    for s in range(2):
        a = pm.interpolate(xs[s], ac, af).double()
        mom += w.mass[s] * a.sum(0).cpu().numpy()
        scale += w.mass[s] * a.abs().sum().item()
    assert np.all(np.abs(mom) < 1e-4 * scale)


def test_fixed_point_mass_is_exact(full):
    w = full["w"]
    pm, codes = full[1]
    rc, rf = pm.zeros_meshes(fixed=True)
    pm.deposit_codes(codes, rc, rf)
    pm.check()
    total = sum(w.counts[s] * mesh.fixed_mass(w.mass[s]) for s in range(2))
    assert int(rf.sum().item()) == total
    assert int(rc.sum().item()) == total


def test_fused_step_equals_plain_path_at_full_size(full):
    w = full["w"]
    pm, codes = full[1]
    out = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in codes]
    pm.step(codes, out, 1.0, 1.0)
    pm.check()
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
        a = oracle_codes_from_lib(out[s], nc, w.vel_bits)
        b = oracle_codes_from_lib(plain, nc, w.vel_bits)
        assert a.vmax == b.vmax and a.counts().sum() == w.counts[s]
        np.testing.assert_array_equal(a.cnt, b.cnt)
        np.testing.assert_array_equal(records(a), records(b))
