"""GPU parity of the CIC deposit (Sec. 2.3) and the Fourier solve (Eqs. 1-3,
two-level split of Sec. 2.1) against the oracle, plus closed-form checks."""
import numpy as np
import pytest
import torch

from oracle import codec, mesh, solve, step
from synth import make_workload
from tests.helpers import cfg_of, lib_codes_from_oracle, rel_rms

pytestmark = pytest.mark.gpu

DENSITY_TOL = 1e-5   # float32 deposit vs float64, relative RMS
MESH_ACC_TOL = 1e-5  # float32 FFT solve vs float64 on the same density


def _pm(cfg):
    from paper_1611_01545_gb300 import PM
    return PM(cfg)


def _decoded(w, vel_bits=None):
    vb = vel_bits or w.vel_bits
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, vb) for s in range(2)]
    xs = [codec.decompress(c, w.n_fine)[0] for c in codes]
    return codes, xs


CASES = [("single64", 16, 32), ("two_level64", 16, 40), ("two_level128_t96", 24, 48)]


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_deposit_float_parity(name, n_cdm, n_nu):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    cfg = cfg_of(w)
    pm = _pm(cfg)
    codes, xs = _decoded(w)
    rc, rf = pm.zeros_meshes()
    for s in range(2):
        pm.deposit(s, torch.from_numpy(xs[s]).cuda(), rc, rf)
    pm.check()
    ref_f = step.density_fine(xs, cfg)
    assert rel_rms(rf.cpu().numpy(), ref_f) < DENSITY_TOL
    if w.coarse_ratio > 1:
        ref_c = step.density_coarse(xs, cfg)
        assert rel_rms(rc.cpu().numpy(), ref_c) < DENSITY_TOL
    # fused decode + deposit from the codes (shared-memory binned)
    rc2, rf2 = pm.zeros_meshes()
    pm.deposit_codes([lib_codes_from_oracle(c) for c in codes], rc2, rf2)
    pm.check()
    assert rel_rms(rf2.cpu().numpy(), ref_f) < DENSITY_TOL
    if w.coarse_ratio > 1:
        assert rel_rms(rc2.cpu().numpy(), ref_c) < DENSITY_TOL
        # coarse density by restriction of the fine one (what the float step uses)
        rc3 = pm.restrict(rf)
        pm.check()
        assert rel_rms(rc3.cpu().numpy(), ref_c) < DENSITY_TOL


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_deposit_fixed_bit_exact(name, n_cdm, n_nu):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    cfg = cfg_of(w, deposit_mode=1)
    pm = _pm(cfg)
    codes, xs = _decoded(w)
    nf, rc_ = w.n_fine, w.coarse_ratio
    ref_f = sum(mesh.cic_deposit_fixed(xs[s], mesh.fixed_mass(w.mass[s]), nf) for s in range(2))
    rc, rf = pm.zeros_meshes(fixed=True)
    for s in range(2):
        pm.deposit_fixed(s, torch.from_numpy(xs[s]).cuda(), rc, rf)
    pm.check()
    np.testing.assert_array_equal(rf.cpu().numpy(), ref_f)
    total = sum(xs[s].shape[0] * mesh.fixed_mass(w.mass[s]) for s in range(2))
    assert int(rf.sum()) == total
    rc2, rf2 = pm.zeros_meshes(fixed=True)
    pm.deposit_codes([lib_codes_from_oracle(c) for c in codes], rc2, rf2)
    pm.check()
    np.testing.assert_array_equal(rf2.cpu().numpy(), ref_f)
    if rc_ > 1:
        ref_c = sum(mesh.cic_deposit_fixed((xs[s] / np.float32(rc_)).astype(np.float32),
                                           mesh.fixed_mass(w.mass[s]), nf // rc_) for s in range(2))
        np.testing.assert_array_equal(rc.cpu().numpy(), ref_c)
        np.testing.assert_array_equal(rc2.cpu().numpy(), ref_c)
        assert int(rc2.sum()) == total


def test_tile_window_matches_literal_tile_deposit():
    w = make_workload("two_level64", n_cdm=16, n_nu=40)
    cfg = cfg_of(w)
    pm = _pm(cfg)
    _, xs = _decoded(w)
    rc, rf = pm.zeros_meshes()
    for s in range(2):
        pm.deposit(s, torch.from_numpy(xs[s]).cuda(), rc, rf)
    T, t, b = w.tile + 2 * w.buffer, w.tile, w.buffer
    nts = w.n_fine // t
    for tile in (0, 5, nts ** 3 - 1):
        got = pm.tile_density(rf, tile).cpu().numpy()
        ix, iy, iz = tile % nts, (tile // nts) % nts, tile // nts ** 2
        origin = np.array([ix * t - b, iy * t - b, iz * t - b], float)
        ref = sum(mesh.tile_deposit(xs[s], w.mass[s], origin, T, w.n_fine) for s in range(2))
        assert rel_rms(got[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1]) < DENSITY_TOL


def _oracle_fine_acc_mesh(rho_f, cfg):
    """Oracle short-range acceleration mesh: each tile's interior from its own FFT solve."""
    n, t, b = cfg["n_fine"], cfg["tile"], cfg["buffer"]
    T = t + 2 * b
    K = solve.fine_kernel(T, cfg["G"], cfg["r_split"], cfg["r_cut"])
    out = np.zeros((3, n, n, n))
    idx = np.arange(T)
    for (ix, iy, iz), o in step.tile_origins(n, t):
        org = (o - b).astype(int)
        win = rho_f[np.ix_((org[2] + idx) % n, (org[1] + idx) % n, (org[0] + idx) % n)]
        a = solve.accel_tile(win, K)
        out[:, iz * t:(iz + 1) * t, iy * t:(iy + 1) * t, ix * t:(ix + 1) * t] = a[:, b:b + t, b:b + t, b:b + t]
    return out


@pytest.mark.parametrize("name,n_cdm,n_nu", CASES)
def test_solve_parity(name, n_cdm, n_nu):
    w = make_workload(name, n_cdm=n_cdm, n_nu=n_nu)
    cfg = cfg_of(w)
    pm = _pm(cfg)
    _, xs = _decoded(w)
    rho_f = step.density_fine(xs, cfg)
    ac, af = pm.zeros_acc()
    if w.coarse_ratio > 1:
        rho_c = step.density_coarse(xs, cfg)
        pm.solve(torch.from_numpy(rho_c.astype(np.float32)).cuda(), torch.from_numpy(rho_f.astype(np.float32)).cuda(),
                 ac, af)
        pm.check()
        ref_c = solve.accel_periodic(rho_c.astype(np.float32).astype(np.float64), float(w.coarse_ratio), w.G,
                                     w.r_split)
        assert rel_rms(ac.cpu().numpy(), ref_c) < MESH_ACC_TOL
        ref_f = _oracle_fine_acc_mesh(rho_f.astype(np.float32).astype(np.float64), cfg)
        assert rel_rms(af.cpu().numpy(), ref_f) < MESH_ACC_TOL
    else:
        pm.solve(None, torch.from_numpy(rho_f.astype(np.float32)).cuda(), None, af)
        pm.check()
        ref = solve.accel_periodic(rho_f.astype(np.float32).astype(np.float64), 1.0, w.G)
        assert rel_rms(af.cpu().numpy(), ref) < MESH_ACC_TOL


@pytest.mark.parametrize("n,m_vec", [(64, (1, 0, 0)), (64, (3, 5, 2)), (128, (7, 1, 4)), (32, (16, 1, 1))])
def test_plane_wave_closed_form_gpu(n, m_vec):
    # Eq. 2-3: rho = A cos(k.x) -> a = -4 pi G A k_hat sin(k.x) / |k| (Nyquist components dropped).
    G = 1 / (4 * np.pi)
    pm = _pm(dict(n_fine=n, coarse_ratio=1, tile=n, buffer=0, cmp_ratio=4, vel_bits=16, G=G, mass=(1.0, 1.0)))
    g = np.arange(n)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    k = 2 * np.pi * np.array(m_vec, float) / n
    ph = k[0] * x + k[1] * y + k[2] * z
    A = 0.3
    ac, af = pm.zeros_acc()
    pm.solve(None, torch.from_numpy((A * np.cos(ph)).astype(np.float32)).cuda(), None, af)
    pm.check()
    kk = np.linalg.norm(k)
    kg = np.where(2 * np.abs(np.array(m_vec)) == n, 0.0, k)
    for d in range(3):
        ref = -4 * np.pi * G * A * kg[d] / kk ** 2 * np.sin(ph)
        np.testing.assert_allclose(af[d].cpu().numpy(), ref, atol=2e-6 * 4 * np.pi * G * A / kk)
