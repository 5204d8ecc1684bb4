"""Pins for the oracle CIC deposit / interpolation (Sec. 2.3 density and
inverse force interpolation): hand-computed weights, mass conservation,
exact reproduction of linear fields, the deposit/interpolation transpose
relation, the tile inclusion rule and the fixed-point deposit."""
import numpy as np
import pytest

from oracle import mesh


def test_single_particle_weights():
    n = 8
    r = mesh.cic_deposit([[2.0, 3.0, 4.0]], 5.0, n)
    assert r[4, 3, 2] == 5.0 and r.sum() == 5.0
    r = mesh.cic_deposit([[0.5, 0.5, 0.5]], 8.0, n)
    assert np.all(r[0:2, 0:2, 0:2] == 1.0) and r.sum() == 8.0
    r = mesh.cic_deposit([[0.25, 0.0, 0.0]], 1.0, n)
    assert r[0, 0, 0] == 0.75 and r[0, 0, 1] == 0.25
    r = mesh.cic_deposit([[7.5, 0.0, 7.75]], 1.0, n)      # periodic wrap in x and z
    assert r[7, 0, 7] == 0.5 * 0.25 and r[0, 0, 0] == 0.5 * 0.75 and r[7, 0, 0] == 0.5 * 0.25


def test_mass_conservation():
    rng = np.random.default_rng(1)
    x = rng.random((5000, 3)) * 16
    m = rng.random(5000)
    assert abs(mesh.cic_deposit(x, m, 16).sum() - m.sum()) < 1e-11 * m.sum()


def test_interp_reproduces_linear_field():
    n = 16
    g = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    f = np.stack([2 * x + 1, -y + 3 * z, x + y + z])
    rng = np.random.default_rng(2)
    p = 1 + rng.random((200, 3)) * (n - 3)              # stay away from the periodic seam
    out = mesh.cic_interp(f, p, n)
    expect = np.stack([2 * p[:, 0] + 1, -p[:, 1] + 3 * p[:, 2], p.sum(1)], axis=1)
    np.testing.assert_allclose(out, expect, atol=1e-12)


def test_deposit_interp_transpose():
    rng = np.random.default_rng(3)
    n = 8
    x = rng.random((300, 3)) * n
    m = rng.random(300)
    f = rng.standard_normal((3, n, n, n))
    rho = mesh.cic_deposit(x, m, n)
    lhs = np.array([np.sum(rho * f[d]) for d in range(3)])
    rhs = (m[:, None] * mesh.cic_interp(f, x, n)).sum(0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_tile_inclusion_and_window():
    rng = np.random.default_rng(4)
    n, T = 32, 16
    x = rng.random((4000, 3)) * n
    origin = np.array([24.0, 4.0, 30.0])                # wraps in x and z
    rho_t = mesh.tile_deposit(x, 1.0, origin, T, n)
    full = mesh.cic_deposit(x, 1.0, n)
    idx = [(int(origin[d]) + np.arange(T)) % n for d in range(3)]
    window = full[np.ix_(idx[2], idx[1], idx[0])]
    # cells 1..T-2 only receive particles whose whole stencil is inside the tile
    np.testing.assert_allclose(rho_t[1:-1, 1:-1, 1:-1], window[1:-1, 1:-1, 1:-1], atol=1e-12)
    # a particle straddling the tile edge is skipped entirely
    r = mesh.tile_deposit([[origin[0] - 0.5, 10.0, origin[2] + 3]], 1.0, origin, T, n)
    assert r.sum() == 0.0
    r = mesh.tile_deposit([[origin[0] + T - 1.5, 10.0, (origin[2] + 3) % n]], 1.0, origin, T, n)
    assert r.sum() == 1.0


def test_fixed_point_exact_mass_and_agreement():
    rng = np.random.default_rng(5)
    n = 16
    x = (rng.random((3000, 3)) * n).astype(np.float32)
    x[x >= n] = 0
    M = mesh.fixed_mass(0.04)
    assert M == round(0.04 * 2 ** 32)
    rho = mesh.cic_deposit_fixed(x, M, n)
    assert rho.dtype == np.int64 and int(rho.sum()) == 3000 * M
    ref = mesh.cic_deposit(x.astype(np.float64), 0.04, n) * 2.0 ** 32
    # weights are quantised to 2^-20 of a cell, so each term is within ~M 2^-19 of its real value
    assert np.max(np.abs(rho - ref)) <= 1e-5 * ref.max()
    # order independence (bit-exact)
    perm = rng.permutation(3000)
    np.testing.assert_array_equal(mesh.cic_deposit_fixed(x[perm], M, n), rho)


def test_fixed_point_corner_split_hand_case():
    # x = 0.25 in every dim: a1 = 2^18; hi = (M 2^18 + 2^19) >> 20 = M/4 for M divisible by 4.
    M = 1 << 32
    r = mesh.cic_deposit_fixed(np.array([[0.25, 0.25, 0.25]], np.float32), M, 4)
    assert r[0, 0, 0] == M * 27 // 64 and r[1, 1, 1] == M // 64 and r.sum() == M


@pytest.mark.parametrize("n", [4, 8])
def test_interp_single_cell_field(n):
    f = np.zeros((3, n, n, n))
    f[0, 1, 1, 1] = 1.0
    out = mesh.cic_interp(f, [[1.5, 1.0, 1.0], [0.5, 0.5, 0.5]], n)
    np.testing.assert_allclose(out[:, 0], [0.5, 0.125])
