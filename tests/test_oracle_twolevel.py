"""Pins for the coarse-from-fine identities of CIC: restricting the fine CIC
density equals depositing the particles on the coarse mesh directly, and
interpolating the prolongated coarse field on the fine mesh equals
interpolating the coarse field directly; restriction conserves mass and is
the transpose of prolongation."""
import numpy as np

from oracle import mesh


def test_restrict_equals_coarse_deposit():
    rng = np.random.default_rng(12)
    n, rc = 32, 4
    x = rng.random((3000, 3)) * n
    m = rng.random(3000) + 0.5
    rho_f = mesh.cic_deposit(x, m, n)
    direct = mesh.cic_deposit(x / rc, m, n // rc)
    np.testing.assert_allclose(mesh.restrict(rho_f, rc), direct, rtol=1e-12, atol=1e-12 * direct.max())
    np.testing.assert_allclose(mesh.restrict(rho_f, rc).sum(), m.sum(), rtol=1e-12)


def test_prolong_interpolation_equals_coarse_interpolation():
    rng = np.random.default_rng(13)
    n, rc = 32, 4
    nc = n // rc
    a_c = rng.standard_normal((3, nc, nc, nc))
    x = rng.random((500, 3)) * n
    a_f = mesh.prolong(a_c, rc)
    np.testing.assert_allclose(mesh.cic_interp(a_f, x, n), mesh.cic_interp(a_c, x / rc, nc), rtol=1e-12, atol=1e-12)


def test_restrict_is_transpose_of_prolong():
    rng = np.random.default_rng(14)
    n, rc = 16, 4
    f = rng.standard_normal((n, n, n))
    g = rng.standard_normal((n // rc,) * 3)
    np.testing.assert_allclose(np.sum(mesh.restrict(f, rc) * g), np.sum(f * mesh.prolong(g, rc)), rtol=1e-12)
