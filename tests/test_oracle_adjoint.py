"""Pins for the oracle adjoint (reverse mode of the single-mesh step):
transposition identities of each linear piece and central finite
differences of the final-density loss."""
import numpy as np
import pytest

from oracle import adjoint, mesh, solve

G = 1.0 / (4 * np.pi)


def test_solve_adjoint_is_transpose():
    rng = np.random.default_rng(1)
    n = 12
    rho = rng.standard_normal((n, n, n))
    lam = rng.standard_normal((3, n, n, n))
    lhs = np.sum(solve.accel_periodic(rho, 1.0, G) * lam)
    rhs = np.sum(rho * adjoint.accel_periodic_adjoint(lam, 1.0, G))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_vector_deposit_is_interpolation_transpose():
    rng = np.random.default_rng(2)
    n = 8
    x = rng.random((50, 3)) * n
    lam = rng.standard_normal((50, 3))
    F = rng.standard_normal((3, n, n, n))
    lhs = np.sum(adjoint.cic_deposit_vector(lam, x, n) * F)
    rhs = np.sum(lam * mesh.cic_interp(F, x, n))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_grad_gather_matches_finite_difference():
    rng = np.random.default_rng(3)
    n = 8
    f = rng.standard_normal((n, n, n))
    x = 1 + 0.2 + rng.random((20, 3)) * 0.6 + rng.integers(0, 5, (20, 3))   # away from cell faces
    g = adjoint.cic_grad_gather(f, x, n)
    eps = 1e-4
    F3 = np.stack([f, f, f])
    for d in range(3):
        e = np.zeros(3)
        e[d] = eps
        fd = (mesh.cic_interp(F3, x + e, n)[:, 0] - mesh.cic_interp(F3, x - e, n)[:, 0]) / (2 * eps)
        np.testing.assert_allclose(g[:, d], fd, rtol=1e-8, atol=1e-10)


def _setup(seed=4, n=16, n0=12, n1=30):
    rng = np.random.default_rng(seed)
    cfg = dict(n_fine=n, coarse_ratio=1, mass=(8.0, 0.04), G=G)
    xs = [rng.random((n0, 3)) * n, rng.random((n1, 3)) * n]
    vs = [rng.standard_normal((n0, 3)) * 0.3, rng.standard_normal((n1, 3)) * 0.5]
    target = rng.random((n, n, n)) * 0.05
    return cfg, xs, vs, target


def _away_from_faces(states, s, i, d, margin):
    return all(margin < (st[0][s][i, d] % 1.0) < 1 - margin for st in states)


def test_gradient_matches_central_differences():
    cfg, xs, vs, target = _setup()
    steps, ck, cd = 3, 0.5, 0.5
    lam_x, lam_v = adjoint.gradient(xs, vs, cfg, ck, cd, steps, target)
    states = adjoint.forward(xs, vs, cfg, ck, cd, steps)
    eps = 1e-3
    checked = 0
    for s in (0, 1):
        for i in range(xs[s].shape[0]):
            for d in range(3):
                if checked >= 12 or not _away_from_faces(states, s, i, d, 2 * eps):
                    continue
                for which, lam in (("x", lam_x), ("v", lam_v)):
                    def L(delta):
                        x2 = [a.copy() for a in xs]
                        v2 = [a.copy() for a in vs]
                        (x2 if which == "x" else v2)[s][i, d] += delta
                        return adjoint.loss(adjoint.forward(x2, v2, cfg, ck, cd, steps)[-1][0], cfg, target)
                    fd = (L(eps) - L(-eps)) / (2 * eps)
                    assert abs(fd - lam[s][i, d]) <= 1e-5 * max(abs(fd), 1e-3), (which, s, i, d, fd, lam[s][i, d])
                checked += 1
    assert checked >= 8


def test_directional_derivative():
    cfg, xs, vs, target = _setup(seed=5)
    steps, ck, cd = 2, 0.5, 0.5
    lam_x, lam_v = adjoint.gradient(xs, vs, cfg, ck, cd, steps, target)
    rng = np.random.default_rng(6)
    dx = [rng.standard_normal(a.shape) for a in xs]
    eps = 1e-4
    def L(t):
        x2 = [a + t * b for a, b in zip(xs, dx)]
        return adjoint.loss(adjoint.forward(x2, vs, cfg, ck, cd, steps)[-1][0], cfg, target)
    fd = (L(eps) - L(-eps)) / (2 * eps)
    an = sum(np.sum(l * b) for l, b in zip(lam_x, dx))
    assert abs(fd - an) <= 1e-2 * abs(an)
