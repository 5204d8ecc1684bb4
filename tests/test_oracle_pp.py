"""Pins for the oracle PP force (Eq. 4): a two-body pair gives Newton's
inverse-square attraction along the separation, equal and opposite; pairs in
different fine cells or closer than r_soft do not interact; total momentum
is conserved; and the grouped sum equals a brute-force all-pairs sum with a
same-cell mask."""
import numpy as np

from oracle import pp

G = 1.0 / (4 * np.pi)


def test_two_body_inverse_square():
    x0 = np.array([[3.2, 5.1, 7.3]])
    x1 = np.array([[3.7, 5.4, 7.9]])
    a0, a1 = pp.pp_accel([x0, x1], (8.0, 0.04), G, 0.05)
    d = x1[0] - x0[0]
    r = np.linalg.norm(d)
    np.testing.assert_allclose(np.linalg.norm(a0[0]), G * 0.04 / r ** 2, rtol=1e-14)
    np.testing.assert_allclose(a0[0] / np.linalg.norm(a0[0]), d / r, rtol=1e-14)      # towards the partner
    np.testing.assert_allclose(8.0 * a0[0], -0.04 * a1[0], rtol=1e-14)                 # third law


def test_no_interaction_across_cells_or_below_softening():
    x = np.array([[1.99, 2.5, 2.5], [2.01, 2.5, 2.5],      # 0.02 apart, different cells
                  [5.1, 5.1, 5.1], [5.13, 5.1, 5.1]])      # same cell, 0.03 < r_soft
    (a,) = pp.pp_accel([x], (1.0,), G, 0.05)
    np.testing.assert_array_equal(a, 0.0)


def test_momentum_and_brute_force():
    rng = np.random.default_rng(7)
    n = 6
    # clustered: 3 cells with many members, plus scattered singles
    xs = [np.concatenate([rng.random((40, 3)) * 0.999 + [1, 2, 3], rng.random((10, 3)) * n]),
          np.concatenate([rng.random((60, 3)) * 0.999 + [1, 2, 3], rng.random((30, 3)) * 0.999 + [4, 0, 5],
                          rng.random((50, 3)) * n])]
    masses = (8.0, 0.04)
    r_soft = 0.05
    acc = pp.pp_accel(xs, masses, G, r_soft)
    mom = sum(m * a.sum(0) for m, a in zip(masses, acc))
    scale = sum(m * np.abs(a).sum() for m, a in zip(masses, acc))
    assert np.all(np.abs(mom) <= 1e-12 * scale)
    # brute force: every ordered pair, masked to same cell and r >= r_soft
    x = np.concatenate(xs)
    m = np.concatenate([np.full(len(a), mm) for a, mm in zip(xs, masses)])
    ref = np.zeros_like(x)
    for i in range(len(x)):
        for j in range(len(x)):
            if i == j or np.any(np.floor(x[i]) != np.floor(x[j])):
                continue
            d = x[j] - x[i]
            r = np.sqrt(d @ d)
            if r >= r_soft:
                ref[i] += G * m[j] * d / r ** 3
    np.testing.assert_allclose(np.concatenate(acc), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
