"""Oracle particle-particle (PP) force -- TEST INFRASTRUCTURE ONLY (imported
by tests/, __graft_entry__.smoke() and bench.py's CPU baseline, never by the
product path).

Eq. 4 (Sec. 2.1): below the mesh scale the short-range PM force is
supplemented by a direct pairwise sum over the particles that share particle
i's cell of the short-range (fine) interpolation mesh,

    F_i = G m_i sum_{j != i, same cell} m_j (x_j - x_i) / |x_j - x_i|^3,

so the acceleration is a_i = F_i / m_i.  The sum is truncated below the
softening length r_soft (Sec. 2.1 chooses r_soft as 0.05 of the mean
inter-particle spacing, L / (20 n_p)).  Readings where the paper is silent:

  * "cell" is the fine-mesh cell [i, i+1)^3 that contains the particle
    (mesh points at integer coordinates, as for CIC), i.e. floor(x);
  * "truncated below r_soft": a pair closer than r_soft contributes nothing
    (no Plummer-type smoothing);
  * both species take part, each with its own mass, CDM-nu pairs included.

Particles of one cell are less than one cell apart, so no periodic image is
needed.  Pins: tests/test_oracle_pp.py.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def pp_accel(xs: Sequence[np.ndarray], masses: Sequence[float], G: float, r_soft: float) -> List[np.ndarray]:
    """Per-particle PP acceleration of each species (float64), Eq. 4 / m_i."""
    xs = [np.asarray(x, np.float64).reshape(-1, 3) for x in xs]
    x = np.concatenate(xs) if xs else np.zeros((0, 3))
    m = np.concatenate([np.full(len(a), float(mi)) for a, mi in zip(xs, masses)])
    acc = np.zeros_like(x)
    if len(x):
        cell = np.floor(x).astype(np.int64)
        key = cell[:, 0] + (1 << 21) * (cell[:, 1] + (1 << 21) * cell[:, 2])
        order = np.argsort(key, kind="stable")
        bounds = np.flatnonzero(np.diff(key[order])) + 1
        for group in np.split(order, bounds):
            if len(group) < 2:
                continue
            d = x[group][None, :, :] - x[group][:, None, :]        # d[i, j] = x_j - x_i
            r = np.sqrt(np.sum(d * d, axis=2))
            with np.errstate(divide="ignore", invalid="ignore"):
                w = np.where(r >= r_soft, m[group][None, :] / r ** 3, 0.0)
            np.fill_diagonal(w, 0.0)
            acc[group] = G * np.einsum("ij,ijk->ik", w, d)
    out, k = [], 0
    for a in xs:
        out.append(acc[k:k + len(a)])
        k += len(a)
    return out
