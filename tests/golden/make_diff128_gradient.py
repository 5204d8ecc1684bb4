"""Writes tests/golden/diff128_gradient.txt: the float64 oracle's gradient of
the differentiable 128^3 trajectory, for the GPU test at the workload's own
shape (tests/test_gpu_adjoint.py::test_diff128_gradient_matches_oracle).

Calls only oracle/ (oracle.adjoint: forward steps, loss, reverse-mode
gradient) and the seeded input recipe of this file, shared with the test
through diff128_inputs().  Run from the repository root:

    python tests/golden/make_diff128_gradient.py

The oracle needs about twenty minutes on one core (ten 128^3 steps forward
and back, twice: from the start and from a start moved by 1e-5 cells, which
measures how far a float32 trajectory's gradient may lie from the float64
one; plus a forward pass for the loss).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUT = os.path.join(HERE, "diff128_gradient.txt")
N_FINE, N_CDM_SIDE = 128, 64
STEPS, EVERY, BETA, C_KICK, C_DRIFT = 10, 2, 0.3, 0.5, 0.5
N_SAMPLE, N_DIRS = 1024, 4
PERTURB = 1e-5


def diff128_inputs():
    """Seeded inputs of the differentiable 128^3 workload: the CDM lattice q
    (64^3 points, spacing 2 fine cells, offset 1), the displacement psi
    (N(0, 0.2^2) cells per coordinate, float32), the 128^3 neutrinos of the
    diff128 recipe with their velocities scaled by 0.2, and a target density
    uniform in [0, 0.02)."""
    from synth import make_workload
    g = (np.arange(N_CDM_SIDE) + 0.5) * (N_FINE / N_CDM_SIDE)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)
    rng = np.random.default_rng(2016)
    psi = (rng.standard_normal(q.shape) * 0.2).astype(np.float32)
    target = (rng.random((N_FINE,) * 3) * 0.02).astype(np.float32)
    w = make_workload("diff128")
    x_nu = w.x[1]
    v_nu = (w.v[1] * 0.2).astype(np.float32)
    cfg = dict(n_fine=N_FINE, coarse_ratio=1, tile=N_FINE, buffer=0, cmp_ratio=4, vel_bits=16,
               G=1 / (4 * np.pi), mass=(8.0, 0.04), count=(q.shape[0], x_nu.shape[0]), deposit_mode=1)
    return cfg, q, psi, x_nu, v_nu, target


def sample_index():
    return np.sort(np.random.default_rng(2018).choice(N_CDM_SIDE ** 3, N_SAMPLE, replace=False))


def directions():
    return [np.random.default_rng(2019 + k).standard_normal((N_CDM_SIDE ** 3, 3)) for k in range(N_DIRS)]


def start(q, psi, n):
    """x0 = q + psi wrapped into [0, n), rounded to float32 as the library forms it."""
    x = (q + psi).astype(np.float32).astype(np.float64)
    return np.mod(x, n)


def main():
    from oracle import adjoint
    cfg, q, psi, x_nu, v_nu, target = diff128_inputs()
    n = cfg["n_fine"]
    x0 = [start(q, psi, n), x_nu.astype(np.float64)]
    v0 = [BETA * psi.astype(np.float64), v_nu.astype(np.float64)]
    t64 = target.astype(np.float64)
    loss = adjoint.loss(adjoint.forward(x0, v0, cfg, C_KICK, C_DRIFT, STEPS)[-1][0], cfg, t64)
    lx, lv = adjoint.gradient(x0, v0, cfg, C_KICK, C_DRIFT, STEPS, t64)
    grad = lx[0] + BETA * lv[0]
    # conditioning: the same gradient from a start moved by PERTURB cells per
    # coordinate (the size of float32 rounding of positions near 64-128 cells):
    # the spread a float32 trajectory can show against the float64 one
    rng = np.random.default_rng(2020)
    xp = [np.mod(x0[0] + PERTURB * rng.standard_normal(x0[0].shape), n), x0[1] + 0.0]
    xp[1] = np.mod(xp[1] + PERTURB * rng.standard_normal(xp[1].shape), n)
    lxp, lvp = adjoint.gradient(xp, v0, cfg, C_KICK, C_DRIFT, STEPS, t64)
    gradp = lxp[0] + BETA * lvp[0]
    idx = sample_index()
    sens = float(np.sqrt(np.mean((gradp[idx] - grad[idx]) ** 2)) / np.sqrt(np.mean(grad[idx] ** 2)))
    with open(OUT, "w") as f:
        f.write("# Float64 oracle (oracle/adjoint.py) gradient dL/dpsi of L = sum_c (rho_K(c) - target(c))^2\n"
                "# after K PM steps of the single periodic 128^3 mesh (Eqs. 1-3 of Sec. 2.1, CIC of Sec. 2.3,\n"
                "# kick-drift), x0 = q + psi (float32-rounded), v0 = beta psi; inputs from diff128_inputs() in\n"
                "# make_diff128_gradient.py, which wrote this file (it calls only oracle/).  sensitivity: the\n"
                "# relative RMS change of the sampled gradient when every start coordinate moves by\n"
                "# N(0, perturb^2) cells.\n")
        f.write(f"steps {STEPS}\nbeta {BETA!r}\nc_kick {C_KICK!r}\nc_drift {C_DRIFT!r}\n")
        f.write(f"loss {float(loss)!r}\n")
        f.write(f"grad_rms {float(np.sqrt(np.mean(grad * grad)))!r}\n")
        f.write(f"perturb {PERTURB!r}\n")
        f.write(f"sensitivity {sens!r}\n")
        for i in idx:
            g = [float(c) for c in grad[i]]
            f.write(f"sample {int(i)} {g[0]!r} {g[1]!r} {g[2]!r}\n")
        for k, d in enumerate(directions()):
            f.write(f"proj {k} {float(np.sum(grad * d))!r} {float(np.sum(np.abs(grad * d)))!r}\n")
    print(OUT)


if __name__ == "__main__":
    main()
