"""Oracle adjoint of the single-mesh PM step -- TEST INFRASTRUCTURE ONLY.

The paper has no adjoint; this is the reverse-mode derivative of the forward
step of oracle/step.py (single periodic mesh, Eqs. 1-3 of Sec. 2.1, CIC of
Sec. 2.3, kick-drift) for a final-density loss, written from the chain rule:

  forward, per step:  rho = sum_p m_p W(x_p - c);  a = A rho (Eqs. 2-3);
                      a_p = sum_c a(c) W(x_p - c);  v' = v + c_k a_p;
                      x' = x + c_d v'   (periodic wrap: derivative 1)
  loss:               L = sum_c (rho_K(c) - rho_target(c))^2

  reverse, per step (lam_x, lam_v are dL/dx', dL/dv' on entry):
      lam_v  += c_d lam_x
      lam_a   = c_k lam_v
      lam_A   = sum_p lam_a_p W(x_p - c)                 (interpolation^T)
      lam_x  += sum_c (lam_a_p . a(c)) grad_x W(x_p - c)  (interpolation, position)
      lam_rho = A^T lam_A                                  (A^T: kernel conj(i k g))
      lam_x  += m_p sum_c lam_rho(c) grad_x W(x_p - c)    (deposit, position)

W is the CIC weight prod_d (1 - |x_d - c_d|); d/dx_d of the lower corner's
factor is -1 and of the upper corner's +1 (one-sided at cell faces, where
CIC has a kink).  Pins: tests/test_oracle_adjoint.py (transposition
identities, central finite differences).
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence

import numpy as np

from . import mesh, solve
from .fft import fft3


def cic_grad_gather(field, x, n: int) -> np.ndarray:
    """sum_c field(c) grad_x W(x - c) for a scalar mesh field (periodic)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    w = (1.0 - f, f)
    dw = (-np.ones_like(f), np.ones_like(f))
    out = np.zeros_like(x)
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        val = field[(i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n]
        out[:, 0] += val * dw[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        out[:, 1] += val * w[dx][:, 0] * dw[dy][:, 1] * w[dz][:, 2]
        out[:, 2] += val * w[dx][:, 0] * w[dy][:, 1] * dw[dz][:, 2]
    return out


def cic_deposit_vector(lam, x, n: int) -> np.ndarray:
    """Transpose of interpolation: sum_p lam_p W(x_p - c), per component [3, n, n, n]."""
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    return np.stack([mesh.cic_deposit(x, lam[:, d], n) for d in range(3)])


def interp_grad(field3, lam, x, n: int) -> np.ndarray:
    """sum_c (lam_p . field(c)) grad_x W(x_p - c) for a vector field [3, n, n, n]."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    w = (1.0 - f, f)
    dw = (-np.ones_like(f), np.ones_like(f))
    out = np.zeros_like(x)
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        idx = ((i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n)
        val = sum(lam[:, d] * field3[d][idx] for d in range(3))
        out[:, 0] += val * dw[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        out[:, 1] += val * w[dx][:, 0] * dw[dy][:, 1] * w[dz][:, 2]
        out[:, 2] += val * w[dx][:, 0] * w[dy][:, 1] * dw[dz][:, 2]
    return out


def accel_periodic_adjoint(lam_a, h: float, G: float, r_s: float = 0.0) -> np.ndarray:
    """A^T for the map rho -> a of solve.accel_periodic: multiplies each
    component's spectrum by the conjugate kernel -i k_d g(k) and sums."""
    n = lam_a.shape[1]
    V = (n * h) ** 3
    m = solve.mode_numbers(n)
    k1 = 2.0 * np.pi * m / (n * h)
    kgrad = np.where(np.abs(m) == n // 2, 0.0, k1)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    g = np.zeros_like(k2)
    nz = k2 > 0
    g[nz] = 4.0 * np.pi * G / (k2[nz] * V)
    if r_s > 0:
        g *= np.exp(-k2 * r_s * r_s)
    gz, gy, gx = np.meshgrid(kgrad, kgrad, kgrad, indexing="ij")
    acc = np.zeros(lam_a.shape[1:], dtype=np.complex128)
    for d, kd in enumerate((gx, gy, gz)):
        acc += -1j * kd * g * fft3(lam_a[d])
    return fft3(acc, inverse=True).real


def forward(xs: Sequence[np.ndarray], vs: Sequence[np.ndarray], cfg: Dict, c_kick: float, c_drift: float,
            steps: int):
    """Single-mesh forward steps in float64; returns the list of states."""
    n = cfg["n_fine"]
    states = [([np.asarray(x, np.float64).copy() for x in xs], [np.asarray(v, np.float64).copy() for v in vs])]
    for _ in range(steps):
        x, v = states[-1]
        rho = sum(mesh.cic_deposit(xi, m, n) for xi, m in zip(x, cfg["mass"]))
        a_mesh = solve.accel_periodic(rho, 1.0, cfg["G"])
        nx, nv = [], []
        for xi, vi in zip(x, v):
            a = mesh.cic_interp(a_mesh, xi, n)
            v1 = vi + c_kick * a
            nx.append(np.mod(xi + c_drift * v1, n))
            nv.append(v1)
        states.append((nx, nv))
    return states


def density(x: Sequence[np.ndarray], cfg: Dict) -> np.ndarray:
    n = cfg["n_fine"]
    return sum(mesh.cic_deposit(xi, m, n) for xi, m in zip(x, cfg["mass"]))


def loss(x_final, cfg, target) -> float:
    return float(np.sum((density(x_final, cfg) - target) ** 2))


def gradient(xs, vs, cfg: Dict, c_kick: float, c_drift: float, steps: int, target):
    """dL/dx0, dL/dv0 per species for L = sum (rho_final - target)^2."""
    n = cfg["n_fine"]
    states = forward(xs, vs, cfg, c_kick, c_drift, steps)
    xK = states[-1][0]
    g_rho = 2.0 * (density(xK, cfg) - target)
    lam_x: List[np.ndarray] = [m * cic_grad_gather(g_rho, xi, n) for xi, m in zip(xK, cfg["mass"])]
    lam_v: List[np.ndarray] = [np.zeros_like(xi) for xi in xK]
    for k in range(steps - 1, -1, -1):
        lam_x, lam_v = reverse_step(states[k][0], cfg, lam_x, lam_v, c_kick, c_drift)
    return lam_x, lam_v


def reverse_step(x, cfg: Dict, lam_x, lam_v, c_kick: float, c_drift: float):
    """Map (dL/dx', dL/dv') after one step to (dL/dx, dL/dv) before it, given
    the pre-step positions x of every species."""
    n = cfg["n_fine"]
    a_mesh = solve.accel_periodic(density(x, cfg), 1.0, cfg["G"])
    lam_x = [np.asarray(a, np.float64).copy() for a in lam_x]
    lam_v = [np.asarray(a, np.float64).copy() for a in lam_v]
    lam_A = np.zeros((3, n, n, n))
    for s in range(len(x)):
        lam_v[s] = lam_v[s] + c_drift * lam_x[s]
        lam_a = c_kick * lam_v[s]
        lam_A += cic_deposit_vector(lam_a, x[s], n)
        lam_x[s] = lam_x[s] + interp_grad(a_mesh, lam_a, x[s], n)
    lam_rho = accel_periodic_adjoint(lam_A, 1.0, cfg["G"])
    for s in range(len(x)):
        lam_x[s] = lam_x[s] + cfg["mass"][s] * cic_grad_gather(lam_rho, x[s], n)
    return lam_x, lam_v
