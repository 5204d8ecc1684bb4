"""Oracle cloud-in-cell (CIC) mass assignment and force interpolation.

The paper's density step is a CIC interpolation of the particles onto the
mesh (Sec. 2.3, the density_interpolation stage of Fig. 2) and the force
step its inverse (inverse_force_interpolation); CDM and neutrinos with their
own masses go to the same mesh (Sec. 2.1, footnote).  Readings where the
paper is silent:

  * mesh points sit at integer coordinates; CIC weight W(u) = max(0, 1-|u|),
    so a particle at x touches floor(x) and floor(x)+1 in each dimension;
  * mesh arrays are indexed [z, y, x] (x fastest in memory);
  * a buffered tile of edge T whose first cell is at ``origin`` receives a
    particle iff both stencil cells lie inside [0, T) in every dimension,
    with tile coordinates u = (x - origin) mod n_fine;
  * the int64 fixed-point deposit (added for bit-reproducibility; the paper
    has none) gives each species the integer mass M = llrint(m 2^32) and
    splits it exactly and conservatively, one dimension at a time (x, y, z):
        a1 = floor(f 2^20) with f = x - floor(x) from the float32 position,
        hi = (M a1 + 2^19) >> 20, lo = M - hi,
    so every particle deposits exactly M in total.

Pins: tests/test_oracle_mesh.py (mass conservation, brute-force corner
weights, periodic wrap, tile inclusion rule, fixed-point exactness).
"""
from __future__ import annotations

import itertools

import numpy as np

FIXED_MASS_BITS = 32
FIXED_WEIGHT_BITS = 20


def _corners():
    return itertools.product((0, 1), repeat=3)  # (dz, dy, dx)


def cic_deposit(x, m, n: int) -> np.ndarray:
    """Periodic CIC deposit on an n^3 mesh; x in mesh units, m scalar or per particle."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), (x.shape[0],))
    rho = np.zeros((n, n, n), dtype=np.float64)
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    w = (1.0 - f, f)
    for dz, dy, dx in _corners():
        wt = w[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        np.add.at(rho, ((i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n), m * wt)
    return rho


def cic_interp(field, x, n: int) -> np.ndarray:
    """Periodic CIC gather of a vector field [3, n, n, n] at positions x (mesh units)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    w = (1.0 - f, f)
    out = np.zeros((x.shape[0], 3), dtype=np.float64)
    for dz, dy, dx in _corners():
        wt = w[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        iz, iy, ix = (i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n
        for d in range(3):
            out[:, d] += wt * field[d][iz, iy, ix]
    return out


def tile_deposit(x, m, origin, T: int, n_fine: int) -> np.ndarray:
    """CIC deposit onto one buffered tile of edge T whose cell 0 is at ``origin``
    (fine units, periodic); particles whose stencil leaves the tile are skipped."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), (x.shape[0],))
    u = np.mod(x - np.asarray(origin, dtype=np.float64), n_fine)
    i0 = np.floor(u).astype(np.int64)
    keep = np.all((i0 >= 0) & (i0 <= T - 2), axis=1)
    u, i0, m = u[keep], i0[keep], m[keep]
    f = u - i0
    w = (1.0 - f, f)
    rho = np.zeros((T, T, T), dtype=np.float64)
    for dz, dy, dx in _corners():
        wt = w[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        np.add.at(rho, (i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx), m * wt)
    return rho


def tile_interp(field, u) -> np.ndarray:
    """CIC gather from a tile's vector field [3, T, T, T] at tile coordinates u
    (the stencil must lie inside the tile)."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    w = (1.0 - f, f)
    out = np.zeros((u.shape[0], 3), dtype=np.float64)
    for dz, dy, dx in _corners():
        wt = w[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]
        for d in range(3):
            out[:, d] += wt * field[d][i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx]
    return out


def fixed_mass(m: float) -> int:
    """Integer mass in units of 2^-32 (round to nearest, ties to even)."""
    return int(np.rint(np.float64(m) * 2.0 ** FIXED_MASS_BITS))


def _split(M: np.ndarray, a1: np.ndarray):
    hi = (M * a1 + (1 << (FIXED_WEIGHT_BITS - 1))) >> FIXED_WEIGHT_BITS
    return M - hi, hi


def cic_deposit_fixed(x_f32, M: int, n: int) -> np.ndarray:
    """Periodic int64 fixed-point CIC deposit of float32 positions (mesh units)."""
    x = np.asarray(x_f32, dtype=np.float32).reshape(-1, 3)
    fl = np.floor(x)
    f = (x - fl).astype(np.float32)                      # exact in float32
    a1 = np.floor(f.astype(np.float64) * 2.0 ** FIXED_WEIGHT_BITS).astype(np.int64)
    i0 = fl.astype(np.int64)
    Mv = np.full(x.shape[0], M, dtype=np.int64)
    rho = np.zeros((n, n, n), dtype=np.int64)
    mx = _split(Mv, a1[:, 0])
    for dx in (0, 1):
        my = _split(mx[dx], a1[:, 1])
        for dy in (0, 1):
            mz = _split(my[dy], a1[:, 2])
            for dz in (0, 1):
                np.add.at(rho, ((i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n), mz[dz])
    return rho


def _coarse_weights(rc: int) -> np.ndarray:
    """w(k) = 1 - |k| / rc for k = -(rc-1) .. rc-1: the coarse CIC tent sampled on fine nodes."""
    k = np.arange(-(rc - 1), rc)
    return 1.0 - np.abs(k) / rc


def restrict(rho_f: np.ndarray, rc: int) -> np.ndarray:
    """Coarse CIC density from the fine one.  A coarse tent Lambda(u / rc) is
    piecewise linear with knots on fine nodes, so it equals the fine-node
    interpolation sum_k w(k) Lambda(u - k); hence the coarse CIC deposit of
    any particles is rho_c(C) = sum_k w(kx) w(ky) w(kz) rho_f(rc C + k)
    (periodic).  Written as the plain triple sum."""
    n = rho_f.shape[0]
    nc = n // rc
    w = _coarse_weights(rc)
    ks = np.arange(-(rc - 1), rc)
    out = np.zeros((nc, nc, nc))
    for iz, kz in enumerate(ks):
        for iy, ky in enumerate(ks):
            for ix, kx in enumerate(ks):
                zz = (rc * np.arange(nc) + kz) % n
                yy = (rc * np.arange(nc) + ky) % n
                xx = (rc * np.arange(nc) + kx) % n
                out += w[iz] * w[iy] * w[ix] * rho_f[np.ix_(zz, yy, xx)]
    return out


def prolong(field_c: np.ndarray, rc: int) -> np.ndarray:
    """Coarse field [.., nc, nc, nc] trilinearly interpolated onto the fine nodes
    (the transpose of restrict).  By the same identity the fine CIC
    interpolation of it at x equals the coarse CIC interpolation at x / rc."""
    nc = field_c.shape[-1]
    n = nc * rc
    j = np.arange(n)
    c0, f = j // rc, (j % rc) / rc
    c1 = (c0 + 1) % nc
    out = 0.0
    for wz, cz in ((1 - f, c0), (f, c1)):
        for wy, cy in ((1 - f, c0), (f, c1)):
            for wx, cx in ((1 - f, c0), (f, c1)):
                out = out + (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]) * \
                    field_c[..., cz[:, None, None], cy[None, :, None], cx[None, None, :]]
    return out
