"""Oracle PM force step: deposit -> solve -> interpolate -> kick-drift -> recompress.

Follows the per-step flow of Sec. 2.1-2.3 (Fig. 2: link list, density
interpolation, Fourier transforms, inverse force interpolation; PP is not
part of this step) with the two-level split of Sec. 2.1:

  * single level (coarse_ratio == 1): one periodic fine mesh, full Green's
    function of Eq. 2, acceleration interpolated from it;
  * two level: long-range acceleration on the coarse mesh (n_fine /
    coarse_ratio per side, Gaussian long-range Green's function) plus the
    short-range acceleration of the particle's home tile; each tile of
    interior t carries a buffer b (edge T = t + 2b), receives the particles
    whose CIC stencil lies inside it, and is solved by its own FFT
    convolution with the truncated short-range kernel (radius R <= b - 2).

Kick-drift (the paper does not spell it out): v' = v + c_kick a, then
x' = (x + c_drift v') wrapped into [0, n_fine).

Config keys: n_fine, coarse_ratio, tile, buffer, cmp_ratio, vel_bits, G,
mass (per species), r_split, r_cut.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from . import codec, mesh, pp, solve


def tile_origins(n_fine: int, t: int):
    nt = n_fine // t
    for iz in range(nt):
        for iy in range(nt):
            for ix in range(nt):
                yield (ix, iy, iz), np.array([ix * t, iy * t, iz * t], dtype=np.float64)


def density_fine(xs: Sequence[np.ndarray], cfg: Dict) -> np.ndarray:
    """Periodic CIC mass per fine cell, both species."""
    n = cfg["n_fine"]
    return sum(mesh.cic_deposit(x, m, n) for x, m in zip(xs, cfg["mass"]))


def density_coarse(xs: Sequence[np.ndarray], cfg: Dict) -> np.ndarray:
    """Periodic CIC mass per coarse cell (positions divided by coarse_ratio)."""
    rc = cfg["coarse_ratio"]
    nc = cfg["n_fine"] // rc
    return sum(mesh.cic_deposit(np.asarray(x, np.float64) / rc, m, nc) for x, m in zip(xs, cfg["mass"]))


def accel_single_level(xs: Sequence[np.ndarray], cfg: Dict) -> List[np.ndarray]:
    n = cfg["n_fine"]
    a_mesh = solve.accel_periodic(density_fine(xs, cfg), 1.0, cfg["G"])
    return [mesh.cic_interp(a_mesh, x, n) for x in xs]


def coarse_accel_mesh(xs, cfg) -> np.ndarray:
    rc = cfg["coarse_ratio"]
    return solve.accel_periodic(density_coarse(xs, cfg), float(rc), cfg["G"], cfg["r_split"])


def fine_accel(xs: Sequence[np.ndarray], cfg: Dict) -> List[np.ndarray]:
    """Short-range acceleration of every particle from its home tile."""
    n, t, b = cfg["n_fine"], cfg["tile"], cfg["buffer"]
    T = t + 2 * b
    if cfg["r_cut"] > b - 2:
        raise ValueError("kernel radius must satisfy R <= buffer - 2")
    K = solve.fine_kernel(T, cfg["G"], cfg["r_split"], cfg["r_cut"])
    xs64 = [np.asarray(x, np.float64).reshape(-1, 3) for x in xs]
    home = [np.floor(x / t).astype(np.int64) for x in xs64]
    out = [np.zeros_like(x) for x in xs64]
    for idx, o in tile_origins(n, t):
        origin = o - b
        rho = sum(mesh.tile_deposit(x, m, origin, T, n) for x, m in zip(xs64, cfg["mass"]))
        a_t = solve.accel_tile(rho, K)
        for s, x in enumerate(xs64):
            sel = np.all(home[s] == np.array(idx), axis=1)
            if np.any(sel):
                u = np.mod(x[sel] - origin, n)
                out[s][sel] = mesh.tile_interp(a_t, u)
    return out


def fine_accel_mesh(xs: Sequence[np.ndarray], cfg: Dict) -> np.ndarray:
    """[3, n, n, n] short-range acceleration assembled from the interiors of
    all tiles (each tile solved as in fine_accel): the fine force values the
    particles' home-tile interpolations draw on."""
    n, t, b = cfg["n_fine"], cfg["tile"], cfg["buffer"]
    T = t + 2 * b
    K = solve.fine_kernel(T, cfg["G"], cfg["r_split"], cfg["r_cut"])
    xs64 = [np.asarray(x, np.float64).reshape(-1, 3) for x in xs]
    out = np.zeros((3, n, n, n))
    for _, o in tile_origins(n, t):
        rho = sum(mesh.tile_deposit(x, m, o - b, T, n) for x, m in zip(xs64, cfg["mass"]))
        a_t = solve.accel_tile(rho, K)
        x0, y0, z0 = (int(c) for c in o)
        out[:, z0:z0 + t, y0:y0 + t, x0:x0 + t] = a_t[:, b:b + t, b:b + t, b:b + t]
    return out


def force_meshes(xs: Sequence[np.ndarray], cfg: Dict) -> List[np.ndarray]:
    """The force meshes a step interpolates from: the periodic mesh (single
    level), or the coarse long-range mesh and the assembled fine mesh."""
    if cfg["coarse_ratio"] == 1:
        return [solve.accel_periodic(density_fine(xs, cfg), 1.0, cfg["G"])]
    return [coarse_accel_mesh(xs, cfg), fine_accel_mesh(xs, cfg)]


def vmax_bound(vmax_in: float, meshes: Sequence[np.ndarray], c_kick: float) -> np.float32:
    """Velocity scale of the bound mode (an option, not the paper's Sec. 2.4
    definition, which is the exact max): a decoded velocity component lies
    below v_max and a CIC-interpolated acceleration component never exceeds
    the largest mesh value of each mesh it sums, so

        |v'_d| <= v_max + |c_kick| * sum_meshes max |a|.

    Returned as the smallest float32 not below that value."""
    b = float(vmax_in) + abs(float(c_kick)) * sum(float(np.max(np.abs(m))) for m in meshes)
    f = np.float32(b)
    if float(f) < b:
        f = np.nextafter(f, np.float32(np.inf))
    return f


def accel(xs: Sequence[np.ndarray], cfg: Dict) -> List[np.ndarray]:
    """Per-particle acceleration of each species (fine-cell units)."""
    if cfg["coarse_ratio"] == 1:
        return accel_single_level(xs, cfg)
    rc = cfg["coarse_ratio"]
    nc = cfg["n_fine"] // rc
    a_c = coarse_accel_mesh(xs, cfg)
    coarse = [mesh.cic_interp(a_c, np.asarray(x, np.float64) / rc, nc) for x in xs]
    fine = fine_accel(xs, cfg)
    return [c + f for c, f in zip(coarse, fine)]


def kick_drift(x, v, a, c_kick: float, c_drift: float, n_fine: int):
    v1 = np.asarray(v, np.float64) + c_kick * np.asarray(a, np.float64)
    x1 = np.mod(np.asarray(x, np.float64) + c_drift * v1, float(n_fine))
    return x1, v1


def to_f32_positions(x, n_fine: int) -> np.ndarray:
    """float32 cast of wrapped positions, keeping them inside [0, n_fine)."""
    x32 = np.asarray(x, np.float64).astype(np.float32)
    x32[x32 >= np.float32(n_fine)] = np.float32(0.0)
    return x32


def step(codes: Sequence[codec.Codes], cfg: Dict, c_kick: float, c_drift: float,
         order: str = "stable", vmax_mode: int = 0):
    """One full PM step from compressed state to compressed state.

    vmax_mode 0 quantises the new velocities with their exact max (Sec. 2.4);
    1 with vmax_bound of each species' input v_max and the force meshes.
    cfg["pp"] = 1 adds the particle-particle acceleration of Eq. 4 (oracle/pp.py,
    softening cfg["r_soft"]) to the PM acceleration before the kick; the bound
    then also covers its largest component.
    Returns (new codes per species, float64 x', v' per species in input order).
    """
    n = cfg["n_fine"]
    n_cmp = n // cfg["cmp_ratio"]
    xv = [codec.decompress(c, n) for c in codes]
    xs = [p[0] for p in xv]
    a = accel(xs, cfg)
    extra = []
    if cfg.get("pp", 0):
        a_pp = pp.pp_accel(xs, cfg["mass"], cfg["G"], cfg["r_soft"])
        a = [ai + pi for ai, pi in zip(a, a_pp)]
        extra = [np.concatenate(a_pp)]
    vm = [None, None]
    if vmax_mode == 1:
        meshes = force_meshes(xs, cfg) + extra
        vm = [vmax_bound(c.vmax, meshes, c_kick) for c in codes]
    new_codes, states = [], []
    for (x, v), acc, vmax in zip(xv, a, vm):
        x1, v1 = kick_drift(x, v, acc, c_kick, c_drift, n)
        new_codes.append(codec.compress(to_f32_positions(x1, n), v1.astype(np.float32), n, n_cmp,
                                        cfg["vel_bits"], vmax=vmax, order=order))
        states.append((x1, v1))
    return new_codes, states
