"""Seeded generators of synthetic CDM + neutrino particle sets.

The shapes follow the two-species workloads of the paper (Sec. 2.1, footnote
on the particle counts: N_nu = 8 N_cdm, both species on one mesh; Sec. 3.1
and 3.2: clustered CDM with near-uniform, thermally hot neutrinos).  Real
cosmological initial conditions need transfer functions that are not
available here, so these recipes stand in for them:

* CDM on a lattice displaced by Gaussian noise, by Zel'dovich displacements of
  a Gaussian field with P(k) ~ k^-2, or drawn from a lognormal density field;
* neutrinos at uniform random positions with isotropic velocities whose
  speeds follow a relativistic Fermi-Dirac shape, p(u) ~ u^2 / (e^u + 1).

Positions are float32 in fine-mesh cell units on [0, n_fine); velocities are
float32 in fine cells per unit time.  Nothing here implements the PM method.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

FOUR_PI_G_ONE = 1.0 / (4.0 * np.pi)  # G such that 4 pi G = 1


def _wrap_f32(x: np.ndarray, n: int) -> np.ndarray:
    """Wrap float64 positions into [0, n) and cast to float32 (never == n)."""
    x = np.mod(x, float(n))
    x32 = x.astype(np.float32)
    x32[x32 >= np.float32(n)] = np.float32(0.0)
    x32[x32 < 0] = np.float32(0.0)
    return x32


def fermi_dirac_speeds(rng: np.random.Generator, n: int, scale: float) -> np.ndarray:
    """Speeds |v| = scale * u with u drawn from p(u) ~ u^2 / (e^u + 1).

    Inverse-CDF sampling from a float64 table on u in [0, 40].
    """
    u = np.linspace(0.0, 40.0, 8193)
    pdf = u * u / (np.exp(u) + 1.0)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return scale * np.interp(rng.random(n), cdf, u)


def isotropic_velocities(rng: np.random.Generator, speeds: np.ndarray) -> np.ndarray:
    d = rng.standard_normal((speeds.shape[0], 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (d * speeds[:, None]).astype(np.float32)


def uniform_positions(rng: np.random.Generator, n: int, n_fine: int) -> np.ndarray:
    return _wrap_f32(rng.random((n, 3)) * n_fine, n_fine)


def lattice_positions(rng: np.random.Generator, n_side: int, n_fine: int, sigma: float) -> np.ndarray:
    """Cubic lattice of n_side^3 points (spacing n_fine/n_side, offset half a
    spacing) displaced by isotropic Gaussian noise of width sigma cells."""
    sp = n_fine / n_side
    g = (np.arange(n_side) + 0.5) * sp
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return _wrap_f32(q + sigma * rng.standard_normal(q.shape), n_fine)


def _gaussian_field(rng: np.random.Generator, n: int, slope: float, smooth: float = 0.0) -> np.ndarray:
    """Real Gaussian random field on n^3 with P(k) ~ k^slope (k=0 removed),
    optionally multiplied by exp(-k^2 smooth^2 / 2) (smooth in grid cells)."""
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kz = np.fft.fftfreq(n) * 2 * np.pi
    kx = np.fft.rfftfreq(n) * 2 * np.pi
    k2 = kz[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0) * np.exp(-0.5 * k2[nz] * smooth * smooth)
    return np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))


def zeldovich_lattice(rng: np.random.Generator, n_side: int, n_fine: int, rms_disp: float = 0.5,
                      vel_factor: float = 0.1, slope: float = -2.0) -> Tuple[np.ndarray, np.ndarray]:
    """Lattice + Zel'dovich displacement psi with div(psi) = -delta, where delta
    is Gaussian with P(k) ~ k^slope.  psi is scaled so rms|psi| = rms_disp fine
    cells; velocities are vel_factor * psi."""
    delta = _gaussian_field(rng, n_side, slope)
    dk = np.fft.rfftn(delta)
    kz = np.fft.fftfreq(n_side) * 2 * np.pi
    kx = np.fft.rfftfreq(n_side) * 2 * np.pi
    KZ, KY, KX = np.meshgrid(kz, kz, kx, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    psi = np.stack([np.fft.irfftn(1j * kd * dk / k2, s=(n_side,) * 3, axes=(0, 1, 2)) for kd in (KX, KY, KZ)],
                    axis=-1)
    psi = psi.reshape(-1, 3)
    psi *= rms_disp / np.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    sp = n_fine / n_side
    g = (np.arange(n_side) + 0.5) * sp
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return _wrap_f32(q + psi, n_fine), (vel_factor * psi).astype(np.float32)


def lognormal_positions(rng: np.random.Generator, n: int, n_fine: int, grid: int, sigma_ln: float = 1.5,
                        slope: float = -2.0, smooth: float = 1.0) -> np.ndarray:
    """n points drawn from the lognormal density exp(sigma g - sigma^2/2) of a
    unit-variance Gaussian field g (P ~ k^slope, smoothed) on a grid^3 mesh,
    uniform within each grid cell."""
    g = _gaussian_field(rng, grid, slope, smooth)
    g = (g - g.mean()) / g.std()
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2).ravel()
    cdf = np.cumsum(rho)
    cdf /= cdf[-1]
    cell = np.minimum(np.searchsorted(cdf, rng.random(n), side="right"), grid ** 3 - 1)
    ix, iy, iz = cell % grid, (cell // grid) % grid, cell // (grid * grid)
    sp = n_fine / grid
    q = np.stack([ix, iy, iz], axis=1) + rng.random((n, 3))
    return _wrap_f32(q * sp, n_fine)


@dataclasses.dataclass
class Workload:
    """Parameters of one synthetic workload plus its particle arrays.

    mesh: n_fine, coarse_ratio (1 = single periodic mesh), tile interior,
    buffer, cmp_ratio (fine cells per compression cell), vel_bits;
    physics: G, per-species masses, r_split / r_cut of the two-level split.
    """
    name: str
    n_fine: int
    coarse_ratio: int
    tile: int
    buffer: int
    cmp_ratio: int
    vel_bits: int
    G: float
    mass: Tuple[float, float]
    r_split: float
    r_cut: float
    x: List[np.ndarray]
    v: List[np.ndarray]
    seed: int
    notes: Dict[str, float] = dataclasses.field(default_factory=dict)

    @property
    def counts(self) -> Tuple[int, int]:
        return (int(self.x[0].shape[0]), int(self.x[1].shape[0]))

    def config(self) -> Dict[str, float]:
        return dict(n_fine=self.n_fine, coarse_ratio=self.coarse_ratio, tile=self.tile,
                    buffer=self.buffer, cmp_ratio=self.cmp_ratio, vel_bits=self.vel_bits,
                    G=self.G, mass=self.mass, count=self.counts, r_split=self.r_split,
                    r_cut=self.r_cut)


# name -> (n_fine, coarse_ratio, tile, buffer, cdm recipe, n_cdm_side, n_nu_side, vel_bits, r_cut, seed)
WORKLOADS = {
    # 64^3 periodic single mesh; 16^3 CDM lattice + noise 0.5, m=8; 32^3 nu, m_nu/m_cdm = 0.005.
    "single64": dict(n_fine=64, coarse_ratio=1, tile=64, buffer=0, cdm="lattice", n_cdm=16, n_nu=32,
                     vel_bits=16, r_cut=0.0, seed=1612),
    # 256^3 fine mesh, coarse ratio 4, 64 tiles of 64^3 + 16-cell buffer; 128^3 Zel'dovich CDM + 256^3 nu.
    "two_level256": dict(n_fine=256, coarse_ratio=4, tile=64, buffer=16, cdm="zeldovich", n_cdm=128,
                         n_nu=256, vel_bits=8, r_cut=14.0, seed=1613),
    # 512^3 fine mesh, 512 tiles of 64^3 + 16; 256^3 lognormal CDM + 512^3 nu.
    "batched512": dict(n_fine=512, coarse_ratio=4, tile=64, buffer=16, cdm="lognormal", n_cdm=256,
                       n_nu=512, vel_bits=16, r_cut=14.0, seed=1614),
    # 128^3 single mesh; 64^3 Zel'dovich CDM + 128^3 nu (differentiable runs).
    "diff128": dict(n_fine=128, coarse_ratio=1, tile=128, buffer=0, cdm="zeldovich", n_cdm=64, n_nu=128,
                    vel_bits=16, r_cut=0.0, seed=1615),
    # 768^3 fine mesh (192^3 coarse: the row / column coarse transforms), 1728 tiles; 96^3 + 192^3.
    "two_level768": dict(n_fine=768, coarse_ratio=4, tile=64, buffer=16, cdm="zeldovich", n_cdm=96,
                         n_nu=192, vel_bits=16, r_cut=14.0, seed=1618),
    # The clustered, batched recipe at a size the oracle finishes in seconds: 64^3 fine mesh, 64 tiles of
    # 16^3 + 8; 32^3 lognormal CDM (per-tile counts 24 .. 2024) + 64^3 nu, 16-bit velocities.
    "clustered64": dict(n_fine=64, coarse_ratio=4, tile=16, buffer=8, cdm="lognormal", n_cdm=32, n_nu=64,
                        vel_bits=16, r_cut=6.0, seed=1620),
    # Small two-level cases that the oracle finishes in seconds.
    "two_level64": dict(n_fine=64, coarse_ratio=4, tile=16, buffer=8, cdm="zeldovich", n_cdm=16, n_nu=32,
                        vel_bits=16, r_cut=6.0, seed=1616),
    "two_level128_t96": dict(n_fine=128, coarse_ratio=4, tile=64, buffer=16, cdm="zeldovich", n_cdm=32,
                             n_nu=64, vel_bits=8, r_cut=14.0, seed=1617),
}


def make_workload(name: str, n_cdm: Optional[int] = None, n_nu: Optional[int] = None,
                  seed: Optional[int] = None, fd_scale: float = 2.0) -> Workload:
    """Build a named workload; n_cdm / n_nu override the per-side particle counts."""
    p = dict(WORKLOADS[name])
    if n_cdm is not None:
        p["n_cdm"] = n_cdm
    if n_nu is not None:
        p["n_nu"] = n_nu
    s = p["seed"] if seed is None else seed
    rng = np.random.default_rng(s)
    nf = p["n_fine"]
    notes: Dict[str, float] = {}
    if p["cdm"] == "lattice":
        xc = lattice_positions(rng, p["n_cdm"], nf, 0.5)
        vc = np.zeros_like(xc)
    elif p["cdm"] == "zeldovich":
        xc, vc = zeldovich_lattice(rng, p["n_cdm"], nf)
    elif p["cdm"] == "lognormal":
        grid = max(8, nf // 4)
        xc = lognormal_positions(rng, p["n_cdm"] ** 3, nf, grid, 1.5, -2.0, smooth=1.0)
        vc = (0.05 * rng.standard_normal(xc.shape)).astype(np.float32)
        t = p["tile"]
        tiles = (xc // t).astype(np.int64)
        nt = nf // t
        cnt = np.bincount(tiles[:, 0] + nt * (tiles[:, 1] + nt * tiles[:, 2]), minlength=nt ** 3)
        notes["tile_count_max"] = float(cnt.max())
        notes["tile_count_min"] = float(cnt.min())
    else:
        raise ValueError(p["cdm"])
    n_nu_total = p["n_nu"] ** 3
    xn = uniform_positions(rng, n_nu_total, nf)
    vn = isotropic_velocities(rng, fermi_dirac_speeds(rng, n_nu_total, fd_scale))
    two_level = p["coarse_ratio"] > 1
    r_cut = p["r_cut"]
    return Workload(name=name, n_fine=nf, coarse_ratio=p["coarse_ratio"], tile=p["tile"],
                    buffer=p["buffer"], cmp_ratio=4, vel_bits=p["vel_bits"], G=FOUR_PI_G_ONE,
                    mass=(8.0, 0.04), r_split=(r_cut / 4.5 if two_level else 0.0), r_cut=r_cut,
                    x=[xc, xn], v=[vc, vn], seed=s, notes=notes)
