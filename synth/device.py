"""Seeded device-side generators for particle sets too large for host arrays:
the 1536^3 two-level set (768^3 CDM + 1536^3 neutrinos, about 4.1e9
particles).  The recipes are those of generators.py, drawn with torch on the
GPU (so the numbers differ from the numpy sets of the same name):

* CDM: cubic lattice + Zel'dovich displacement psi (div psi = -delta, delta
  Gaussian with P(k) ~ k^-2), scaled to rms |psi| = 0.5 fine cells,
  velocities 0.1 psi;
* neutrinos: uniform positions, isotropic velocities with Fermi-Dirac speeds
  |v| = scale u, p(u) ~ u^2 / (e^u + 1), produced one z slab at a time (the
  slab's share of the uniform set, drawn within the slab) so that a caller
  can turn each slab into codes and keep only those.

Positions are float32 in fine cells on [0, n_fine), clamped below the slab
and box edges; nothing here implements the PM method.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np
import torch


def _below(v: float) -> float:
    """The largest float32 strictly below v."""
    return float(np.nextafter(np.float32(v), np.float32(-np.inf)))


def zeldovich_lattice(seed: int, n_side: int, n_fine: int, rms_disp: float = 0.5, vel_factor: float = 0.1,
                      slope: float = -2.0, device: str = "cuda") -> Tuple[torch.Tensor, torch.Tensor]:
    """Lattice + Zel'dovich displacements on the device: x, v float32 [n_side^3, 3]
    (x fastest in the lattice order)."""
    g = torch.Generator(device=device).manual_seed(seed)
    n = n_side
    w = torch.randn((n, n, n), generator=g, device=device)
    dk = torch.fft.rfftn(w)
    del w
    kz = torch.fft.fftfreq(n, device=device) * 2 * np.pi
    kx = torch.fft.rfftfreq(n, device=device) * 2 * np.pi
    k2 = kz[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (slope / 4.0), torch.zeros_like(k2))
    dk *= amp
    del amp
    k2[0, 0, 0] = 1.0
    dk /= k2
    del k2
    psi = torch.empty((n ** 3, 3), dtype=torch.float32, device=device)
    ks = (kx[None, None, :], kz[None, :, None], kz[:, None, None])
    for d in range(3):
        psi[:, d] = torch.fft.irfftn(1j * ks[d] * dk, s=(n, n, n)).reshape(-1)
    del dk
    rms = torch.sqrt(torch.mean(torch.sum(psi.double() ** 2, dim=1)))
    psi *= float(rms_disp / rms)
    sp = n_fine / n
    q = (torch.arange(n, device=device, dtype=torch.float32) + 0.5) * sp
    x = psi.clone()
    x[:, 0] += q.repeat(n * n)
    x[:, 1] += q.repeat_interleave(n).repeat(n)
    x[:, 2] += q.repeat_interleave(n * n)
    x = torch.remainder(x, float(n_fine)).clamp_(0.0, _below(n_fine))
    v = psi.mul_(vel_factor)
    return x, v


def _fd_table(device: str):
    u = np.linspace(0.0, 40.0, 8193)
    pdf = u * u / (np.exp(u) + 1.0)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return torch.from_numpy(cdf).to(device), torch.from_numpy(u).to(device)


def neutrino_slab(seed: int, slab: int, n_slabs: int, n_per_slab: int, n_fine: int, fd_scale: float = 2.0,
                  velocities_only: bool = False, device: str = "cuda"):
    """Slab `slab` of n_slabs equal z slabs: n_per_slab uniform positions with
    z in the slab, and Fermi-Dirac isotropic velocities.  Returns (x, v), or v
    alone when velocities_only (same numbers as the full call)."""
    g = torch.Generator(device=device).manual_seed(seed * 1000003 + slab)
    r = torch.rand((n_per_slab, 3), generator=g, device=device, dtype=torch.float64)
    uu = torch.rand(n_per_slab, generator=g, device=device, dtype=torch.float64)
    d = torch.randn((n_per_slab, 3), generator=g, device=device)
    cdf, u = _fd_table(device)
    i = torch.searchsorted(cdf, uu).clamp_(1, cdf.numel() - 1)
    t = (uu - cdf[i - 1]) / (cdf[i] - cdf[i - 1])
    speed = (fd_scale * (u[i - 1] + t * (u[i] - u[i - 1]))).float()
    v = d / torch.linalg.norm(d, dim=1, keepdim=True) * speed[:, None]
    if velocities_only:
        return v
    h = n_fine / n_slabs
    z0 = slab * h
    x = torch.empty((n_per_slab, 3), dtype=torch.float32, device=device)
    x[:, 0] = (r[:, 0] * n_fine).float().clamp_(0.0, _below(n_fine))
    x[:, 1] = (r[:, 1] * n_fine).float().clamp_(0.0, _below(n_fine))
    x[:, 2] = (z0 + r[:, 2] * h).float().clamp_(float(z0), _below(z0 + h))
    return x, v
