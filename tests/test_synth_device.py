"""The device-side generators of the largest workload, run here on the CPU at
small sizes: value ranges, the slab bounds the slab-by-slab assembly relies
on, reproducibility of the velocity-only call, the Zel'dovich displacement
normalisation and the Fermi-Dirac mean speed (closed form)."""
import math

import numpy as np
import torch

from synth import device as dev


def test_zeldovich_lattice_normalisation_and_order():
    n_side, nf = 16, 64
    x, v = dev.zeldovich_lattice(3, n_side, nf, device="cpu")
    assert x.shape == (n_side ** 3, 3) and x.dtype == torch.float32
    assert float(x.min()) >= 0.0 and float(x.max()) < nf
    # v = 0.1 psi with rms |psi| = 0.5 fine cells
    assert abs(float(torch.sqrt((v.double() ** 2).sum(1).mean())) - 0.05) < 1e-6
    # particle p sits near lattice point (ix, iy, iz), x fastest
    sp = nf / n_side
    g = (torch.arange(n_side, dtype=torch.float64) + 0.5) * sp
    q = torch.stack([g.repeat(n_side * n_side), g.repeat_interleave(n_side).repeat(n_side),
                     g.repeat_interleave(n_side * n_side)], dim=1)
    d = torch.remainder(x.double() - q + nf / 2, nf) - nf / 2
    assert torch.allclose(d, v.double() / 0.1, atol=1e-4)


def test_neutrino_slabs():
    nf, ns, per = 64, 16, 20000
    h = nf / ns
    speeds = []
    for k in (0, 7, 15):
        x, v = dev.neutrino_slab(5, k, ns, per, nf, device="cpu")
        assert float(x[:, 2].min()) >= k * h and float(x[:, 2].max()) < (k + 1) * h
        assert float(x[:, :2].min()) >= 0.0 and float(x[:, :2].max()) < nf
        assert torch.equal(v, dev.neutrino_slab(5, k, ns, per, nf, velocities_only=True, device="cpu"))
        speeds.append(v.double().norm(dim=1))
    # mean of u for p(u) ~ u^2 / (e^u + 1): (7/8) 3! zeta(4) / ((3/4) 2! zeta(3))
    zeta3 = 1.2020569031595942
    mean_u = (7.0 / 8.0) * 6.0 * math.pi ** 4 / 90.0 / ((3.0 / 4.0) * 2.0 * zeta3)
    s = torch.cat(speeds)
    assert abs(float(s.mean()) - 2.0 * mean_u) < 0.02 * 2.0 * mean_u
    # isotropic: each component's mean is near zero
    assert np.all(np.abs(v.double().mean(0).numpy()) < 0.1)
