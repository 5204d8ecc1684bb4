"""Compression-accuracy study (the test of Sec. 2.4 on the synthetic sets).

Two runs from identical initial conditions are compared through their
density and velocity power spectra at the final step:

  * "uncompressed": float32 positions and velocities stepped with the
    library's plain per-stage calls (deposit, solve, kick + drift);
  * "restarts": the same, but the state is compressed to the Sec. 2.4 codes
    and decompressed again ("restarted") R times during the run (the paper
    uses 10 restarts);
  * "single": the final uncompressed state compressed once (the paper's
    comparison line: the error of one compression);
  * "resident": the state kept compressed throughout, one fused pm_step per
    step (this library's own mode: a compression every step).

Spectra are measured on an n^3 CIC mesh per species (n = the fine mesh),
deposited by the library (pm_deposit_weights): density contrast delta =
rho / mean - 1, and the momentum density sum_p v_d W / mean summed over d
for the velocity power (the paper does not define its velocity field;
momentum density avoids empty-cell division).  P(k) is averaged over
unit-width shells of |k| (fundamental units), as in oracle/power.py, which
pins the estimator; tests/test_analysis_cpu.py checks this torch version
against it.  This is analysis tooling: the PM step itself never calls it.
"""
from __future__ import annotations

import argparse
import json
from typing import Dict, Sequence

import torch


def power_spectrum(field: torch.Tensor):
    """(shells 1..n/2, P per shell) of a real n^3 field; estimator of oracle/power.py."""
    f = field.double()
    n = f.shape[-1]
    F = torch.fft.rfftn(f, dim=(-3, -2, -1))
    p = (F.real ** 2 + F.imag ** 2) / n ** 3
    m = torch.fft.fftfreq(n, 1.0 / n, device=f.device, dtype=torch.float64)
    mx = torch.arange(n // 2 + 1, device=f.device, dtype=torch.float64)
    kz, ky, kx = torch.meshgrid(m, m, mx, indexing="ij")
    shell = torch.round(torch.sqrt(kx * kx + ky * ky + kz * kz)).long()
    # modes 0 < kx < n/2 stand for themselves and their conjugate partner
    one = torch.ones_like(mx)
    weight = torch.where((mx > 0) & (mx < n / 2), 2.0 * one, one).expand_as(kx)
    nsh = n // 2
    sel = (shell >= 1) & (shell <= nsh)
    idx = shell[sel] - 1
    cnt = torch.zeros(nsh, dtype=torch.float64, device=f.device).index_add_(0, idx, weight[sel])
    tot = torch.zeros(nsh, dtype=torch.float64, device=f.device).index_add_(0, idx, (p * weight)[sel])
    return torch.arange(1, nsh + 1), (tot / cnt).cpu()


def spectra(pm, x: torch.Tensor, v: torch.Tensor) -> Dict[str, torch.Tensor]:
    """Density and velocity (momentum-density) power of one species: number
    and momentum densities deposited by the library (pm_deposit_weights,
    weights 1, v_x, v_y, v_z), spectra in float64."""
    n = pm.n_fine
    N = x.shape[0]
    mean = N / n ** 3
    w = torch.cat([torch.ones((N, 1), dtype=torch.float32, device=x.device), v.float()], dim=1)
    f = pm.deposit_weights(x, w).double()
    _, pd = power_spectrum(f[0] / mean - 1.0)
    pv = sum(power_spectrum(f[1 + d] / mean)[1] for d in range(3))
    return {"density": pd, "velocity": pv}


def compression_study(workload: str = "two_level64", steps: int = 22, restarts: int = 10, c: float = 0.25,
                      n_cdm=None, n_nu=None, vel_bits=None) -> Dict:
    """Run the four arms and return per-species power ratios minus one by shell."""
    from . import PM
    from synth import make_workload

    w = make_workload(workload, n_cdm=n_cdm, n_nu=n_nu)
    cfg = w.config()
    if vel_bits is not None:
        cfg["vel_bits"] = vel_bits
    pm = PM(cfg)
    n = w.n_fine
    x0 = [torch.from_numpy(a).cuda() for a in w.x]
    v0 = [torch.from_numpy(a).cuda() for a in w.v]

    def roundtrip(xs, vs):
        out = []
        for s in range(2):
            codes = pm.compress(s, xs[s], vs[s], out=pm.empty_codes(xs[s].shape[0], esc_cap=xs[s].shape[0] // 255 + 1))
            out.append(pm.decompress(s, codes))
        return [o[0] for o in out], [o[1] for o in out]

    # uncompressed and restarted runs
    every = max(1, steps // (restarts + 1))
    xu, vu = [a.clone() for a in x0], [a.clone() for a in v0]
    xr, vr = [a.clone() for a in x0], [a.clone() for a in v0]
    n_restarts = 0
    for k in range(1, steps + 1):
        pm.step_plain(xu, vu, c, c, fixed=False)
        pm.step_plain(xr, vr, c, c, fixed=False)
        if k % every == 0 and n_restarts < restarts:
            xr, vr = roundtrip(xr, vr)
            n_restarts += 1
    xs1, vs1 = roundtrip(xu, vu)
    # resident: compressed codes stepped by pm_step
    a = [pm.compress(s, x0[s], v0[s], out=pm.empty_codes(x0[s].shape[0], esc_cap=x0[s].shape[0] // 255 + 1))
         for s in range(2)]
    b = [pm.empty_codes(cd.n, esc_cap=cd.esc.shape[0]) for cd in a]
    for _ in range(steps):
        pm.step(a, b, c, c)
        a, b = b, a
    xf, vf = zip(*[pm.decompress(s, a[s]) for s in range(2)])
    pm.check()
    result = {"workload": workload, "steps": steps, "restarts": n_restarts, "c_kick": c, "c_drift": c,
              "n_mesh": n, "vel_bits": cfg["vel_bits"], "species": {}}
    for s, name in enumerate(("cdm", "nu")):
        ref = spectra(pm, xu[s], vu[s])
        arms = {"restarts": spectra(pm, xr[s], vr[s]), "single": spectra(pm, xs1[s], vs1[s]),
                "resident": spectra(pm, xf[s], vf[s])}
        sp = {"P_density": ref["density"].tolist(), "P_velocity": ref["velocity"].tolist(),
              "shot_noise": n ** 3 / x0[s].shape[0]}
        for arm, p in arms.items():
            sp[arm] = {q: (p[q] / ref[q] - 1.0).tolist() for q in ("density", "velocity")}
        result["species"][name] = sp
    pm.close()
    return result


def summary(result: Dict) -> Dict:
    """max |P_arm / P - 1| for density up to k_Nyq/2 and velocity up to k_Nyq/3 (the
    ranges the paper quotes), and for nu also below k_noise (P_density > shot noise)."""
    n = result["n_mesh"]
    out = {}
    for name, sp in result["species"].items():
        jd, jv = n // 4, n // 6
        pd = sp["P_density"]
        j_noise = next((j for j, p in enumerate(pd) if p < sp["shot_noise"]), len(pd))
        row = {"k_noise_shell": j_noise}
        for arm in ("restarts", "single", "resident"):
            d, v = sp[arm]["density"], sp[arm]["velocity"]
            row[arm] = {"density_to_nyq2": max(abs(a) for a in d[:jd]),
                        "velocity_to_nyq3": max(abs(a) for a in v[:jv]),
                        "density_below_k_noise": max([abs(a) for a in d[:min(jd, j_noise)]] or [0.0])}
        out[name] = row
    return out


def main(argv: Sequence[str] = None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="two_level64")
    p.add_argument("--steps", type=int, default=22)
    p.add_argument("--restarts", type=int, default=10)
    p.add_argument("--c", type=float, default=0.25)
    p.add_argument("--vel-bits", type=int, default=None, choices=[8, 16])
    args = p.parse_args(argv)
    r = compression_study(args.workload, args.steps, args.restarts, args.c, vel_bits=args.vel_bits)
    print(json.dumps({"config": {k: r[k] for k in ("workload", "steps", "restarts", "c_kick", "n_mesh", "vel_bits")},
                      "summary": summary(r)}))


if __name__ == "__main__":
    main()
