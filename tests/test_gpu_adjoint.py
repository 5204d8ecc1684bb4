"""GPU reverse mode of the single-mesh step against the float64 oracle
adjoint: the transposed solve, one reverse step, and the gradient of a
final-density loss through a checkpointed multi-step trajectory."""
import numpy as np
import pytest
import torch

from oracle import adjoint, solve
from synth import make_workload
from tests.helpers import rel_rms

pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-3   # float32 adjoint vs float64 oracle, relative RMS


def _pm(cfg):
    from paper_1611_01545_gb300 import PM
    return PM(cfg)


def _cfg(n=32, counts=(512, 4096)):
    return dict(n_fine=n, coarse_ratio=1, tile=n, buffer=0, cmp_ratio=4, vel_bits=16, G=1 / (4 * np.pi),
                mass=(8.0, 0.04), count=counts, deposit_mode=1)


def test_solve_adjoint_is_transpose_gpu():
    pm = _pm(_cfg(32))
    g = torch.Generator(device="cuda").manual_seed(3)
    rho = torch.randn((32,) * 3, device="cuda", generator=g)
    lam = torch.randn((3,) + (32,) * 3, device="cuda", generator=g)
    _, af = pm.zeros_acc()
    pm.solve(None, rho, None, af)
    lr = torch.empty_like(rho)
    pm.solve_adjoint(lam, lr)
    pm.check()
    lhs = float((af.double() * lam.double()).sum())
    rhs = float((rho.double() * lr.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    ref = adjoint.accel_periodic_adjoint(lam.cpu().numpy().astype(np.float64), 1.0, 1 / (4 * np.pi))
    assert rel_rms(lr.cpu().numpy(), ref) < 1e-5


def _particles(seed, n, n0, n1):
    rng = np.random.default_rng(seed)
    xs = [(rng.random((k, 3)) * n).astype(np.float32) for k in (n0, n1)]
    vs = [(rng.standard_normal((k, 3)) * 0.3).astype(np.float32) for k in (n0, n1)]
    return xs, vs


def test_one_reverse_step_matches_oracle():
    n = 32
    cfg = _cfg(n)
    pm = _pm(cfg)
    xs, _ = _particles(5, n, 512, 4096)
    rng = np.random.default_rng(6)
    lx = [rng.standard_normal(x.shape).astype(np.float32) for x in xs]
    lv = [rng.standard_normal(x.shape).astype(np.float32) for x in xs]
    gx = [torch.from_numpy(a).cuda() for a in lx]
    gv = [torch.from_numpy(a).cuda() for a in lv]
    pm.step_adjoint([torch.from_numpy(x).cuda() for x in xs], gx, gv, 0.5, 0.5)
    pm.check()
    rx, rv = adjoint.reverse_step([x.astype(np.float64) for x in xs], cfg, lx, lv, 0.5, 0.5)
    for s in range(2):
        assert rel_rms(gv[s].cpu().numpy(), rv[s]) < ADJ_TOL
        assert rel_rms(gx[s].cpu().numpy(), rx[s]) < ADJ_TOL, (s, rel_rms(gx[s].cpu().numpy(), rx[s]))


def test_reverse_step_with_supplied_acceleration_is_identical():
    """pm_step_adjoint_acc with the forward step's own mesh (fixed-point deposit:
    the recompute is bit-identical) gives pm_step_adjoint's result, up to the
    order of the float reductions into the adjoint mesh."""
    from paper_1611_01545_gb300.pm import PMError
    n = 32
    pm = _pm(_cfg(n))
    xs, vs = _particles(8, n, 512, 4096)
    xt = [torch.from_numpy(x).cuda() for x in xs]
    rng = np.random.default_rng(9)
    lam = [[torch.from_numpy(rng.standard_normal(x.shape).astype(np.float32)).cuda() for x in xs] for _ in range(2)]
    ref = [[t.clone() for t in grp] for grp in lam]
    af = pm.step_plain([x.clone() for x in xt], [torch.from_numpy(v).cuda() for v in vs], 0.5, 0.5, fixed=True)
    pm.step_adjoint(xt, ref[0], ref[1], 0.5, 0.5)
    pm.step_adjoint(xt, lam[0], lam[1], 0.5, 0.5, acc_fine=af)
    pm.check()
    for a, b in zip(lam[0] + lam[1], ref[0] + ref[1]):
        assert rel_rms(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
    st = (pm.lib.pm_step_adjoint_acc.argtypes[1]._type_ * 2)()
    with pytest.raises(PMError):
        pm._err(pm.lib.pm_step_adjoint_acc(pm.h, st, st, None, 0.5, 0.5, None))


@pytest.mark.parametrize("beta,every", [(0.0, 2), (0.3, 2), (0.3, 3)])
def test_trajectory_gradient_matches_oracle(beta, every):
    """every=3 over 4 steps gives a 3-step segment (two recomputed steps) and a
    1-step segment (none recomputed)."""
    from paper_1611_01545_gb300.diff import trajectory_loss
    w = make_workload("diff128", n_cdm=8, n_nu=16)
    n = 32
    w.x = [np.mod(x * (n / 128.0), n).astype(np.float32) for x in w.x]
    cfg = _cfg(n, counts=(8 ** 3, 16 ** 3))
    pm = _pm(cfg)
    rng = np.random.default_rng(7)
    q = w.x[0]
    psi = (rng.standard_normal(q.shape) * 0.3).astype(np.float32)
    vnu = (w.v[1] * 0.2).astype(np.float32)
    target = (rng.random((n, n, n)) * 0.02).astype(np.float32)
    steps, ck, cd = 4, 0.5, 0.5
    psi_t = torch.from_numpy(psi).cuda().requires_grad_(True)
    L = trajectory_loss(pm, psi_t, torch.from_numpy(q).cuda(), torch.from_numpy(w.x[1]).cuda(),
                        torch.from_numpy(vnu).cuda(), torch.from_numpy(target).cuda(), beta, steps, every, ck, cd)
    L.backward()
    pm.check()
    x0 = [np.mod(q.astype(np.float64) + psi, n), w.x[1].astype(np.float64)]
    v0 = [beta * psi.astype(np.float64), vnu.astype(np.float64)]
    lx, lv = adjoint.gradient(x0, v0, cfg, ck, cd, steps, target.astype(np.float64))
    ref_loss = adjoint.loss(adjoint.forward(x0, v0, cfg, ck, cd, steps)[-1][0], cfg, target)
    assert abs(float(L.detach()) - ref_loss) <= 1e-4 * ref_loss
    ref_grad = lx[0] + beta * lv[0]
    assert rel_rms(psi_t.grad.cpu().numpy(), ref_grad) < ADJ_TOL


def test_trajectory_gradient_matches_central_differences_gpu():
    """The GPU gradient against central differences of the GPU forward pass
    itself (eps = 1e-3 cells along random directions; the fixed-point deposit
    makes the forward deterministic, float32 positions and the CIC kinks limit
    the agreement to about a percent)."""
    from paper_1611_01545_gb300.diff import trajectory_loss
    w = make_workload("diff128", n_cdm=8, n_nu=16)
    n = 32
    w.x = [np.mod(x * (n / 128.0), n).astype(np.float32) for x in w.x]
    cfg = _cfg(n, counts=(8 ** 3, 16 ** 3))
    pm = _pm(cfg)
    rng = np.random.default_rng(11)
    q = torch.from_numpy(w.x[0]).cuda()
    psi = torch.from_numpy((rng.standard_normal(w.x[0].shape) * 0.3).astype(np.float32)).cuda()
    xnu = torch.from_numpy(w.x[1]).cuda()
    vnu = torch.from_numpy((w.v[1] * 0.2).astype(np.float32)).cuda()
    target = torch.from_numpy((rng.random((n, n, n)) * 0.02).astype(np.float32)).cuda()
    args = (q, xnu, vnu, target, 0.3, 4, 2, 0.5, 0.5)
    p = psi.clone().requires_grad_(True)
    trajectory_loss(pm, p, *args).backward()
    g = p.grad.double()
    eps = 1e-3
    # along the gradient itself, then along random directions, whose directional
    # derivative sums terms of both signs: the tolerance scales with sum |g_i d_i|
    dirs = [p.grad.detach().clone()] + [torch.from_numpy(rng.standard_normal(w.x[0].shape).astype(np.float32)).cuda()
                                        for _ in range(2)]
    for k, d in enumerate(dirs):
        d /= d.abs().max()        # every coordinate moves by up to eps: far above float32 rounding
        lp = float(trajectory_loss(pm, psi + eps * d, *args).detach())
        lm = float(trajectory_loss(pm, psi - eps * d, *args).detach())
        fd = (lp - lm) / (2 * eps)
        an = float((g * d.double()).sum())
        scale = float((g * d.double()).abs().sum())
        assert abs(fd - an) <= 2e-2 * scale, (k, fd, an, scale)
    pm.check()


def _golden_diff128():
    """The float64 oracle's gradient of the 128^3 differentiable workload
    (tests/golden/diff128_gradient.txt, written by make_diff128_gradient.py
    beside it, which calls only oracle/) and that script's input recipe."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_diff128_gradient",
                                                  os.path.join(here, "make_diff128_gradient.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rec = {"sample": [], "proj": []}
    with open(os.path.join(here, "diff128_gradient.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key in ("sample", "proj"):
                rec[key].append([float(v) for v in vals])
            else:
                rec[key] = float(vals[0])
    return mod, rec


def test_diff128_gradient_matches_oracle():
    """The differentiable workload at its own shape: 128^3 mesh, 64^3 CDM +
    128^3 neutrinos, 10 steps, checkpoints every 2 steps.  The GPU loss and
    gradient (float32, fixed-point deposits) against the float64 oracle's:
    the loss, 1024 sampled gradient components, and the projections of the
    whole gradient on four random directions (relative to sum |g_i d_i|).
    Over ten 128^3 steps the gradient is ill conditioned at the scale of
    float32 rounding (CIC gradients change at cell faces): the tolerance is
    three times the relative change of the oracle's own gradient when every
    start coordinate moves by 1e-5 cells (stored beside the gradient), and
    at least the 1e-3 of the small trajectories."""
    from paper_1611_01545_gb300.diff import trajectory_loss
    mod, rec = _golden_diff128()
    cfg, q, psi, x_nu, v_nu, target = mod.diff128_inputs()
    assert int(rec["steps"]) == mod.STEPS
    pm = _pm(cfg)
    psi_t = torch.from_numpy(psi).cuda().requires_grad_(True)
    L = trajectory_loss(pm, psi_t, torch.from_numpy(q).cuda(), torch.from_numpy(x_nu).cuda(),
                        torch.from_numpy(v_nu).cuda(), torch.from_numpy(target).cuda(), mod.BETA, mod.STEPS,
                        mod.EVERY, mod.C_KICK, mod.C_DRIFT)
    L.backward()
    pm.check()
    assert abs(float(L.detach()) - rec["loss"]) <= 1e-4 * rec["loss"]
    g = psi_t.grad.double().cpu().numpy()
    sample = np.array(rec["sample"])
    idx = sample[:, 0].astype(np.int64)
    np.testing.assert_array_equal(idx, mod.sample_index())
    tol = max(ADJ_TOL, 3.0 * rec["sensitivity"])
    err = rel_rms(g[idx], sample[:, 1:])
    print(f"diff128 gradient: sampled relative RMS {err:.2e} (oracle sensitivity {rec['sensitivity']:.2e}, "
          f"tolerance {tol:.2e})")
    assert err < tol
    for (k, proj, scale), d in zip(rec["proj"], mod.directions()):
        got = float(np.sum(g * d))
        assert abs(got - proj) <= tol * scale, (k, got, proj, scale)
