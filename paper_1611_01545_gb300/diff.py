"""Differentiable PM trajectories: a torch.autograd.Function over the library's
forward step and its reverse mode (single periodic mesh).

The loss is L = sum_c (rho_K(c) - target(c))^2 of the density after K steps,
the variable the initial CDM displacement field psi (x0 = q + psi wrapped
into the box, v0 = beta psi); neutrinos start from fixed phase-space
positions.  The forward pass keeps the state every `every` steps, and with
it the force mesh of the segment's last step; the backward pass recomputes
each segment from its checkpoint up to the positions before its last step
(the fixed-point deposit makes the recompute bit-identical), keeping the
recomputed steps' force meshes, and runs the reverse steps with those
meshes.  All mesh and particle arithmetic runs in libpm's kernels; torch
supplies memory and the loss's elementwise terms.
"""
from __future__ import annotations

from typing import List

import torch

from .pm import PM

MASS_UNIT = 2.0 ** -32   # fixed-point mass unit of the int64 deposit


def _wrap(x: torch.Tensor, n: int) -> torch.Tensor:
    x = torch.remainder(x, float(n))
    return torch.where(x >= n, torch.zeros_like(x), x)


def final_density(pm: PM, xs: List[torch.Tensor]) -> torch.Tensor:
    _, rf = pm.density(xs, fixed=True)
    return rf.to(torch.float64) * MASS_UNIT


class PMTrajectoryLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, pm, q, x_nu, v_nu, target, beta, steps, every, c_kick, c_drift):
        n = pm.n_fine
        x = [_wrap(q + psi.detach(), n).contiguous(), x_nu.clone()]
        v = [(beta * psi.detach()).contiguous(), v_nu.clone()]
        checkpoints = []
        for k in range(steps):
            if k % every == 0:
                checkpoints.append([k, [t.clone() for t in x], [t.clone() for t in v], None])
            acc = pm.step_plain(x, v, c_kick, c_drift, fixed=True)
            if k % every == every - 1 or k == steps - 1:
                checkpoints[-1][3] = acc     # the force mesh of the segment's last step
        rho = final_density(pm, x)
        diff = rho - target.to(torch.float64)
        ctx.pm, ctx.beta, ctx.steps, ctx.every = pm, beta, steps, every
        ctx.ck, ctx.cd = c_kick, c_drift
        ctx.checkpoints = checkpoints
        ctx.save_for_backward(diff.to(torch.float32), x[0], x[1])
        return torch.sum(diff * diff)     # float64: a sum of many squares

    @staticmethod
    def backward(ctx, gout):
        pm = ctx.pm
        diff, xK0, xK1 = ctx.saved_tensors
        lam_rho = (2.0 * gout.to(torch.float32) * diff).contiguous()
        lam_x = [torch.zeros_like(xK0), torch.zeros_like(xK1)]
        lam_v = [torch.zeros_like(xK0), torch.zeros_like(xK1)]
        for s, xk in enumerate((xK0, xK1)):
            pm.deposit_adjoint(s, xk, lam_rho, lam_x[s])
        for idx in range(len(ctx.checkpoints) - 1, -1, -1):
            k0, x0, v0, acc_last = ctx.checkpoints[idx]
            k1 = ctx.checkpoints[idx + 1][0] if idx + 1 < len(ctx.checkpoints) else ctx.steps
            # pre-step positions of steps k0 .. k1-1: the checkpoint and k1-k0-1
            # recomputed steps (the segment's last step is never re-run: its
            # adjoint needs only the positions before it, and its force mesh
            # was kept by the forward pass).  A recomputed step keeps its force
            # mesh for its reverse step, so no reverse step recomputes one.
            pre = [[x0, None]]
            if k1 - k0 > 1:
                x = [t.clone() for t in x0]
                v = [t.clone() for t in v0]
                for _ in range(k0, k1 - 1):
                    pre[-1][1] = pm.step_plain(x, v, ctx.ck, ctx.cd, fixed=True)
                    pre.append([[t.clone() for t in x], None])
            pre[-1][1] = acc_last
            for xs, acc in reversed(pre):
                pm.step_adjoint(xs, lam_x, lam_v, ctx.ck, ctx.cd, acc_fine=acc)
        grad = lam_x[0] + ctx.beta * lam_v[0]
        return grad, None, None, None, None, None, None, None, None, None, None


def trajectory_loss(pm: PM, psi, q, x_nu, v_nu, target, beta=0.0, steps=10, every=2, c_kick=1.0, c_drift=1.0):
    """L(psi) = sum (rho_K - target)^2 after `steps` PM steps (a float64 scalar);
    differentiable in psi."""
    return PMTrajectoryLoss.apply(psi, pm, q, x_nu, v_nu, target, float(beta), int(steps), int(every),
                                  float(c_kick), float(c_drift))
