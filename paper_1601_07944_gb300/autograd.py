"""Differentiable SSP-RK3 time integration through the library's discrete adjoint.

``solve(mesh, c0, dt, nsteps, every=k)`` returns c(T) after ``nsteps`` steps and
is a ``torch.autograd.Function``: the forward pass keeps a checkpoint of the
state every ``k`` steps; the backward pass walks the segments last to first,
recomputes the states inside a segment from its checkpoint and applies the
transposed step (entirely in the CUDA kernels) from the last state of the
segment back to its first.  With ``keep_stages`` (the default) the recomputation
keeps every step's two stage values (``dg_rk_step_stages``) and the transposed
step takes them (``dg_adjoint_step_stages``) instead of recomputing them, for
3k states of memory per segment; without it the recomputation keeps the k
states (``dg_rk_step``) and ``dg_adjoint_step`` recomputes the stages.  Both
give the same gradient, bit for bit.  Memory is nsteps/k checkpoints plus one
segment's states.
"""
from __future__ import annotations

import torch


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c0, mesh, dt, nsteps, every, keep_stages):
        c = c0.detach().clone()
        ckpts = [c0.detach().clone()]
        for s in range(nsteps):
            mesh.rk_step(c, dt, 1)
            if (s + 1) % every == 0 and s + 1 < nsteps:
                ckpts.append(c.clone())
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.every, ctx.keep = mesh, dt, nsteps, every, keep_stages
        ctx.ckpts = ckpts
        return c

    @staticmethod
    def backward(ctx, grad):
        mesh, dt, nsteps, every = ctx.mesh, ctx.dt, ctx.nsteps, ctx.every
        lam = grad.detach().contiguous().clone()
        out = torch.empty_like(lam)
        nseg = len(ctx.ckpts)
        for seg in range(nseg - 1, -1, -1):
            first = seg * every
            last = min(nsteps, first + every)
            if ctx.keep:
                # every step of the segment with its stage values
                steps = []
                c = ctx.ckpts[seg].clone()
                for _ in range(first, last):
                    cn, u1, u2 = c.clone(), torch.empty_like(c), torch.empty_like(c)
                    mesh.rk_step_stages(c, dt, u1, u2)
                    steps.append((cn, u1, u2))
                for cn, u1, u2 in reversed(steps):
                    mesh.adjoint_step_stages(cn, u1, u2, dt, lam, out=out)
                    lam, out = out, lam
            else:
                states = [ctx.ckpts[seg]]
                for _ in range(first, last - 1):
                    nxt = states[-1].clone()
                    mesh.rk_step(nxt, dt, 1)
                    states.append(nxt)
                for st in reversed(states):
                    mesh.adjoint_step(st, dt, lam, out=out)
                    lam, out = out, lam
        ctx.ckpts = None
        return lam, None, None, None, None, None


def solve(mesh, c0: torch.Tensor, dt: float, nsteps: int, every: int = 20, keep_stages: bool = True) -> torch.Tensor:
    """c(T) after nsteps SSP-RK3 steps; differentiable with respect to c0."""
    if every < 1:
        raise ValueError("every must be >= 1")
    return _Solve.apply(c0, mesh, float(dt), int(nsteps), int(every), bool(keep_stages))


def density_misfit(mesh_det_j: torch.Tensor, c: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """1/2 sum_e det J_e sum_j (c_rho - c_rho_target)^2 = 1/2 int (rho_h - rho_target)^2
    (the basis is orthonormal on the reference triangle)."""
    d = c[:, 0, :] - target[:, 0, :]
    return 0.5 * torch.sum(mesh_det_j[:, None] * d * d)
