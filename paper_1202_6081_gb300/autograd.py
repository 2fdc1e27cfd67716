"""Gradient of a flow objective with respect to a per-cell body force, by
the library's discrete adjoint (not in the paper: the reverse mode of its
update).

``kinetic_energy_after(solver, F, nsteps, every)`` returns
J = sum_x rho |u|^2 / 2 after ``nsteps`` steps from the solver's current
state under the force field F (device FP32 [3, nz, ny, nx]), as a
differentiable torch scalar.  Forward: steps with a checkpoint of the state
every ``every`` steps.  Backward: for each segment, last to first, the
segment's states are recomputed from its checkpoint into a ring of buffers
(``lbm_step_into``), then ``lbm_adjoint_step`` runs from the segment's last
step back to its first, accumulating dJ/dF on the device; the final state
seeds the adjoint (``lbm_kinetic_energy_seed``).  Every step runs in the CUDA
kernels of liblbm.so; torch holds the buffers.
"""
from __future__ import annotations

import torch


class _KineticEnergyAfter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, nsteps, every):
        if not (F.is_cuda and F.dtype == torch.float32 and F.is_contiguous()):
            raise ValueError("F must be a contiguous CUDA float32 tensor [3, nz, ny, nx]")
        if nsteps < 1 or every < 1:
            raise ValueError("nsteps and every must be >= 1")
        solver.set_force_field(F)
        ckpts = [solver.current_buffer().clone()]
        for t in range(nsteps):
            solver.step(1)
            if (t + 1) % every == 0 and t + 1 < nsteps:
                ckpts.append(solver.current_buffer().clone())
        J = solver.kinetic_energy()
        ctx.solver = solver
        ctx.nsteps = nsteps
        ctx.every = every
        ctx.ckpts = ckpts
        ctx.save_for_backward(F)
        return torch.tensor(J, dtype=torch.float64, device=F.device)

    @staticmethod
    def backward(ctx, gJ):
        (F,) = ctx.saved_tensors
        S, nsteps, every, ckpts = ctx.solver, ctx.nsteps, ctx.every, ctx.ckpts
        S.set_force_field(F)
        gF = torch.zeros_like(F)
        lam = S.new_adjoint_field()
        lam2 = S.new_adjoint_field()
        ring = [S.new_state_buffer() for _ in range(min(every, nsteps) + 1)]
        nseg = len(ckpts)
        for s in reversed(range(nseg)):
            t0 = s * every
            t1 = min(t0 + every, nsteps)
            ring[0].copy_(ckpts[s])
            for i in range(t1 - t0):
                S.step_into(ring[i], ring[i + 1])
            if s == nseg - 1:
                S.kinetic_energy_seed(ring[t1 - t0], lam, gF)
            for i in reversed(range(t1 - t0)):
                S.adjoint_step(ring[i], lam, lam2, gF)
                lam, lam2 = lam2, lam
        ctx.ckpts = None
        return gF * gJ.to(gF.dtype), None, None, None


def kinetic_energy_after(solver, F, nsteps, every=20):
    """Differentiable J(F) = sum_x rho |u|^2 / 2 after nsteps steps."""
    return _KineticEnergyAfter.apply(F, solver, int(nsteps), int(every))
