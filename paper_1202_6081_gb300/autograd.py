"""Gradient of a flow objective with respect to a per-cell body force, by
the library's discrete adjoint (not in the paper: the reverse mode of its
update).

``macroscopic_after(solver, F, nsteps, every, f0)`` returns the density and
velocity fields (rho, u) after ``nsteps`` steps, differentiable with respect
to the force field F and, when given, the initial state f0 (FP64
[Q, nz, ny, nx]): any torch objective of (rho, u) can be back-propagated
through the run.  Its backward seeds the adjoint with
``lbm_macroscopic_seed`` from the incoming gradients of rho and u.

``kinetic_energy_after(solver, F, nsteps, every)`` returns
J = sum_x rho |u|^2 / 2 after ``nsteps`` steps from the solver's current
state under the force field F (device FP32 [3, nz, ny, nx]), as a
differentiable torch scalar.  Forward: steps with a checkpoint of the state
every ``every`` steps.  Backward: for each segment, last to first, the
segment's states are recomputed from its checkpoint into a ring of buffers
(``lbm_step_into``), then ``lbm_adjoint_step`` runs from the segment's last
step back to its first, accumulating dJ/dF on the device; the final state
seeds the adjoint (``lbm_kinetic_energy_seed``).  The recomputation of the
next segment runs on a second stream, beside the adjoint steps of the
current one.  Every step runs in the CUDA
kernels of liblbm.so; torch holds the buffers.
"""
from __future__ import annotations

import torch


class _KineticEnergyAfter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, nsteps, every):
        _check_force(F)
        if nsteps < 1 or every < 1:
            raise ValueError("nsteps and every must be >= 1")
        solver.set_force_field(F)
        ckpts = _forward_with_checkpoints(solver, nsteps, every)
        J = solver.kinetic_energy()
        ctx.solver, ctx.nsteps, ctx.every, ctx.ckpts = solver, nsteps, every, ckpts
        ctx.save_for_backward(F)
        return torch.tensor(J, dtype=torch.float64, device=F.device)

    @staticmethod
    def backward(ctx, gJ):
        (F,) = ctx.saved_tensors
        S = ctx.solver
        S.set_force_field(F)
        gF = torch.zeros_like(F)

        def seed(buf, lam):
            S.kinetic_energy_seed(buf, lam, gF)

        _backward_segments(S, ctx.nsteps, ctx.every, ctx.ckpts, seed, gF)
        ctx.ckpts = None
        return gF * gJ.to(gF.dtype), None, None, None


def _check_force(F):
    if not (F.is_cuda and F.dtype == torch.float32 and F.is_contiguous()):
        raise ValueError("F must be a contiguous CUDA float32 tensor [3, nz, ny, nx]")


def _forward_with_checkpoints(solver, nsteps, every):
    """nsteps steps in runs of `every` (one library call per run, so long
    runs go out as CUDA graphs), with a copy of the state at the start of
    each run."""
    ckpts = [solver.current_buffer().clone()]
    done = 0
    while done < nsteps:
        n = min(every, nsteps - done)
        solver.step(n)
        done += n
        if done < nsteps:
            ckpts.append(solver.current_buffer().clone())
    return ckpts


def _second_ring_fits(ring):
    """Whether a second ring like `ring` fits in the device memory still free
    (the driver's free memory plus the blocks torch holds cached), with 1 GiB
    to spare.  Host tensors (test fakes): always."""
    if not ring[0].is_cuda:
        return True
    dev = ring[0].device
    free, _ = torch.cuda.mem_get_info(dev)
    cached = torch.cuda.memory_reserved(dev) - torch.cuda.memory_allocated(dev)
    need = sum(b.numel() * b.element_size() for b in ring)
    return free + cached >= need + (1 << 30)


def _backward_segments(S, nsteps, every, ckpts, seed, gF):
    """Adjoint sweep over the checkpointed segments, last to first; `seed`
    fills the adjoint field from the final state.  Returns the adjoint of
    the initial state (a pitched FP32 field).

    Two rings of state buffers when they fit: while the adjoint steps of
    segment s run on the caller's stream from one ring, a second stream
    recomputes the states of segment s - 1 into the other, so the two
    memory-bound sweeps share the GPU (events order each ring's reuse).
    Otherwise one ring, each segment recomputed after the adjoint steps of
    the one after it."""
    lam = S.new_adjoint_field()
    lam2 = S.new_adjoint_field()
    m = min(every, nsteps) + 1
    nseg = len(ckpts)
    rings = [[S.new_state_buffer() for _ in range(m)]]
    two = nseg > 1 and _second_ring_fits(rings[0])
    if two:
        rings.append([S.new_state_buffer() for _ in range(m)])
    cuda = two and rings[0][0].is_cuda  # host-side fakes run the same schedule in order
    if cuda:
        dev = rings[0][0].device
        main = torch.cuda.current_stream(dev)
        side = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]  # ring r holds its segment
        free = [torch.cuda.Event(), torch.cuda.Event()]   # ring r may be overwritten
        side.wait_stream(main)  # checkpoints, force field and buffers are ready

    def bounds(s):
        t0 = s * every
        return t0, min(t0 + every, nsteps)

    def recompute(s, ring):
        # the adjoint steps need the states t0 .. t1 - 1; the state at t1 is
        # recomputed only in the last segment, where it seeds the adjoint
        t0, t1 = bounds(s)
        ring[0].copy_(ckpts[s])
        for i in range(t1 - t0 if s == nseg - 1 else t1 - t0 - 1):
            S.step_into(ring[i], ring[i + 1])

    recompute(nseg - 1, rings[0])
    r = 0
    for s in reversed(range(nseg)):
        if two and s > 0:
            if cuda:
                with torch.cuda.stream(side):
                    if s < nseg - 1:
                        side.wait_event(free[1 - r])  # its last adjoint sweep is done
                    recompute(s - 1, rings[1 - r])
                    ready[1 - r].record(side)
            else:
                recompute(s - 1, rings[1 - r])
        t0, t1 = bounds(s)
        ring = rings[r]
        if s == nseg - 1:
            seed(ring[t1 - t0], lam)
        for i in reversed(range(t1 - t0)):
            S.adjoint_step(ring[i], lam, lam2, gF)
            lam, lam2 = lam2, lam
        if not two:
            if s > 0:
                recompute(s - 1, rings[0])
            continue
        if cuda:
            free[r].record(main)
            if s > 0:
                main.wait_event(ready[1 - r])
        r = 1 - r
    return lam


class _MacroscopicAfter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, f0, solver, nsteps, every):
        _check_force(F)
        if nsteps < 1 or every < 1:
            raise ValueError("nsteps and every must be >= 1")
        solver.set_force_field(F)
        if f0 is not None:
            solver.set_state(f0)
        ckpts = _forward_with_checkpoints(solver, nsteps, every)
        rho, u = solver.macroscopic()
        ctx.solver, ctx.nsteps, ctx.every, ctx.ckpts = solver, nsteps, every, ckpts
        ctx.has_f0 = f0 is not None
        ctx.save_for_backward(F)
        return rho, u

    @staticmethod
    def backward(ctx, g_rho, g_u):
        (F,) = ctx.saved_tensors
        S = ctx.solver
        S.set_force_field(F)
        gF = torch.zeros_like(F)

        def seed(buf, lam):
            S.macroscopic_seed(buf, g_rho, g_u, lam, gF)

        lam0 = _backward_segments(S, ctx.nsteps, ctx.every, ctx.ckpts, seed, gF)
        ctx.ckpts = None
        g_f0 = S.adjoint_view(lam0).double() if ctx.has_f0 else None
        return gF, g_f0, None, None, None


def macroscopic_after(solver, F, nsteps, every=20, f0=None):
    """Differentiable (rho, u) after nsteps steps under the force field F
    (from the initial state f0 if given, else the solver's current state)."""
    return _MacroscopicAfter.apply(F, f0, solver, int(nsteps), int(every))


def kinetic_energy_after(solver, F, nsteps, every=20):
    """Differentiable J(F) = sum_x rho |u|^2 / 2 after nsteps steps."""
    return _KineticEnergyAfter.apply(F, solver, int(nsteps), int(every))
