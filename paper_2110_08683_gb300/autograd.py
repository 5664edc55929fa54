"""Reverse mode of a GP-MOOD rollout as a torch.autograd.Function.

Every step's tape is its three stage inputs and the final radii of its three
stages (12 + 3/8 doubles a cell).  The reverse pass needs the tapes in
reverse order; where they fit in the memory budget the forward records them
all as it goes (the forward then costs the same as a plain rollout plus the
tape writes), otherwise the forward keeps the state and time every `every`
steps (checkpoints), queueing its steps without waiting for them, and the
reverse pass steps each segment again from its checkpoint, which reproduces
the forward bit for bit (the same kernels on the same data, so the same
time steps and MOOD decisions), recording its tapes.  A re-recorded segment
also keeps its face-state tapes (the reconstructed states of every face)
when they fit the memory budget, so that the adjoint does not reconstruct
them again.  Then the hand-written adjoint of each step runs in reverse
with the radii and dt held at their forward values.  Torch only provides
the device memory.
"""
from __future__ import annotations

import torch


def tape_bytes(model):
    """device bytes of one step's tape"""
    nc = model.nx * model.ny
    return 3 * 4 * nc * 8 + 3 * nc


def state_tape_bytes(model):
    """device bytes of one step's face-state tape"""
    return model.state_tape_bytes()


def default_budget():
    """half of the device memory free now"""
    free, _ = torch.cuda.mem_get_info()
    return free // 2


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, model, nsteps, every, cfl, budget, states):
        assert U0.is_cuda and U0.dtype == torch.float64 and U0.is_contiguous()
        ny, nx = model.ny, model.nx
        dev = U0.device
        if budget is None:
            budget = default_budget()
        resident = every is None and nsteps * tape_bytes(model) <= budget
        if every is None:
            # checkpoints (one state each) plus one segment of tapes in the budget
            every = max(1, min(nsteps, int(budget // max(tape_bytes(model), 1)) // 2))
        model.set_state(U0.detach())
        ckpts, dts, ts = [], [], []
        tape = otape = None
        if resident:
            tape = torch.empty((nsteps, 3, 4, ny, nx), dtype=torch.float64, device=dev)
            otape = torch.empty((nsteps, 3, ny, nx), dtype=torch.uint8, device=dev)
            t = 0.0
            for k in range(nsteps):
                dt = model.step_record(tape[k].data_ptr(), otape[k].data_ptr(), cfl=cfl)
                dts.append(dt)
                ts.append(t)
                t += dt
        else:
            # a checkpoint (state and time) at the start of every segment; the
            # segment's steps are queued without waiting for them
            for k0 in range(0, nsteps, every):
                c = torch.empty_like(U0)
                model.get_state(c)
                ckpts.append((k0, c, model.flags(maps=False)[2]["t"]))
                for _ in range(k0, min(k0 + every, nsteps)):
                    model.step_async(cfl)
            model.sync()
        out = torch.empty_like(U0)
        model.get_state(out)
        ctx.model, ctx.nsteps, ctx.every, ctx.resident = model, nsteps, every, resident
        ctx.ckpts, ctx.dts, ctx.ts = ckpts, dts, ts
        ctx.tape, ctx.otape = tape, otape
        ctx.cfl, ctx.budget, ctx.states = cfl, budget, states
        return out

    @staticmethod
    def backward(ctx, gout):
        model = ctx.model
        lam = gout.contiguous().clone()
        tmp = torch.empty_like(lam)
        torch.cuda.synchronize()
        if ctx.resident:
            for k in reversed(range(ctx.nsteps)):
                model.step_adjoint(ctx.tape[k].data_ptr(), ctx.otape[k].data_ptr(), ctx.dts[k],
                                   ctx.ts[k], lam.data_ptr(), tmp.data_ptr())
                lam, tmp = tmp, lam
            ctx.tape = ctx.otape = None
            return lam, None, None, None, None, None, None
        every = ctx.every
        ny, nx = model.ny, model.nx
        tape = torch.empty((every, 3, 4, ny, nx), dtype=torch.float64, device=gout.device)
        otape = torch.empty((every, 3, ny, nx), dtype=torch.uint8, device=gout.device)
        # the segment's face-state tapes, where they fit the budget
        stape, sb = None, 0
        if ctx.states:
            sb = state_tape_bytes(model)
            if every * (sb + tape_bytes(model)) <= ctx.budget:
                try:
                    stape = torch.empty(every * sb, dtype=torch.uint8, device=gout.device)
                except torch.cuda.OutOfMemoryError:
                    stape = None
        for k0, U, t0 in reversed(ctx.ckpts):
            k1 = min(k0 + every, ctx.nsteps)
            model.set_state(U)
            model.set_time(t0)
            # the segment again: the same steps as the forward, now recorded
            dts, ts, t = [], [], t0
            for k in range(k0, k1):
                if stape is not None:
                    dt = model.step_record_states(tape[k - k0].data_ptr(),
                                                  otape[k - k0].data_ptr(),
                                                  stape.data_ptr() + (k - k0) * sb, cfl=ctx.cfl)
                else:
                    dt = model.step_record(tape[k - k0].data_ptr(), otape[k - k0].data_ptr(),
                                           cfl=ctx.cfl)
                dts.append(dt)
                ts.append(t)
                t += dt
            for k in reversed(range(k0, k1)):
                i = k - k0
                if stape is not None:
                    model.step_adjoint_states(tape[i].data_ptr(), otape[i].data_ptr(),
                                              stape.data_ptr() + i * sb, dts[i], ts[i],
                                              lam.data_ptr(), tmp.data_ptr())
                else:
                    model.step_adjoint(tape[i].data_ptr(), otape[i].data_ptr(), dts[i], ts[i],
                                       lam.data_ptr(), tmp.data_ptr())
                lam, tmp = tmp, lam
        return lam, None, None, None, None, None, None


def rollout(U0, model, nsteps, every=None, cfl=None, budget=None, states=True):
    """U_N of `nsteps` CFL steps from U0 (CUDA float64 (4, ny, nx)), differentiable.

    every=None: keep all tapes resident when nsteps tapes fit in `budget`
    bytes (default: half the free device memory), else checkpoint segments
    sized to the budget.  every=k: checkpoints every k steps, segments
    recomputed in the reverse pass, with their face-state tapes when
    `states` and they fit the budget."""
    return Rollout.apply(U0, model, nsteps, every,
                         model.prob["cfl"] if cfl is None else cfl, budget, states)
