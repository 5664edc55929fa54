"""Reverse mode of a GP-MOOD rollout as a torch.autograd.Function.

Forward: N steps of the CUDA path (CFL time steps), keeping the state every
`every` steps (checkpoints) and every step's dt.  Backward: segment by
segment from the last, the segment is stepped again from its checkpoint with
the recorded dt's, which reproduces the forward bit for bit (the same
kernels, so the same MOOD decisions), recording each step's tape (stage
inputs and radii); then the hand-written adjoint of each step runs in
reverse with the radii and dt held at their forward values.  Torch only
provides the device memory.
"""
from __future__ import annotations

import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, model, nsteps, every, cfl):
        assert U0.is_cuda and U0.dtype == torch.float64 and U0.is_contiguous()
        model.set_state(U0.detach())
        ckpts, dts, ts = [], [], []
        t = 0.0
        for k in range(nsteps):
            if k % every == 0:
                c = torch.empty_like(U0)
                model.get_state(c)
                ckpts.append((k, c, t))
            dt = model.step(cfl, want_dt=True)
            dts.append(dt)
            ts.append(t)
            t += dt
        out = torch.empty_like(U0)
        model.get_state(out)
        ctx.model, ctx.nsteps, ctx.every = model, nsteps, every
        ctx.ckpts, ctx.dts, ctx.ts = ckpts, dts, ts
        return out

    @staticmethod
    def backward(ctx, gout):
        model, every = ctx.model, ctx.every
        ny, nx = model.ny, model.nx
        dev = gout.device
        lam = gout.contiguous().clone()
        tmp = torch.empty_like(lam)
        tape = torch.empty((every, 3, 4, ny, nx), dtype=torch.float64, device=dev)
        otape = torch.empty((every, 3, ny, nx), dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        for k0, U, t0 in reversed(ctx.ckpts):
            k1 = min(k0 + every, ctx.nsteps)
            model.set_state(U)
            model.set_time(t0)
            for k in range(k0, k1):
                model.step_record(tape[k - k0].data_ptr(), otape[k - k0].data_ptr(),
                                  dt=ctx.dts[k])
            for k in reversed(range(k0, k1)):
                model.step_adjoint(tape[k - k0].data_ptr(), otape[k - k0].data_ptr(), ctx.dts[k],
                                   ctx.ts[k], lam.data_ptr(), tmp.data_ptr())
                lam, tmp = tmp, lam
        return lam, None, None, None, None


def rollout(U0, model, nsteps, every=20, cfl=None):
    """U_N of `nsteps` CFL steps from U0 (CUDA float64 (4, ny, nx)), differentiable."""
    return Rollout.apply(U0, model, nsteps, every, model.prob["cfl"] if cfl is None else cfl)
