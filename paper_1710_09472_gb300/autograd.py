"""torch.autograd.Function over the library's window totals and adjoint.

WindowCurrent.apply(E_field, B, tau, sim, t_begin, t_end, checkpoint_every)
returns the FP64 tensor [sum rho, sum j_x, sum j_y, sum j_z] summed over the
states after steps t_begin+1 .. t_end of a run that starts from the
simulation's current state, with E_field the per-cell field ([D, *shape],
float32, on the device), B (3,) and tau (scalar).  Its backward restores the
start state and calls lbm_adjoint with uniform loss weights taken from the
incoming gradient, returning dL/dE(x), dL/dB and dL/dtau.  PyTorch supplies
memory and the stream only; both directions run in the library's kernels.

Two effects of backward() that a caller should know:
  - the incoming FP64 gradient is passed to lbm_adjoint as FP32 per-cell loss
    weights (w_rho, w_j), so it is rounded to FP32 (relative 6e-8) before the
    reverse sweep; the sweep itself accumulates the parameter gradients in
    FP64;
  - the simulation is left at the restored start state (the state before
    forward() ran), not at step t_end: a caller that wants to step on from
    t_end after backward() must save that state after forward() and load it.
"""
from __future__ import annotations

import torch


class WindowCurrent(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E_field, B, tau, sim, t_begin: int, t_end: int, checkpoint_every: int = 0):
        if not E_field.is_cuda or E_field.dtype != torch.float32:
            raise TypeError("E_field must be a float32 CUDA tensor")
        ctx.sim = sim
        ctx.t = (int(t_begin), int(t_end), int(checkpoint_every))
        ctx.state = sim.save_state()
        ctx.shape = E_field.shape
        ctx.B_dtype = B.dtype if isinstance(B, torch.Tensor) else torch.float64
        ctx.B_dev = B.device if isinstance(B, torch.Tensor) else E_field.device
        ctx.tau_dev = tau.device if isinstance(tau, torch.Tensor) else E_field.device
        Bl = [float(x) for x in (B.tolist() if isinstance(B, torch.Tensor) else B)]
        tl = float(tau.item() if isinstance(tau, torch.Tensor) else tau)
        sim.set_E_field(E_field.detach().contiguous().view(-1))
        sim.set_params(tl, B=Bl)
        out = sim.window_totals(ctx.t[0], ctx.t[1])
        return torch.tensor(out, dtype=torch.float64, device=E_field.device)

    @staticmethod
    def backward(ctx, grad):
        sim = ctx.sim
        sim.load_state(ctx.state)
        g = grad.detach().double().cpu().tolist()
        dev = torch.device("cuda", torch.cuda.current_device())
        w_rho = torch.full((sim.N,), g[0], dtype=torch.float32, device=dev)
        w_j = torch.tensor(g[1: 1 + sim.D], dtype=torch.float32, device=dev).repeat_interleave(sim.N)
        dE = torch.empty(sim.D * sim.N, dtype=torch.float64, device=dev)
        res = sim.adjoint(ctx.t[0], ctx.t[1], w_rho, w_j, ctx.t[2], dL_dE=dE)
        gE = dE.view(ctx.shape).to(torch.float32)
        gB = torch.tensor(res["dL_dB"], dtype=ctx.B_dtype, device=ctx.B_dev)
        gtau = torch.tensor(res["dL_dtau"], dtype=torch.float64, device=ctx.tau_dev)
        return gE, gB, gtau, None, None, None, None
