"""torch.autograd.Function around the hand-written discrete adjoint.

``WenoThetaEuler1D.apply(u0, ...)`` advances nprob independent 1D Euler problems
(``u0``: CUDA float64 tensor ``[nprob, 3, n]``) by ``n_steps`` TVD-RK3 steps with the
WENO-theta scheme; its backward pass calls ``weno_theta_adjoint`` (reverse mode of the exact
map, branches frozen as the forward took them, checkpoints every ``checkpoint_every`` steps).
Both directions run in the CUDA library; this module only allocates workspaces and marshals.
"""
from __future__ import annotations

import torch

from . import binding as B


def _problem(bc, alpha_R, mode, gamma):
    return B.problem(B.WT_FLUX_EULER1D, bc=bc, alpha_R=alpha_R, mode=mode, gamma=gamma)


class WenoThetaEuler1D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, lo, hi, cfl, n_steps, checkpoint_every=32, bc=B.WT_BC_OUTFLOW, alpha_R=50.0,
                mode=B.WT_MODE_FAST, gamma=1.4):
        if u0.dtype != torch.float64 or not u0.is_cuda or u0.dim() != 3 or u0.shape[1] != 3:
            raise ValueError("u0 must be a CUDA float64 tensor of shape [nprob, 3, n]")
        u0 = u0.contiguous()
        nprob, _, n = u0.shape
        prob = _problem(bc, alpha_R, mode, gamma)
        grid = B.grid_1d(n, lo, hi)
        segs = []
        for p in range(nprob):
            s = B.WtSegment()
            s.offset, s.n, s.lo, s.hi, s.bc_lo, s.bc_hi = p * n, n, lo, hi, bc, bc
            segs.append(s)
        packed = u0.permute(1, 0, 2).reshape(3, nprob * n).contiguous()
        ws = B.alloc_workspace(B.workspace_bytes(prob, None, nprob * n, nprob), u0.device)
        B.weno_theta_step_batched(prob, segs, packed, nprob * n, cfl, n_steps, ws)
        uT = packed.reshape(3, nprob, n).permute(1, 0, 2).contiguous()
        ctx.save_for_backward(u0)
        ctx.args = (prob, grid, nprob, cfl, n_steps, checkpoint_every)
        return uT

    @staticmethod
    def backward(ctx, gT):
        (u0,) = ctx.saved_tensors
        prob, grid, nprob, cfl, n_steps, K = ctx.args
        ws = B.alloc_workspace(B.adjoint_workspace_bytes(prob, grid, nprob, n_steps, K), u0.device)
        g0 = torch.empty_like(u0)
        B.weno_theta_adjoint(prob, grid, nprob, u0, cfl, n_steps, K, gT.contiguous(), g0, ws)
        return g0, None, None, None, None, None, None, None, None, None
