"""The data misfit of Sec. 3 as a differentiable torch function.

``HelmholtzMisfit.apply(gamma, ctx)`` returns Phi(gamma) = 1/2 sum |W (d - Q u)|^2
with u the Helmholtz wavefields of every source and frequency (Sec. 2).  The
backward pass is the hand-written adjoint of the CUDA library: adjoint solves
A^H lambda = Q^T W^T W r and the reduction
dPhi/dgamma = -sum_b omega_b^2 Re(conj(u_b) lambda_b) (``fwi_gradient``).

Two memory strategies, as for checkpointed training:
  * ``save``      the forward pass runs forward + adjoint at once and keeps only
                  the gradient (nz*nx FP64) for backward;
  * ``recompute`` the forward pass runs the forward solve only (misfit); the
                  backward pass recomputes the wavefields, then runs the adjoint.
``auto`` picks ``recompute`` when the forward wavefields (complex128, all
blocks) exceed ``mem_budget_bytes``.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import FWI, Opts, default_opts


class HelmholtzMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, fwi: FWI, inst: int = 0, opts: Opts | None = None,
                mode: str = "auto", mem_budget_bytes: float = 8e9):
        if gamma.dim() != 2:
            raise ValueError("gamma must be [nz, nx]")
        fwi.set_model(inst, gamma.detach())
        lay = fwi.layout()
        if mode == "auto":
            mode = "recompute" if 16.0 * lay["field_elems"] > mem_budget_bytes else "save"
        ctx.fwi, ctx.inst, ctx.opts, ctx.mode = fwi, inst, opts, mode
        ctx.shape = gamma.shape
        ctx.gamma = gamma.detach()
        if mode == "save":
            mis, g, _ = fwi.gradient(opts)
            ctx.grad = _inst_slice(fwi, inst, g)
            val = mis[inst]
        elif mode == "recompute":
            _, mis, _ = fwi.forward(opts, want_data=False)
            val = mis[inst]
        else:
            raise ValueError(mode)
        return torch.tensor(val, dtype=torch.float64, device=gamma.device)

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.mode == "save":
            g = ctx.grad
        else:
            ctx.fwi.set_model(ctx.inst, ctx.gamma)          # wavefields are recomputed here
            _, gall, _ = ctx.fwi.gradient(ctx.opts)
            g = _inst_slice(ctx.fwi, ctx.inst, gall)
        gt = torch.from_numpy(np.ascontiguousarray(g.reshape(ctx.shape))).to(grad_out.device)
        return grad_out * gt, None, None, None, None, None


def _inst_slice(fwi: FWI, inst: int, g: np.ndarray) -> np.ndarray:
    off = 0
    for i, gr in enumerate(fwi.grids):
        n = gr.nx * gr.nz
        if i == inst:
            return g[off:off + n].copy()
        off += n
    raise IndexError(inst)


def misfit(gamma: torch.Tensor, fwi: FWI, inst: int = 0, opts: Opts | None = None, mode: str = "auto",
           mem_budget_bytes: float = 8e9) -> torch.Tensor:
    """Differentiable misfit of instance ``inst`` at model ``gamma`` ([nz, nx], FP64)."""
    return HelmholtzMisfit.apply(gamma, fwi, inst, opts if opts is not None else default_opts(), mode,
                                 mem_budget_bytes)
