"""torch.autograd wrappers over the library (argument marshalling only: every
derivative is computed by the library's kernels).

* Energy: per-replica energies of positions x; the hand-written backward is
  the library's force, dE/dx = -F (exact at the charge minimiser).
* ForceMatchingLoss: the force-matching loss of a fixed batch as a function
  of the 144 parameters (field order of ctbop_params); the backward is
  ctbop_param_grad (analytic parameter derivatives, charge response by an
  adjoint solve), in the system's precision policy (FP64, or FP32 terms with
  FP64 sums).
"""
import numpy as np
import torch

from . import ctbop


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, system):
        xd = x.detach().to(torch.float64).contiguous()
        system.set_positions(xd.cpu().numpy() if not xd.is_cuda else xd)
        system.compute()
        E = torch.as_tensor(system.get("energy"), dtype=x.dtype, device=x.device)
        F = torch.as_tensor(system.get("forces"), dtype=x.dtype, device=x.device)
        ctx.save_for_backward(F)
        ctx.rep = torch.as_tensor(system.replica_index(), device=x.device)
        return E

    @staticmethod
    def backward(ctx, gE):
        (F,) = ctx.saved_tensors
        return -(gE[ctx.rep][:, None] * F), None


class ForceMatchingLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, system, w_E=None, E_ref=None, w_F=None, F_ref=None):
        v = theta.detach().to(torch.float64).cpu().numpy()
        system.set_params_struct(ctbop.params_from_vector(v))
        loss, G = system.param_grad(w_E=w_E, E_ref=E_ref, w_F=w_F, F_ref=F_ref)
        ctx.save_for_backward(torch.as_tensor(ctbop.params_vector(G), dtype=theta.dtype, device=theta.device))
        return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, gL):
        (G,) = ctx.saved_tensors
        return gL * G, None, None, None, None, None
