"""The FWI objective as a differentiable torch function.

f(m) = sum_{w,s} 1/2 ||P_r H_w(m)^{-1} q_s - d_s||^2 (Sec. 2, eq. (mainprob)) with
its adjoint-state gradient (Appendix A) as the backward pass.  Every PDE solve,
misfit and gradient kernel runs in libhelm.so; this module only decides which
C-ABI calls run in forward and in backward (the forward-field policy):

  "eager"      forward = misfit_and_gradient (2 solves per pair), backward
               multiplies the saved gradient by the incoming scalar;
  "store"      forward = helm_misfit keeping the forward fields U and data
               residuals R (1 solve per pair), backward = helm_gradient
               (the adjoint solve per pair) -- memory nfreq*nsrc*n_comp*16 B;
  "store_c64"  the same with U rounded to complex64 (8 B per node and pair):
               f is unchanged (computed from the FP64 field), g carries the
               rounding of U, a relative perturbation of at most 2^-24 per
               part of each stored value (measured ~2e-8 relative in g);
  "recompute"  forward = helm_misfit (1 solve per pair, nothing kept),
               backward = misfit_and_gradient (forward solves repeated);
  "auto"       "store" when the complex128 fields fit the memory budget, else
               "store_c64" when the complex64 fields do, else "recompute".
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import helm


@dataclass
class FWIProblem:
    """Acquisition, data and solver plan of one objective (all tensors on the plan's device)."""
    plan: "helm.Plan"
    freqs_hz: np.ndarray
    src_idx: torch.Tensor
    Q: torch.Tensor
    rec_idx: torch.Tensor
    d_obs: torch.Tensor
    wavelet: Optional[torch.Tensor] = None
    mask: Optional[torch.Tensor] = None
    policy: str = "eager"
    store_budget_bytes: Optional[int] = None

    def field_bytes(self, bytes_per_value: int = 16) -> int:
        return int(len(np.atleast_1d(self.freqs_hz)) * self.Q.shape[1] * self.plan.n_comp * bytes_per_value)

    def resolve_policy(self) -> str:
        if self.policy in ("eager", "store", "store_c64", "recompute"):
            return self.policy
        if self.policy != "auto":
            raise ValueError(f"unknown policy {self.policy!r}")
        budget = self.store_budget_bytes
        if budget is None:
            free, _ = torch.cuda.mem_get_info(self.plan.device)
            budget = free // 2
        if self.field_bytes(16) <= budget:
            return "store"
        return "store_c64" if self.field_bytes(8) <= budget else "recompute"


class FWIObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, problem: FWIProblem):
        p = problem
        policy = p.resolve_policy()
        ctx.problem, ctx.policy = p, policy
        if policy == "eager":
            f, g, _ = helm.misfit_and_gradient(p.plan, m, p.freqs_hz, p.src_idx, p.Q, p.rec_idx, p.d_obs,
                                               wavelet=p.wavelet, mask=p.mask)
            ctx.save_for_backward(g)
        elif policy in ("store", "store_c64"):
            dt = torch.complex64 if policy == "store_c64" else torch.complex128
            f, R, U, _ = helm.helm_misfit(p.plan, m, p.freqs_hz, p.src_idx, p.Q, p.rec_idx, p.d_obs, wavelet=p.wavelet,
                                          mask=p.mask, keep_residuals=True, keep_fields=True, field_dtype=dt)
            ctx.save_for_backward(m, R, U)
        else:
            f, _, _, _ = helm.helm_misfit(p.plan, m, p.freqs_hz, p.src_idx, p.Q, p.rec_idx, p.d_obs,
                                          wavelet=p.wavelet, mask=p.mask)
            ctx.save_for_backward(m)
        return f.reshape(())

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        p = ctx.problem
        if ctx.policy == "eager":
            (g,) = ctx.saved_tensors
        elif ctx.policy in ("store", "store_c64"):
            m, R, U = ctx.saved_tensors
            g, _ = helm.helm_gradient(p.plan, m.detach().contiguous(), p.freqs_hz, p.rec_idx, R, U, mask=p.mask)
        else:
            (m,) = ctx.saved_tensors
            _, g, _ = helm.misfit_and_gradient(p.plan, m.detach().contiguous(), p.freqs_hz, p.src_idx, p.Q,
                                               p.rec_idx, p.d_obs, wavelet=p.wavelet, mask=p.mask)
        return grad_out * g.reshape(ctx.problem.plan.n_phys), None


def fwi_objective(m: torch.Tensor, problem: FWIProblem) -> torch.Tensor:
    """Differentiable f(m) for a physical model m (float64, [n_phys], on the plan's device)."""
    return FWIObjective.apply(m, problem)
