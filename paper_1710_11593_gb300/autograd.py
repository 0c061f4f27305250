"""torch.autograd wrapper: gradients of the solve with respect to the source f and the
fractional order gamma.

Forward: u = A(gamma)^-1 f through ftoep_solve.  Backward: the adjoint field
lam = A^-T dL/du (ftoep_adjoint: a time-reversed solve of the same Toeplitz systems) gives
dL/df = lam and dL/dgamma = -<lam, (dA/dgamma) u>, where dA/dgamma is the derivative of
the scheme's weights (the spatial operator does not depend on gamma).  Zero initial data.

Checkpointing: ``recompute=False`` keeps u for the backward pass (one field of memory);
``recompute=True`` keeps only f and re-solves for u in the backward pass.

Plans: a plan (weights, spectra, block inverses, workspace) is built once per problem
(kind, gamma, N, M, space, precision, T, L, lam) and kept in a small least-recently-used
cache, so repeated forward passes of one problem reuse it; the autograd graph holds a
reference to its plan, so backward may run more than once (``retain_graph=True``) and a
plan evicted from the cache stays alive until its last graph is freed.
``clear_plan_cache()`` releases the cached plans.
"""
from __future__ import annotations

from collections import OrderedDict
from typing import Optional

import torch

from . import ftoep

_CACHE_SIZE = 2
_plans: "OrderedDict[tuple, ftoep.Plan]" = OrderedDict()


def _plan_for(spec: ftoep.ProblemSpec) -> ftoep.Plan:
    key = (spec.kind, spec.gamma, spec.N, spec.M, spec.space, spec.precision, spec.T, spec.L, spec.lam)
    plan = _plans.get(key)
    if plan is not None:
        _plans.move_to_end(key)
        return plan
    plan = ftoep.Plan([spec])
    _plans[key] = plan
    while len(_plans) > _CACHE_SIZE:
        _plans.popitem(last=False)  # closed when its last reference goes
    return plan


def clear_plan_cache() -> None:
    """Drop the cached plans (each is closed once no autograd graph refers to it)."""
    _plans.clear()


class FractionalSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, gamma: torch.Tensor, kind: Optional[int] = None, space: int = 1,
                precision: int = ftoep.FP64, T: float = 1.0, L: float = 1.0, lam: float = 1.0,
                recompute: bool = False):
        g = float(gamma.detach().cpu())
        if kind is None:
            kind = ftoep.L1_SUBDIFFUSION if g < 1.0 else ftoep.L1_HYPERBOLIC
        M, N = (1, f.shape[0]) if f.dim() == 1 else (f.shape[0], f.shape[1])
        spec = ftoep.ProblemSpec(kind, g, N, M, space, precision, T, L, lam)
        plan = _plan_for(spec)
        fc = f.detach().contiguous()
        u = plan.solve(fc)
        ctx.plan = plan
        ctx.recompute = recompute
        ctx.gamma_meta = (gamma.dtype, gamma.device)
        if recompute:
            ctx.save_for_backward(fc)
        else:
            ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        (saved,) = ctx.saved_tensors
        plan = ctx.plan
        u = plan.solve(saved) if ctx.recompute else saved
        need_gamma = ctx.needs_input_grad[1]
        dldf, dg = plan.adjoint(grad_u.contiguous(), u, want_gamma=need_gamma)
        dtype, device = ctx.gamma_meta
        dgamma = torch.tensor(float(dg[0]), dtype=dtype, device=device) if need_gamma else None
        return dldf, dgamma, None, None, None, None, None, None, None


def fractional_solve(f: torch.Tensor, gamma: torch.Tensor, **kw) -> torch.Tensor:
    """u = solve(f; gamma), differentiable in f and gamma (see FractionalSolve)."""
    return FractionalSolve.apply(f, gamma, kw.get("kind"), kw.get("space", 1), kw.get("precision", ftoep.FP64),
                                 kw.get("T", 1.0), kw.get("L", 1.0), kw.get("lam", 1.0), kw.get("recompute", False))
