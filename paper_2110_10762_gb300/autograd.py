"""torch.autograd.Function over the discrete Parareal adjoint.

ParaRealFn.apply(u0, kappa, spec) returns lambda_N^K, the final-time state
after K synchronous Parareal iterations (Algorithm 1, Eq. (11), no early
stop); its backward calls parareal_adjoint, so gradients of any loss of
lambda_N with respect to the initial state u0 and the node diffusivity kappa
come from the hand-written reverse sweep in libparareal (no autograd tape).

spec: dict with dim, n (x, y, z sizes), T (end time, T0 = 0), N (slices),
f_steps, K (iterations), g_rtol (coarse CG tolerance; default 1e-13), and
optionally f_scheme ("explicit", default, or "implicit" for 1D implicit fine
steps) and g_solver ("cg", default, or "thomas" in 1D).
"""
from __future__ import annotations

import torch

from . import api


def _problem(spec, u0, kappa, K):
    from ._abi import PR_EXPLICIT_EULER, PR_IMPLICIT_EULER, PR_SOLVER_CG, PR_SOLVER_THOMAS
    f_scheme = PR_IMPLICIT_EULER if spec.get("f_scheme") == "implicit" else PR_EXPLICIT_EULER
    g_solver = PR_SOLVER_THOMAS if spec.get("g_solver") == "thomas" else PR_SOLVER_CG
    return api.make_problem(dim=spec["dim"], n=spec["n"], T0=0.0, T=spec["T"], N=spec["N"],
                            u0=u0, kappa=kappa, f_scheme=f_scheme, f_steps=spec["f_steps"],
                            f_prec=64, g_solver=g_solver, g_rtol=spec.get("g_rtol", 1e-13),
                            tol=0.0, max_iter=K)


class ParaRealFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0: torch.Tensor, kappa: torch.Tensor | None, spec: dict):
        u0c = u0.detach().contiguous()
        kc = kappa.detach().contiguous() if kappa is not None else None
        K = int(spec["K"])
        M = u0c.numel()
        handle = api.parareal_create(u0c.device.index or 0, torch.cuda.current_stream(u0c.device))
        try:
            api.parareal_set_problem(handle, _problem(spec, u0c, kc, K))
            lam = torch.empty((spec["N"] + 1) * M, dtype=torch.float64, device=u0c.device)
            api.parareal_run_sync(handle, lam)
        finally:
            api.parareal_destroy(handle)
        ctx.save_for_backward(u0c, kc if kc is not None else torch.empty(0, device=u0c.device))
        ctx.has_kappa = kc is not None
        ctx.spec = dict(spec)
        return lam[spec["N"] * M:].clone()

    @staticmethod
    def backward(ctx, grad_lamN: torch.Tensor):
        u0c, kc = ctx.saved_tensors
        kc = kc if ctx.has_kappa else None
        spec = ctx.spec
        K = int(spec["K"])
        g = grad_lamN.detach().to(torch.float64).contiguous()
        handle = api.parareal_create(u0c.device.index or 0, torch.cuda.current_stream(u0c.device))
        try:
            api.parareal_set_problem(handle, _problem(spec, u0c, kc, K))
            gu0 = torch.empty_like(u0c)
            gk = torch.empty_like(kc) if kc is not None else None
            api.parareal_adjoint(handle, g, K, gu0, gk)
        finally:
            api.parareal_destroy(handle)
        return gu0, gk, None


def parareal_final_state(u0: torch.Tensor, kappa: torch.Tensor | None, spec: dict) -> torch.Tensor:
    """lambda_N^K as a differentiable function of (u0, kappa)."""
    return ParaRealFn.apply(u0, kappa, spec)
