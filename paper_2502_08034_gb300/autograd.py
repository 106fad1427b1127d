"""torch.autograd bridge: the steady state as a differentiable function of the per-voxel
reactive-area multiplier field and the velocity scale.

Forward runs the steady-state solve and the U_mt solve in the CUDA library; backward runs
its discrete adjoint (``rfb_soc_adjoint``), one adjoint solve per objective whose incoming
gradient is nonzero. ``precision`` ("fp64" or "mixed") selects both. Only the converged
states are kept (in the solver handle), so no activation checkpointing is involved; for
the same reason a backward must come before any other call that changes the solver's
states, which it checks.
"""
from __future__ import annotations

import torch

from . import rfb


class SocObjective(torch.autograd.Function):
    """(area_mult [N], beta []) -> (I_tot [A], U, U_mt).

    ``solver`` is an ``rfb.Solver``; ``s_in``/``eta`` the operating point; ``tol`` the
    residual tolerance of the forward solves and the relative tolerance of the adjoint
    solves; ``precision`` "fp64" or "mixed" (FP32 sweeps with FP64-confirmed defects, for
    the solves and the adjoints). dU_mt/d(area_mult) is identically zero (U_mt has no
    kinetics)."""

    @staticmethod
    def forward(ctx, area_mult, beta, solver, s_in, eta, tol, precision="fp64"):
        solver.set_area_mult(area_mult.detach().to(torch.float64).contiguous())
        b = float(beta)
        r = solver.solve(s_in, eta, tol, precision=precision, velocity_scale=b)
        u_mt, _ = solver.umt(tol, precision=precision, velocity_scale=b)
        ctx.solver = solver
        ctx.generation = solver.state_generation
        ctx.tol = tol
        ctx.precision = precision
        ctx.device = area_mult.device
        ctx.n = area_mult.numel()
        ctx.shape = area_mult.shape
        dev = area_mult.device
        f = lambda x: torch.tensor(x, dtype=torch.float64, device=dev)
        return f(r["I_tot"]), f(r["U"]), f(u_mt)

    @staticmethod
    def backward(ctx, g_i, g_u, g_umt):
        sv = ctx.solver
        if sv.state_generation != ctx.generation:
            # the adjoint differentiates the handle's current states, which are no longer
            # the ones this forward computed
            raise RuntimeError(
                "the solver was used again after this forward (a solve, U_mt solve, state or "
                "area-multiplier change, upsampling or batch solve): its adjoint would "
                "differentiate that later state; run the forward again before backward")
        grad_m = torch.zeros(ctx.n, dtype=torch.float64, device=ctx.device)
        grad_b = 0.0
        for g, obj in ((g_i, "I_tot"), (g_u, "U"), (g_umt, "U_mt")):
            if g is None:
                continue
            gv = float(g)
            if gv == 0.0:
                continue
            out = torch.empty(ctx.n, dtype=torch.float64, device=ctx.device) \
                if ctx.device.type == "cuda" else None
            dm, db, _ = sv.adjoint(obj, ctx.tol, out=out, precision=ctx.precision)
            dm_t = dm if isinstance(dm, torch.Tensor) else torch.from_numpy(dm).to(ctx.device)
            grad_m += gv * dm_t
            grad_b += gv * db
        grad_beta = torch.tensor(grad_b, dtype=torch.float64, device=ctx.device)
        return grad_m.reshape(ctx.shape), grad_beta, None, None, None, None, None


def soc_objective(solver: "rfb.Solver", area_mult: torch.Tensor, beta: torch.Tensor,
                  s_in: float, eta: float, tol: float = 1e-12, precision: str = "fp64"):
    """Differentiable (I_tot, U, U_mt) of the steady state."""
    return SocObjective.apply(area_mult, beta, solver, s_in, eta, tol, precision)
