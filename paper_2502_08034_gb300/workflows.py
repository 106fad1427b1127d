"""Multi-call workflows over the C ABI, shared by the benchmark and the tests.

upsample_chain: iterative upsampling (Sec. III.A), coarsest level first.
reduce_over_ranks: replica bookkeeping when one process runs per GPU (no collective on
the data path; the timed region is the maximum over ranks, the work is summed).
"""
from __future__ import annotations


def upsample_chain(solvers, cases, tol, umt=True, precision="mixed"):
    """Solve the coarsest level cold, then prolong (rfb_soc_upsample) and solve each
    finer level warm; returns (per-level results, U_mt of the finest level or None)."""
    out = []
    for q, (sv, c) in enumerate(zip(solvers, cases)):
        if q == 0:
            sv.reset_state()
        else:
            sv.upsample_from(solvers[q - 1])
        out.append(sv.solve(c.s_in, c.eta, tol, precision=precision))
    u = solvers[-1].umt(tol, precision=precision) if umt else None
    return out, u


def reduce_over_ranks(dist, elapsed_ms, units, device="cpu"):
    """Max of the timed region and sum of the work units over ranks (replicas); with
    dist None (one process) the inputs are returned as floats."""
    import torch
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
