"""Write the oracle's results on the full-size workloads to tests/golden/fullsize_*.npz.

Calls only the CPU oracle (oracle/soc.py) and the seeded input generator
(paper_2502_08034_gb300/synth.py, with its host potential-flow solver); nothing here
runs the CUDA solver. The GPU parity tests (tests/test_gpu_fullsize_golden.py) rebuild
the same inputs on the GPU and compare their results with these files.

Workloads (the inputs of the benchmark and of the full-size tests):
  mixed256   256x256x512, porosity 0.85, d ~ U[6, 10], 0.5 cm/s, eta = -0.05 V,
             s_in = 0.3 (the benchmark lattice)
  adjoint128 128x128x256, porosity 0.8, d = 8, 1 cm/s, eta = -0.10 V, s_in = 0.5, with
             lognormal area multipliers (sigma 0.3, seed 40): steady state, U_mt, and
             the gradients of I_tot, U and U_mt (adjoint, Sec. II / the paper's
             sensitivity question)
  upsample256 the 256x256x512 level (h = 2.5 um) of the upsampling workload
             (porosity 0.82, d = 8 at 512x512x1024, seed 5, 1 cm/s, eta = -0.10 V,
             s_in = 0.5)

Each file holds, besides the operating point:
  - flow checks: superficial velocity, W on 4096 sampled fluid z-faces and U / V on
    2048 sampled x / y faces (the test first checks that its GPU-built flow agrees);
  - the steady state s (Algorithm 7's explicit loop with local steps, to residual
    <= 1e-13, or <= 1e-12 where FP64 rounding stops the loop first) at 100,000 seeded
    fluid cells plus every
    fluid cell of the inlet and outlet planes, and the outputs (Sec. II.C);
  - U_mt (Eq. umt-def) from the same loop on the U_mt operator (benchmark and
    differentiation lattices);
  - for adjoint128: dI/dm at the 64 finite-difference voxels (seed 41) and at 20,000
    sampled wall cells, d/dbeta of I_tot, U and U_mt (the oracle's explicit transposed
    iteration to a relative residual of 1e-13).

Usage: python tests/golden/make_fullsize.py [mixed256|adjoint128|upsample256 ...]
(about 1-2 hours of CPU per 33.5M-cell workload; the flow uses every core).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import soc  # noqa: E402
from paper_2502_08034_gb300 import synth  # noqa: E402

N_SAMPLE = 100_000
TOL = 1e-13          # target residual of the oracle's steady states
TOL_ACCEPT = 1e-12   # accepted if the FP64 rounding floor stops the loop above TOL
MAX_SWEEPS = 40_000


def out_path(name):
    return os.path.join(HERE, "fullsize_%s.npz" % name)


def build_case(name):
    if name == "mixed256":
        return synth.large_mixed_case(flow_device="cpu"), None
    if name == "adjoint128":
        case = synth.adjoint_case(flow_device="cpu")
        return case, synth.lognormal_area_mult(case.solid, 0.3, 40)
    if name == "upsample256":
        return synth.upsampling_cases(flow_device="cpu", only_level=1)[0], None
    raise ValueError(name)


def sample_cells(case):
    """100,000 seeded fluid cells plus every fluid cell of the inlet and outlet planes."""
    fl = np.flatnonzero(case.solid.ravel() == 0)
    rng = np.random.default_rng(20250208)
    pick = rng.choice(fl, min(N_SAMPLE, fl.size), replace=False)
    nxny = case.dims[0] * case.dims[1]
    planes = fl[(fl < nxny) | (fl >= case.n - nxny)]
    return np.unique(np.concatenate([pick, planes])).astype(np.int32)


def flow_samples(case):
    rng = np.random.default_rng(7)
    W = case.W
    wf = np.flatnonzero(W.ravel() != 0)
    wi = np.sort(rng.choice(wf, 4096, replace=False))
    uf = np.flatnonzero(case.U.ravel() != 0)
    ui = np.sort(rng.choice(uf, 2048, replace=False))
    vf = np.flatnonzero(case.V.ravel() != 0)
    vi = np.sort(rng.choice(vf, 2048, replace=False))
    return dict(flow_q=float(case.info["superficial_q"]), flow_W_idx=wi,
                flow_W=W.ravel()[wi], flow_U_idx=ui, flow_U=case.U.ravel()[ui],
                flow_V_idx=vi, flow_V=case.V.ravel()[vi])


def problem(case, m=None, **over):
    kw = dict(solid=case.solid, U=case.U, V=case.V, W=case.W, h=case.h, D=case.D,
              s_in=case.s_in, k0=case.k0, alpha=case.alpha, n_e=case.n_e, T=case.T,
              c0=case.c0, eta=case.eta, area_mult=m)
    kw.update(over)
    return soc.Problem(**kw)


def solve(op, s_in, direct):
    """Steady state to residual <= TOL: the sparse solve (direct), else Algorithm 7's
    explicit loop with local steps from the cold start s = s_in, run in stretches of 500
    sweeps (the loop keeps nothing but the state between them) so that progress is
    logged and a stall at the FP64 rounding floor ends it: the loop stops once the
    residual is <= TOL, or <= TOL_ACCEPT and no longer halving over 2000 sweeps."""
    t = time.time()
    if direct:
        s = soc.steady_state(op)
        n = 0
    else:
        s = soc.initial_state(op, s_in)
        n, hist = 0, []
        while n < MAX_SWEEPS:
            s, k = soc.explicit_iterate(op, 0.4, TOL, s0=s, check_every=100, local_dt=True,
                                        max_steps=500)
            n += k
            r = soc.residual(op, s)
            hist.append(r)
            print("    %d sweeps: residual %.3e (%.0f s)" % (n, r, time.time() - t), flush=True)
            if r <= TOL or (r <= TOL_ACCEPT and len(hist) > 4 and r > 0.5 * hist[-5]):
                break
    r = soc.residual(op, s)
    print("  solve: %d sweeps, residual %.3e, %.0f s" % (n, r, time.time() - t), flush=True)
    assert r <= TOL_ACCEPT, r
    return s, n, r


def make(name):
    t0 = time.time()
    case, m = build_case(name)
    print("%s: %s, porosity %.4f, flow %s (%.0f s)" % (name, case.dims, case.porosity,
                                                      case.info, time.time() - t0), flush=True)
    direct = case.n <= 40_000
    p = problem(case, m)
    op = soc.assemble(p)
    s, sweeps, res = solve(op, case.s_in, direct)
    o = soc.outputs(p, op, s)
    idx = sample_cells(case)
    rec = dict(name=name, dims=np.array(case.dims), h=case.h, s_in=case.s_in, eta=case.eta,
               k0=case.k0, u_mean=case.u_mean, n_fluid=int((case.solid == 0).sum()),
               idx=idx, s=s[idx], sweeps=sweeps, residual=res, tau=op.tau,
               I_tot=o.I_tot, F_in=o.F_in, F_out=o.F_out, F_in_adv=o.F_in_adv, U=o.U,
               mass_balance_rel=o.mass_balance_rel, **flow_samples(case))
    del op
    sm = None
    if name != "upsample256":   # U_mt at full size: the benchmark and differentiation lattices
        # U_mt (Eq. umt-def): reaction off, s_in = 0, electrode cells held at 1
        opm = soc.assemble(p, mode="umt")
        sm, _, _ = solve(opm, 0.0, direct)
        rec["U_mt"] = soc.umt(p, sm)
        del opm
    if name == "adjoint128":
        fl = case.solid.ravel() == 0
        nw = soc.n_wall(case.solid.astype(bool)).ravel()
        rng = np.random.default_rng(41)   # the finite-difference voxels of the GPU test
        vox = rng.choice(np.flatnonzero(fl & (nw > 0)), 64, replace=False)
        wall = np.flatnonzero(fl & (nw > 0))
        wsel = np.unique(np.concatenate([
            np.random.default_rng(43).choice(wall, 20000, replace=False), vox]))
        for obj, sobj in (("I_tot", s), ("U", s), ("U_mt", sm)):
            t = time.time()
            a = soc.adjoint(p, sobj, obj)
            print("  adjoint %s: %.0f s" % (obj, time.time() - t), flush=True)
            rec["dm_%s" % obj] = a["d_area_mult"][wsel]
            rec["dbeta_%s" % obj] = a["d_beta"]
        rec["fd_voxels"] = vox
        rec["grad_idx"] = wsel
    np.savez_compressed(out_path(name), **rec)
    print("%s written (%.0f s): I_tot %.6e U %.6e U_mt %s" % (
        out_path(name), time.time() - t0, o.I_tot, o.U, rec.get("U_mt")), flush=True)


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["adjoint128", "mixed256", "upsample256"]:
        make(nm)
