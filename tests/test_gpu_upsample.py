"""Iterative upsampling (Sec. III.A): GPU prolongation against the oracle's, and the
upsampled solve reaching the same fixed point as a cold start in fewer sweeps."""
import functools
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np
import pytest

from oracle import soc
from tests._cases import problem_from_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _levels(fine=(32, 32, 64), levels=2):
    from paper_2502_08034_gb300 import synth
    return synth.multilevel_cases(fine, levels, 0.82, 4.0, 5, 0.01, -0.10, 0.5, 1e-10)


def test_prolongation_matches_oracle():
    from paper_2502_08034_gb300 import rfb
    coarse, fine = _levels()
    rng = np.random.default_rng(5)
    fl = coarse.solid.ravel() == 0
    sc = np.where(fl, rng.uniform(0.1, 0.9, coarse.n), 0.0)
    with rfb.Solver.from_case(coarse) as c, rfb.Solver.from_case(fine) as f:
        c.set_state(sc)
        c.step(coarse.s_in, coarse.eta, 0)
        f.upsample_from(c)
        got = f.get_state()
    ref = soc.prolong(sc, coarse.solid, fine.solid, coarse.s_in)
    assert np.abs(got - ref).max() < 1e-15
    # some fine fluid cells do sit under solid coarse parents
    parent_solid = coarse.solid.repeat(2, 0).repeat(2, 1).repeat(2, 2).astype(bool)
    assert np.any(parent_solid & (fine.solid == 0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_upsampled_solve_reaches_the_cold_start_fixed_point(precision):
    from paper_2502_08034_gb300 import rfb
    coarse, fine = _levels()
    tol = 1e-10
    with rfb.Solver.from_case(coarse) as c, rfb.Solver.from_case(fine) as f:
        rc = c.solve(coarse.s_in, coarse.eta, tol, precision=precision)
        f.upsample_from(c)
        s_up0 = f.get_state()
        ru = f.solve(fine.s_in, fine.eta, tol, precision=precision, check_every=10)
        s_up = f.get_state()
        f.reset_state()
        f.step(fine.s_in, fine.eta, 0)
        s_cold0 = f.get_state()
        f.reset_state()
        r0 = f.solve(fine.s_in, fine.eta, tol, precision=precision, check_every=10)
        s_cold = f.get_state()
    assert ru["residual"] <= tol and r0["residual"] <= tol
    assert np.abs(s_up - s_cold).max() < 1e-8
    ref = soc.steady_state(soc.assemble(problem_from_case(fine, soc)))
    assert np.abs(s_up - ref).max() < 1e-7
    # the prolonged coarse solution starts closer to the fixed point (its residual is
    # larger: injection leaves 2x2x2 blocks whose jumps the advective term sees) and needs
    # no more sweeps than a cold start
    fl = fine.solid.ravel() == 0
    e_up = np.sqrt(np.mean((s_up0 - ref)[fl] ** 2))
    e_cold = np.sqrt(np.mean((s_cold0 - ref)[fl] ** 2))
    assert e_up < e_cold, (e_up, e_cold)
    assert ru["sweeps"] <= r0["sweeps"], (ru["sweeps"], r0["sweeps"], rc["sweeps"])


def test_upsample_argument_checks():
    from paper_2502_08034_gb300 import rfb
    coarse, fine = _levels()
    with rfb.Solver.from_case(coarse) as c, rfb.Solver.from_case(fine) as f:
        with pytest.raises(rfb.RfbError) as e:
            f.upsample_from(c)            # coarse has no state yet
        assert e.value.status == rfb.RFB_ERR_STATE
        c.step(coarse.s_in, coarse.eta, 1)
        with pytest.raises(rfb.RfbError) as e:
            c.upsample_from(f)            # dims are not 2x
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG


def _oracle_slab_residual(case, s, k0, k1):
    """tau * RMS of the oracle's RHS(s) over planes [k0, k1) of a large lattice, from an
    oracle assembly of planes [k0 - 1, k1 + 1) (the rows of the inner planes are exact;
    the inlet / outlet planes are exact when the slab reaches them)."""
    nz, ny, nx = case.solid.shape
    a, b = max(0, k0 - 1), min(nz, k1 + 1)
    p = soc.Problem(np.ascontiguousarray(case.solid[a:b]), case.U[a:b], case.V[a:b],
                    case.W[a:b + 1], case.h, case.D, case.s_in, k0=case.k0, eta=case.eta)
    op = soc.assemble(p)
    sl = s.reshape(nz, ny, nx)[a:b].ravel()
    r = soc.rhs(op, sl).reshape(b - a, ny, nx)[k0 - a:k1 - a]
    fl = case.solid[k0:k1].ravel() == 0
    full = soc.assemble(problem_from_case(case, soc)) if case.n < 3_000_000 else None
    tau = full.tau if full is not None else None
    if tau is None:
        Q = case.h ** 2 * float(np.sum(np.where(case.solid[0] == 0, case.W[0], 0.0)))
        tau = int((case.solid == 0).sum()) * case.h ** 3 / Q
    return tau * float(np.sqrt(np.mean(r.ravel()[fl] ** 2)))


def test_upsampling_workload_512x512x1024_full_size():
    """The largest single-GPU run at full size: 128x128x256 -> 256x256x512 ->
    512x512x1024 (268M cells, porosity 0.82, d = 8 at the finest level), mixed precision
    to residual 1e-8 at each level. Checked by properties that hold at any size: the
    oracle's residual of the GPU state on inlet, middle and outlet slabs, the mass
    balance, the maximum principle and U <= U_mt."""
    from paper_2502_08034_gb300 import rfb, synth
    from paper_2502_08034_gb300.workflows import upsample_chain
    cases = synth.upsampling_cases(flow_device="cuda")
    solvers = [rfb.Solver.from_case(c, device_inputs=True) for c in cases]
    try:
        levels, _ = upsample_chain(solvers, cases, 1e-8, umt=False)
        fine, case = solvers[-1], cases[-1]
        s = fine.get_state()
        r = levels[-1]
        u_mt, _ = fine.umt(1e-8, precision="mixed")
    finally:
        for sv in solvers:
            sv.close()
    assert all(x["residual"] <= 1e-8 for x in levels)
    assert r["mass_balance_rel"] < 1e-5
    fl = case.solid.ravel() == 0
    kin = soc.kinetics(case.eta)
    assert s[fl].min() >= min(case.s_in, kin.s_eq) - 1e-6
    assert s[fl].max() <= max(case.s_in, kin.s_eq) + 1e-6
    assert 0.0 <= r["U"] <= u_mt <= 1.0
    nz = case.dims[2]
    for k0, k1 in ((0, 8), (nz // 2 - 4, nz // 2 + 4), (nz - 8, nz)):
        assert _oracle_slab_residual(case, s, k0, k1) < 1e-6, (k0, k1)
