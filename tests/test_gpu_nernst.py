"""Nernst model on the GPU (Sec. II.D, Algorithm 8): its steady state is the SBV one, so
states, outputs and the overpotential field are compared with the oracle's direct SBV
solution and with the oracle's own Nernst iteration; plus warm starts and refusals."""
import dataclasses
import functools

import numpy as np
import pytest

from oracle import soc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0_PAPER = 7.2e-5   # the paper's rate constant (parameter table), fast kinetics


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _case(dims=(16, 16, 32), k0=K0_PAPER):
    from paper_2502_08034_gb300 import synth
    c = synth.build_case("nernst%dx%dx%d" % dims, dims, 0.80, 4.0, 11, 0.01, -0.10, 0.5, 1e-12)
    return dataclasses.replace(c, k0=k0)


def _problem(case, **over):
    kw = dict(k0=case.k0, eta=case.eta, alpha=case.alpha)
    kw.update(over)
    return soc.Problem(case.solid, case.U, case.V, case.W, case.h, case.D, case.s_in, **kw)


@functools.lru_cache(maxsize=None)
def _oracle(dims, k0=K0_PAPER):
    p = _problem(_case(dims, k0))
    op = soc.assemble(p)
    return p, op, soc.steady_state(op)


@pytest.mark.parametrize("dims", [(16, 16, 32), (24, 20, 37)])
@pytest.mark.parametrize("dt_mode", ["local", "global"])
def test_nernst_state_is_the_sbv_steady_state(dims, dt_mode):
    from paper_2502_08034_gb300 import rfb
    case = _case(dims)
    p, op, ref = _oracle(dims)
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve_nernst(case.s_in, case.eta, 1e-13, omega=1.0, dt_mode=dt_mode,
                            max_sweeps=2_000_000)
        s = sv.get_state()
        eta_t = sv.get_overpotential()
    assert r["residual"] <= 1e-13
    assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max()
    elec = op.unknown & (op.kappa > 0)
    kin = op.kin
    assert np.abs(eta_t[elec] - (kin.Vt - np.log(ref[elec] / (1 - ref[elec])))).max() < 1e-7
    assert np.all(eta_t[~elec] == 0.0)
    o = soc.outputs(p, op, ref)
    assert abs(r["I_tot"] - o.I_tot) <= 1e-10 * abs(o.I_tot)


def test_nernst_matches_the_oracle_iteration():
    """omega = 0.5: the GPU and the oracle's Nernst loops reach the same state."""
    from paper_2502_08034_gb300 import rfb
    case = _case()
    p, _, _ = _oracle((16, 16, 32))
    s_o, eta_o, _ = soc.nernst_iterate(p, 0.5, 1e-12)
    with rfb.Solver.from_case(case) as sv:
        sv.solve_nernst(case.s_in, case.eta, 1e-12, omega=0.5)
        s = sv.get_state()
        eta_t = sv.get_overpotential()
    assert np.abs(s - s_o).max() <= 1e-9
    assert np.abs(eta_t - eta_o).max() <= 1e-6


def test_nernst_slow_kinetics_workload_matches_the_fp64_solve():
    """The 48x48x96 plain FP64 workload (k0 = 1e-7): Nernst and SBV give the same state."""
    from paper_2502_08034_gb300 import rfb, synth
    case = synth.fiber_channel_case()
    with rfb.Solver.from_case(case) as sv:
        sv.solve(case.s_in, case.eta, 1e-11, precision="fp64")
        ref = sv.get_state()
        sv.reset_state()
        r = sv.solve_nernst(case.s_in, case.eta, 1e-11, omega=1.0)
        s = sv.get_state()
    assert r["residual"] <= 1e-11
    assert np.abs(s - ref).max() <= 1e-9 * np.abs(ref).max()


def test_warm_start_and_adjoint_after_nernst():
    from paper_2502_08034_gb300 import rfb
    case = _case()
    with rfb.Solver.from_case(case) as sv:
        sv.solve(case.s_in, case.eta, 1e-13, precision="fp64")
        r = sv.solve_nernst(case.s_in, case.eta, 1e-12)
        assert r["sweeps"] == 0 and r["residual"] <= 1e-12
        eta_t = sv.get_overpotential()
        assert np.isfinite(eta_t).all() and np.abs(eta_t).max() > 0
        dm, db, ra = sv.adjoint("I_tot", 1e-11)
        assert ra["residual"] <= 1e-11 and np.isfinite(dm).all()
        sv.reset_state()
        with pytest.raises(rfb.RfbError) as e:
            sv.get_overpotential()
        assert e.value.status == rfb.RFB_ERR_STATE


def test_nernst_refused_options():
    from paper_2502_08034_gb300 import rfb
    case = _case()
    with rfb.Solver.from_case(case) as sv:
        for kw in (dict(omega=0.0), dict(omega=1.5), dict(precision="mixed")):
            with pytest.raises(rfb.RfbError) as e:
                sv.solve_nernst(case.s_in, case.eta, 1e-8, **kw)
            assert e.value.status == rfb.RFB_ERR_INVALID_ARG
    for c, kmode in ((dataclasses.replace(case, alpha=0.3), 0), (case, 1),
                     (dataclasses.replace(case, k0=0.0), 0)):
        with rfb.Solver.from_case(c, kinetics_mode=kmode) as sv:
            with pytest.raises(rfb.RfbError) as e:
                sv.solve_nernst(c.s_in, c.eta, 1e-8)
            assert e.value.status == rfb.RFB_ERR_INVALID_ARG
