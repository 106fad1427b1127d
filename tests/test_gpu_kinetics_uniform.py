"""Kinetics mode 1 (Butler-Volmer source at a uniform activation overpotential,
Eq. source-term-bv-gen) on the GPU: FP64 states, outputs and adjoints against the
oracle's Newton solution of the nonlinear steady problem, and the options it refuses."""
import dataclasses
import functools

import numpy as np
import pytest

from oracle import soc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _case(dims=(16, 16, 32), k0=2e-6, s_in=0.3, eta=-0.10, seed=11):
    from paper_2502_08034_gb300 import synth
    c = synth.build_case("kin1_%dx%dx%d" % dims, dims, 0.80, 4.0, seed, 0.01, eta, s_in, 1e-12)
    return dataclasses.replace(c, k0=k0)


def _problem(case, **over):
    kw = dict(k0=case.k0, eta=case.eta, alpha=case.alpha, kinetics_mode=1)
    kw.update(over)
    return soc.Problem(case.solid, case.U, case.V, case.W, case.h, case.D, case.s_in, **kw)


@functools.lru_cache(maxsize=None)
def _oracle(dims, inlet_bc="face", with_m=False, alpha=0.5):
    case = _case(dims)
    m = None
    if with_m:
        from paper_2502_08034_gb300 import synth
        m = synth.lognormal_area_mult(case.solid, 0.3, 40)
    p = _problem(case, inlet_bc=inlet_bc, area_mult=m, alpha=alpha)
    op = soc.assemble(p)
    s = soc.steady_state(op)
    return p, op, s, m


@pytest.mark.parametrize("dims", [(16, 16, 32), (24, 20, 37)])
@pytest.mark.parametrize("dt_mode", ["local", "global"])
def test_fp64_state_matches_oracle_newton(dims, dt_mode):
    from paper_2502_08034_gb300 import rfb
    case = _case(dims)
    p, op, ref, _ = _oracle(dims)
    with rfb.Solver.from_case(case, kinetics_mode=rfb.KIN_UNIFORM_ETA) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-13, precision="fp64", dt_mode=dt_mode,
                     max_sweeps=5_000_000)
        s = sv.get_state()
    assert r["residual"] <= 1e-13
    assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max()
    fl = case.solid.ravel() == 0
    assert s[fl].max() < 1.0 and s[fl].min() >= case.s_in - 1e-12   # the clip never binds
    o = soc.outputs(p, op, ref)
    assert abs(r["I_tot"] - o.I_tot) <= 1e-10 * abs(o.I_tot)
    assert abs(r["F_out"] - o.F_out) <= 1e-10 * abs(o.F_out)
    assert r["mass_balance_rel"] < 1e-9


def test_ghost_inlet_area_multiplier_and_alpha():
    from paper_2502_08034_gb300 import rfb
    dims = (16, 16, 32)
    case = _case(dims)
    for inlet_bc, with_m, alpha in (("ghost", False, 0.5), ("face", True, 0.5),
                                    ("face", False, 0.3)):
        p, op, ref, m = _oracle(dims, inlet_bc, with_m, alpha)
        c2 = dataclasses.replace(case, alpha=alpha)
        with rfb.Solver.from_case(c2, area_mult=m, kinetics_mode=1) as sv:
            r = sv.solve(case.s_in, case.eta, 1e-13, precision="fp64", inlet_bc=inlet_bc,
                         max_sweeps=5_000_000)
            s = sv.get_state()
        assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max(), (inlet_bc, with_m, alpha)
        assert abs(r["I_tot"] - soc.outputs(p, op, ref).I_tot) <= 1e-10 * abs(r["I_tot"])


def test_outputs_on_an_arbitrary_state():
    """current() and current_noalloc() evaluate the mode-1 source on any state."""
    from paper_2502_08034_gb300 import rfb
    dims = (16, 16, 32)
    case = _case(dims)
    p, op, _, _ = _oracle(dims)
    rng = np.random.default_rng(5)
    s = np.where(case.solid.ravel() == 0, rng.uniform(0.05, 0.95, case.n), 0.0)
    with rfb.Solver.from_case(case, kinetics_mode=1) as sv:
        sv.step(case.s_in, case.eta, 0, precision="fp64")
        sv.set_state(s)
        a = sv.current()
        b = sv.current_noalloc()
    o = soc.outputs(p, op, s)
    for r in (a, b):
        assert abs(r["I_tot"] - o.I_tot) <= 1e-12 * abs(o.I_tot)
        assert abs(r["residual"] - o.residual) <= 1e-12 * o.residual


@pytest.mark.parametrize("objective", ["I_tot", "U"])
def test_adjoint_matches_oracle(objective):
    from paper_2502_08034_gb300 import rfb, synth
    dims = (16, 16, 32)
    case = _case(dims)
    m = synth.lognormal_area_mult(case.solid, 0.3, 40)
    p = _problem(case, area_mult=m)
    ref = soc.adjoint(p, None, objective)
    with rfb.Solver.from_case(case, area_mult=m, kinetics_mode=1) as sv:
        sv.solve(case.s_in, case.eta, 1e-14, precision="fp64", max_sweeps=5_000_000)
        dm, db, r = sv.adjoint(objective, 1e-13)
        # a second forward solve after the adjoint re-assembles the transport operator
        r2 = sv.solve(case.s_in, case.eta, 1e-14, precision="fp64", max_sweeps=5_000_000)
    scale = np.abs(ref["d_area_mult"]).max()
    assert np.abs(dm - ref["d_area_mult"]).max() <= 1e-9 * scale
    assert abs(db - ref["d_beta"]) <= 1e-9 * abs(ref["d_beta"])
    assert r["residual"] <= 1e-13
    assert r2["residual"] <= 1e-14 and r2["sweeps"] == 0


def test_refused_options_and_umt():
    from paper_2502_08034_gb300 import rfb
    case = _case((16, 16, 32))
    with rfb.Solver.from_case(case, kinetics_mode=1) as sv:
        with pytest.raises(rfb.RfbError) as e:
            sv.solve(case.s_in, case.eta, 1e-8, precision="mixed")
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
        with pytest.raises(rfb.RfbError) as e:
            rfb.Batch([sv])
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
        # U_mt has no kinetics: the same handle runs it in mixed precision
        u1, _ = sv.umt(1e-10, precision="mixed")
    with rfb.Solver.from_case(case) as sv0:
        u0, _ = sv0.umt(1e-10, precision="mixed")
    assert u1 == u0
    with pytest.raises(rfb.RfbError) as e:
        rfb.Solver.from_case(case, kinetics_mode=2)
    assert e.value.status == rfb.RFB_ERR_INVALID_ARG


def test_zero_inlet_state_is_the_trivial_fixed_point():
    """With s_in = 0 the rate s^alpha (1-s)^(1-alpha) vanishes on the cold start, which is
    then steady: the solve returns at once with s = 0."""
    from paper_2502_08034_gb300 import rfb
    case = _case((16, 16, 32))
    with rfb.Solver.from_case(case, kinetics_mode=1) as sv:
        r = sv.solve(0.0, case.eta, 1e-12, precision="fp64")
        s = sv.get_state()
    assert r["sweeps"] == 0 and r["residual"] == 0.0 and np.all(s == 0.0)
