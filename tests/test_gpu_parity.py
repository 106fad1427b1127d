"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: FP64 mode 1e-10 relative in s and I_tot after both sides are converged far
below it (the oracle solves RHS = 0 directly); mixed mode 1e-6 max-abs in s; one
explicit FP64 sweep matches the oracle's s + dt (L s + b) to rounding (1e-14).
"""
import numpy as np
import pytest

from oracle import soc
from tests._cases import fiber_case, mixed_case_small, problem_from_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


def _solver(case, **kw):
    from paper_2502_08034_gb300 import rfb
    return rfb.Solver.from_case(case, **kw)


def _oracle(case, **over):
    p = problem_from_case(case, soc, **over)
    return p, soc.assemble(p)


# ------------------------------------------------------------------ one sweep, outputs

@pytest.mark.parametrize("dims", [(16, 16, 32), (37, 21, 19), (5, 7, 11)])
def test_one_fp64_sweep_matches_oracle(dims):
    case = fiber_case(dims, diameter=3.0 if min(dims) < 10 else 8.0)
    p, op = _oracle(case)
    rng = np.random.default_rng(7)
    fl = case.solid.ravel() == 0
    s0 = np.where(fl, rng.uniform(0.2, 0.9, case.n), 0.0)
    dt = soc.dt_global(op, 0.4)
    ref = s0 + dt * soc.rhs(op, s0)
    ref[~fl] = 0.0
    with _solver(case) as sv:
        sv.set_state(s0)
        sv.step(case.s_in, case.eta, 1, dt_mode="global")
        s1 = sv.get_state()
    assert np.abs(s1 - ref).max() < 1e-14


def test_outputs_match_oracle_on_arbitrary_state():
    case = fiber_case((16, 16, 32))
    p, op = _oracle(case)
    rng = np.random.default_rng(11)
    fl = case.solid.ravel() == 0
    s0 = np.where(fl, rng.uniform(0.0, 1.0, case.n), 0.0)
    o = soc.outputs(p, op, s0)
    with _solver(case) as sv:
        sv.set_state(s0)
        sv.step(case.s_in, case.eta, 0)
        r = sv.current()
    for k in ("I_tot", "F_in", "F_out", "F_in_adv"):
        assert abs(r[k] - getattr(o, k)) <= 1e-12 * abs(getattr(o, k)), k
    assert abs(r["residual"] - o.residual) <= 1e-12 * o.residual
    assert abs(r["U"] - o.U) <= 1e-12 * abs(o.U)


# ------------------------------------------------------------------ converged parity

@pytest.mark.parametrize("dt_mode", ["local", "global"])
def test_fp64_steady_state_parity_small(dt_mode):
    case = fiber_case((16, 16, 32))
    p, op = _oracle(case)
    s_ref = soc.steady_state(op)
    o = soc.outputs(p, op, s_ref)
    with _solver(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-13, dt_mode=dt_mode, precision="fp64")
        s = sv.get_state()
    assert r["residual"] <= 1e-13
    assert np.abs(s - s_ref).max() / np.abs(s_ref).max() < 1e-10
    assert abs(r["I_tot"] - o.I_tot) / abs(o.I_tot) < 1e-10
    assert r["mass_balance_rel"] < 1e-9


def test_fp64_parity_plain_fp64_workload_48x48x96():
    """The plain-FP64 workload (48x48x96, d = 8, porosity 0.80, 1 cm/s, -0.10 V,
    s_in = 0.5, CFL 0.4) at full size: parity at 1e-10 relative."""
    case = fiber_case((48, 48, 96))
    p, op = _oracle(case)
    s_ref = soc.steady_state(op)
    o = soc.outputs(p, op, s_ref)
    with _solver(case, device_inputs=True) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-13, precision="fp64")
        s = sv.get_state()
    assert np.abs(s - s_ref).max() / np.abs(s_ref).max() < 1e-10
    assert abs(r["I_tot"] - o.I_tot) / abs(o.I_tot) < 1e-10
    assert abs(r["U"] - o.U) / abs(o.U) < 1e-10


def test_mixed_precision_parity_small_large_recipe():
    """The mixed-precision recipe (porosity 0.85, d ~ U[6,10], 0.5 cm/s, -0.05 V,
    s_in = 0.3) at 32x32x64: FP32 sweeps + FP64 defect correction within 1e-6 max-abs."""
    case = mixed_case_small((32, 32, 64))
    p, op = _oracle(case)
    s_ref = soc.steady_state(op)
    o = soc.outputs(p, op, s_ref)
    with _solver(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-10, precision="mixed")
        s = sv.get_state()
    assert np.abs(s - s_ref).max() < 1e-6
    assert abs(r["I_tot"] - o.I_tot) / abs(o.I_tot) < 1e-5
    assert r["mass_balance_rel"] < 1e-6


@pytest.mark.parametrize("dims,dt_mode", [((37, 21, 19), "local"), ((36, 20, 24), "global"),
                                          ((36, 20, 24), "local")])
def test_mixed_precision_parity_vector_and_scalar_kernels(dims, dt_mode):
    """nx % 4 != 0 runs the scalar FP32 sweep, nx % 4 == 0 the 4-cells-per-thread one."""
    case = fiber_case(dims, diameter=4.0)
    p, op = _oracle(case)
    s_ref = soc.steady_state(op)
    with _solver(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-11, precision="mixed", dt_mode=dt_mode)
        s = sv.get_state()
    assert r["residual"] <= 1e-11
    assert np.abs(s - s_ref).max() < 1e-7


def test_umt_parity():
    case = fiber_case((16, 16, 32))
    p, _ = _oracle(case)
    ref = soc.umt(p)
    with _solver(case) as sv:
        u64, r = sv.umt(1e-13, precision="fp64")
        u32, _ = sv.umt(1e-10, precision="mixed")
    assert abs(u64 - ref) < 1e-10
    assert abs(u32 - ref) < 1e-6
    assert 0.0 <= u64 <= 1.0


# ------------------------------------------------------------------ edge cases

def test_no_reaction_keeps_inlet_value_and_equilibrium_inlet_is_steady():
    case = fiber_case((16, 16, 32))
    with _solver(case) as sv:
        pass
    import dataclasses
    c0 = dataclasses.replace(case, k0=0.0)
    fl = case.solid.ravel() == 0
    with _solver(c0) as sv:
        sv.solve(0.37, case.eta, 1e-12)
        s = sv.get_state()
    assert np.abs(s[fl] - 0.37).max() < 1e-10
    s_eq = soc.kinetics(case.eta).s_eq
    with _solver(case) as sv:
        sv.solve(s_eq, case.eta, 1e-12)
        s = sv.get_state()
    assert np.abs(s[fl] - s_eq).max() < 1e-10


def test_host_and_device_inputs_agree_and_checkpoint_resume_is_bitwise():
    case = fiber_case((16, 16, 32))
    with _solver(case) as a, _solver(case, device_inputs=True) as b:
        a.step(case.s_in, case.eta, 300)
        b.step(case.s_in, case.eta, 300)
        sa, sb = a.get_state(), b.get_state()
        assert np.array_equal(sa, sb)
        a.step(case.s_in, case.eta, 200)
        s_ref = a.get_state()
    with _solver(case) as c:
        c.set_state(sb)
        c.step(case.s_in, case.eta, 200)
        assert np.array_equal(c.get_state(), s_ref)


def test_invalid_velocity_fields_are_rejected():
    from paper_2502_08034_gb300 import rfb
    case = fiber_case((16, 16, 32))
    U = case.U.copy()
    U[:, :, 0] = 1e-3          # flow through a side wall
    with pytest.raises(rfb.RfbError) as e:
        rfb.Solver(case.dims, case.h, case.solid, U, case.V, case.W, case.D, case.k0)
    assert e.value.status == rfb.RFB_ERR_INVALID_ARG
    W = case.W.copy()
    W[0] = -np.abs(W[0])       # backflow through the inlet
    with pytest.raises(rfb.RfbError):
        rfb.Solver(case.dims, case.h, case.solid, case.U, case.V, W, case.D, case.k0)
    V = case.V.copy()
    V[1, 3, 3] = np.nan
    with pytest.raises(rfb.RfbError):
        rfb.Solver(case.dims, case.h, case.solid, case.U, V, case.W, case.D, case.k0)


def test_not_converged_leaves_a_valid_state():
    case = fiber_case((16, 16, 32))
    with _solver(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-14, max_sweeps=10, allow_not_converged=True)
        assert r["status"] == 4 and r["sweeps"] == 10
        s = sv.get_state()
        assert np.all(np.isfinite(s))
        c = sv.current()
        assert c["residual"] == pytest.approx(r["residual"], rel=1e-12)
