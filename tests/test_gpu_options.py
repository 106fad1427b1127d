"""Solve options that bound the work: opts.timeout_ms on single solves, adjoints and
batches (the state stays valid and readable), and its validation."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _case():
    from paper_2502_08034_gb300 import synth
    return synth.fiber_channel_case()      # 48 x 48 x 96


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_timeout_stops_a_solve_with_a_valid_state(precision):
    from paper_2502_08034_gb300 import rfb
    case = _case()
    with rfb.Solver.from_case(case) as sv:
        # a tolerance below the rounding floor: only the timeout ends the solve
        r = sv.solve(case.s_in, case.eta, 1e-30, precision=precision, timeout_ms=300,
                     check_every=50, allow_not_converged=True)
        msg = rfb.lib().rfb_soc_last_error(sv.h).decode()   # the next call clears it
        s = sv.get_state()
    assert r["status"] == rfb.RFB_ERR_NOT_CONVERGED
    assert "timeout" in msg
    assert 300 <= r["time_ms"] < 5000
    assert r["sweeps"] > 0 and np.all(np.isfinite(s))


def test_timeout_stops_an_adjoint_and_a_batch():
    from paper_2502_08034_gb300 import rfb
    case = _case()
    with rfb.Solver.from_case(case) as sv:
        sv.solve(case.s_in, case.eta, 1e-12, precision="fp64")
        with pytest.raises(rfb.RfbError) as e:
            sv.adjoint("I_tot", 1e-30, timeout_ms=200, check_every=50)
        assert e.value.status == rfb.RFB_ERR_NOT_CONVERGED
        sv.reset_state()
        with rfb.Batch([sv]) as b:
            res, info = b.solve([case.s_in], [case.eta], [1e-30], timeout_ms=300,
                                check_every=50, allow_not_converged=True)
        assert res[0]["sweeps"] > 0 and np.isfinite(res[0]["residual"])
        with pytest.raises(rfb.RfbError) as e:
            sv.solve(case.s_in, case.eta, 1e-8, timeout_ms=-1)
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG


def test_outputs_after_a_umt_solve_at_another_velocity_scale():
    """rfb_soc_current evaluates the last solve's operating point, velocity scale
    included, even after a U_mt solve (or an adjoint) used another scale in between."""
    from paper_2502_08034_gb300 import rfb
    from tests._cases import fiber_case
    case = fiber_case((16, 16, 32))
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-12, precision="fp64", velocity_scale=1.0)
        before = sv.current()
        sv.umt(1e-10, precision="fp64", velocity_scale=2.0)
        after = sv.current()
    for k in ("residual", "I_tot", "F_in", "F_out", "F_in_adv", "U", "outlet_mean",
              "mass_balance_rel"):
        assert after[k] == before[k], k
    assert before["I_tot"] == pytest.approx(r["I_tot"], rel=1e-12)
