"""Iterative upsampling (Sec. III.A): GPU prolongation against the oracle's, and the
upsampled solve reaching the same fixed point as a cold start in fewer sweeps."""
import functools

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
