"""The Butler-Volmer model with electromigration on the GPU (rfb_soc_solve_bv) against the
oracle (oracle/bv.py), through the C ABI: concentrations, potential and outputs on small
lattices (several tiles of the flat grid, ragged in every direction), model refinement
from the converged SBV state against a cold start, and the refused options."""
import dataclasses
import functools

import numpy as np
import pytest

from oracle import bv, soc
from tests._cases import fiber_case, problem_from_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _case(dims, k0=2e-5):
    c = fiber_case(dims, diameter=4.0, u_mean=0.002, eta=-0.10, s_in=0.2)
    return dataclasses.replace(c, k0=k0)


@functools.lru_cache(maxsize=None)
def _oracle(dims, k0=2e-5):
    case = _case(dims, k0)
    p = problem_from_case(case, soc)
    q = bv.BVParams()
    s0 = soc.steady_state(soc.assemble(p))
    C, phi, _ = bv.solve(p, q, s0=s0, tol=1e-13)
    return p, q, C, phi, bv.outputs(p, q, C, phi)


@pytest.mark.parametrize("dims", [(8, 8, 12), (20, 14, 26)])
def test_bv_state_matches_the_oracle(dims):
    from paper_2502_08034_gb300 import rfb
    case = _case(dims)
    p, q, C, phi, o = _oracle(dims)
    with rfb.Solver.from_case(case) as sv:
        sv.solve(case.s_in, case.eta, 1e-13, precision="fp64")     # SBV first: refinement
        r = sv.solve_bv(case.s_in, case.eta, 1e-12, start="sbv")
        g = sv.get_bv_state()
    fl = p.solid.ravel() == 0
    for k in ("O", "R", "H"):
        err = np.abs(g[k][fl] - C[k][fl]).max() / np.abs(C[k][fl]).max()
        assert err <= 1e-10, (k, err)
    perr = np.abs(g["phi"][fl] - phi[fl]).max() / np.abs(phi[fl]).max()
    assert perr <= 1e-7, perr
    for k in ("I_tot", "U", "s_out", "I_membrane"):
        assert r[k] == pytest.approx(o[k], rel=1e-9), k
    assert r["phi_max"] == pytest.approx(o["phi_max"], rel=1e-6, abs=1e-7 * abs(o["phi_min"]))
    print("BV %s: %d sweeps, %d potential solves, %d CG iterations, phi in [%.3e, %.3e] V, "
          "max phi rel err %.1e" % (dims, r["sweeps"], r["cycles"], r["cg_iterations"],
                                     r["phi_min"], r["phi_max"], perr))


def test_model_refinement_reaches_the_cold_start_fixed_point_in_fewer_sweeps():
    from paper_2502_08034_gb300 import rfb
    dims = (20, 14, 26)
    case = _case(dims)
    with rfb.Solver.from_case(case) as sv:
        cold = sv.solve_bv(case.s_in, case.eta, 1e-11, start="cold")
        gc = sv.get_bv_state()
        sv.solve(case.s_in, case.eta, 1e-13, precision="fp64")
        warm = sv.solve_bv(case.s_in, case.eta, 1e-11, start="sbv")
        gw = sv.get_bv_state()
    fl = case.solid.ravel() == 0
    assert np.abs(gc["R"][fl] - gw["R"][fl]).max() <= 1e-8 * case.c0
    assert warm["sweeps"] < cold["sweeps"]


def test_bv_refusals():
    from paper_2502_08034_gb300 import rfb
    case = _case((8, 8, 12))
    with rfb.Solver.from_case(case) as sv:
        for kw in (dict(precision="mixed"), dict(dt_mode="global")):
            with pytest.raises(rfb.RfbError) as e:
                sv.solve_bv(case.s_in, case.eta, 1e-10, **kw)
            assert e.value.status == rfb.RFB_ERR_INVALID_ARG
        with pytest.raises(rfb.RfbError) as e:
            sv.solve_bv(case.s_in, case.eta, 1e-10, start="sbv")   # no SBV state yet
        assert e.value.status == rfb.RFB_ERR_STATE
        with pytest.raises(rfb.RfbError) as e:
            sv.solve_bv(case.s_in, case.eta, 1e-10, c_H_in=10.0)   # below 2 c0
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
        with pytest.raises(rfb.RfbError) as e:
            sv.get_bv_state()
        assert e.value.status == rfb.RFB_ERR_STATE
