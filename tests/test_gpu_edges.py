"""Edge cases of the GPU path against the oracle: a lattice with no fluid cell, no flow
(velocity scale 0: the diffusion-reaction problem with the inlet Dirichlet condition), a
3 x 3 x n fiber-walled channel (nx = 3: the scalar FP32 kernel) and the thinnest lattice
(nz = 2)."""

import numpy as np
import pytest

from oracle import soc
from tests._cases import channel_1d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


def _solver(solid, U, V, W, h, D=4e-10, k0=1e-6, **kw):
    from paper_2502_08034_gb300 import rfb
    nz, ny, nx = solid.shape
    return rfb.Solver((nx, ny, nz), h, solid.astype(np.uint8), U, V, W, D, k0, **kw)


def test_lattice_without_fluid_cells_is_rejected():
    """Nothing to solve: create refuses a lattice without fluid cells."""
    from paper_2502_08034_gb300 import rfb
    n = 8
    solid = np.ones((n, 4, 4), dtype=np.uint8)
    U = np.zeros((n, 4, 5)); V = np.zeros((n, 5, 4)); W = np.zeros((n + 1, 4, 4))
    with pytest.raises(rfb.RfbError) as e:
        _solver(solid, U, V, W, 1.25e-6)
    assert e.value.status == rfb.RFB_ERR_INVALID_ARG and "no fluid" in str(e.value)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_no_flow_is_the_inlet_diffusion_reaction_problem(precision):
    """velocity_scale = 0: no advection, tau falls back to (nz h)^2 / D; still a nonsingular
    problem (the inlet Dirichlet face and the reaction), matched against the oracle."""
    from paper_2502_08034_gb300 import rfb, synth
    case = synth.build_case("noflow", (16, 16, 32), 0.80, 4.0, 11, 0.01, -0.10, 0.5, 1e-12)
    p = soc.Problem(case.solid, case.U, case.V, case.W, case.h, case.D, case.s_in,
                    k0=case.k0, eta=case.eta, beta=0.0)
    op = soc.assemble(p)
    ref = soc.steady_state(op)
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-11, precision=precision, velocity_scale=0.0,
                     max_sweeps=20_000_000)
        s = sv.get_state()
    assert r["residual"] <= 1e-11
    assert abs(r["tau"] - op.tau) <= 1e-12 * op.tau
    tol = 1e-9 if precision == "fp64" else 1e-7
    assert np.abs(s - ref).max() <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("inlet_bc", ["face", "ghost"])
def test_fiber_walled_channel_nx3(precision, inlet_bc):
    """3 x 3 x 40: the centre column is a 1D channel with four fiber neighbours per cell;
    its exact discrete solution is pinned by the oracle's closed form."""
    n, w, h = 40, 0.01, 1.25e-6
    solid, U, V, W, _ = channel_1d(n, w, h)
    p = soc.Problem(solid, U, V, W, h, 4e-10, 0.2, k0=1e-6, eta=-0.08, inlet_bc=inlet_bc)
    ref = soc.steady_state(soc.assemble(p))
    with _solver(solid, U, V, W, h, k0=1e-6) as sv:
        r = sv.solve(0.2, -0.08, 1e-12, precision=precision, inlet_bc=inlet_bc)
        s = sv.get_state()
    tol = 1e-10 if precision == "fp64" else 1e-7
    assert r["residual"] <= 1e-12
    assert np.abs(s - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_thinnest_lattice_nz2():
    """nz = 2: every fluid cell is an inlet or an outlet cell."""
    from paper_2502_08034_gb300 import rfb, synth
    case = synth.build_case("thin", (16, 16, 2), 0.95, 1.0, 3, 0.01, -0.10, 0.5, 1e-12)
    p = soc.Problem(case.solid, case.U, case.V, case.W, case.h, case.D, case.s_in,
                    k0=case.k0, eta=case.eta)
    ref = soc.steady_state(soc.assemble(p))
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-13, precision="fp64")
        s = sv.get_state()
    assert r["residual"] <= 1e-13
    assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max()
