"""The Stokes-flow input fixtures (no GPU): the analytic flow rate of a square duct at
second order in h, linearity in the pressure drop, no slip and symmetry around an
obstacle (sparse LU), the matrix-free MINRES solver against it, and the magnitude of the
logpile's flow rate against the one the paper reports (Sec. IV)."""
import math

import numpy as np
import pytest

from paper_2502_08034_gb300 import synth


def _duct_q_exact(a, G, mu):
    """Fully developed flow rate of a square duct of side a under pressure gradient G:
    G a^4 / (12 mu) (1 - 192 / pi^5 sum over odd m of tanh(m pi / 2) / m^5)."""
    s = sum(math.tanh(m * math.pi / 2) / m ** 5 for m in range(1, 400, 2))
    return G * a ** 4 / (12 * mu) * (1 - 192 / math.pi ** 5 * s)


def test_square_duct_flow_rate_at_second_order():
    """An open lattice is a square duct with no-slip side walls; with zero normal gradient
    at both ends the flow is fully developed everywhere, driven by dp over the (nz + 1) h
    between the two ghost pressure planes."""
    nz, h, dp = 6, 1e-6, 1.0
    errs = []
    for n in (8, 16, 32):
        U, V, W, info = synth.stokes_flow(np.zeros((nz, n, n), dtype=bool), h, dp=dp)
        q_exact = _duct_q_exact(n * h, dp / ((nz + 1) * h), synth.MU_WATER)
        errs.append(info["q_m3_s"] / q_exact - 1.0)
        planes = h * h * W.sum(axis=(1, 2))
        assert np.ptp(planes) <= 1e-9 * planes.mean()          # z-invariant
        assert np.abs(U).max() <= 1e-9 * W.max() and np.abs(V).max() <= 1e-9 * W.max()
        assert info["max_div_rel"] < 1e-9
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert errs[2] < 0.005 and all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


def _obstacle():
    solid = np.zeros((12, 9, 10), dtype=bool)
    solid[4:8, 3:6, :] = True           # a bar across the channel, touching both x walls
    return solid


def test_flow_is_linear_in_the_pressure_drop():
    s = _obstacle()
    a = synth.stokes_flow(s, 1e-6, dp=1.0)
    b = synth.stokes_flow(s, 1e-6, dp=3.0)
    for x, y in zip(a[:3], b[:3]):
        assert np.allclose(3.0 * x, y, rtol=1e-9, atol=1e-12 * np.abs(y).max())


def test_no_slip_mass_conservation_and_symmetry_around_an_obstacle():
    s = _obstacle()
    U, V, W, info = synth.stokes_flow(s, 1e-6, dp=1.0)
    # no flow through a face of the bar or of a side wall
    assert np.all(U[:, :, 1:-1][s[:, :, 1:] | s[:, :, :-1]] == 0.0)
    assert np.all(V[:, 1:-1, :][s[:, 1:, :] | s[:, :-1, :]] == 0.0)
    assert np.all(W[1:-1][s[1:] | s[:-1]] == 0.0)
    assert np.all(U[:, :, [0, -1]] == 0.0) and np.all(V[:, [0, -1], :] == 0.0)
    assert info["max_div_rel"] < 1e-9
    # every plane carries the inlet's flow; the flow goes around the bar (over and under)
    fl = ~s
    q = info["q_m3_s"]
    for k in range(1, s.shape[0]):
        assert abs(1e-12 * W[k][fl[k - 1] & fl[k]].sum() - q) <= 1e-9 * q
    assert np.abs(V).max() > 0.05 * W.max()
    # the bar is symmetric about the channel's mid-plane in x (and spans all of x):
    # the flow is mirror-symmetric in x
    assert np.allclose(W, W[:, :, ::-1], atol=1e-12 * W.max())
    assert np.allclose(V, V[:, :, ::-1], atol=1e-12 * W.max())


@pytest.mark.parametrize("solid", [_obstacle(), np.zeros((6, 12, 12), dtype=bool)],
                         ids=["obstacle", "duct"])
def test_matrix_free_minres_matches_the_sparse_lu_fixture(solid):
    """The matrix-free MINRES solver (PyTorch, any device) and the sparse-LU one solve the
    same discrete Stokes problem: their fields agree to the MINRES tolerance."""
    a = synth.stokes_flow(solid, 1e-6, dp=2.0)
    b = synth.stokes_flow_minres(solid, 1e-6, dp=2.0, tol=1e-12)
    scale = np.abs(a[2]).max()
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-10 * scale
    assert abs(b[3]["q_m3_s"] / a[3]["q_m3_s"] - 1.0) <= 1e-12
    assert b[3]["max_div_rel"] < 1e-10


def test_logpile_flow_rate_is_of_the_papers_magnitude():
    """Sec. IV reports 3.45 mL/h through the logpile at 100 Pa (cut cells at 1.25 um). The
    voxel logpile is not converged at the cell sizes a CPU reaches: 3.457 mL/h at 10 um
    (rods two cells across) and 2.919 at 5 um. So this checks only the magnitude (within
    20 %) and what the solver requires of the field; the fixture itself is pinned by the
    duct, the sparse-LU solve, linearity and symmetry above."""
    solid = synth.remove_unconnected(synth.logpile_solid(10e-6))
    U, V, W, info = synth.stokes_flow_minres(solid, 10e-6, dp=100.0, tol=1e-10)
    q_ml_h = info["q_m3_s"] * 3600e6
    assert abs(q_ml_h / 3.45 - 1.0) < 0.2, q_ml_h
    # what the solver's create requires of a flow field: no inflow through the outlet or
    # outflow through the inlet, nothing through fiber faces or side walls
    assert np.all(W[0] >= 0.0) and np.all(W[-1] >= 0.0)
    assert np.all(W[1:-1][solid[1:] | solid[:-1]] == 0.0)
    assert np.all(U[:, :, 1:-1][solid[:, :, 1:] | solid[:, :, :-1]] == 0.0)
    assert np.all(V[:, 1:-1, :][solid[:, 1:, :] | solid[:, :-1, :]] == 0.0)
    assert np.all(U[:, :, [0, -1]] == 0.0) and np.all(V[:, [0, -1], :] == 0.0)
