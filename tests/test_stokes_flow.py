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


def _random_open(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.random(shape) < 0.7


def test_multigrid_coarse_stencil_is_the_galerkin_product():
    """The coarse level of the velocity multigrid equals P^T A P / beta, with A assembled
    entry by entry from the fine stencil and P the piecewise-constant prolongation over
    2 x 2 x 2 blocks, both as explicit sparse matrices (odd extents: partial blocks)."""
    torch = pytest.importorskip("torch")
    import scipy.sparse as sp
    shape = (5, 6, 7)
    o_np = _random_open(shape, 3)
    rng = np.random.default_rng(4)
    d_np = np.where(o_np, 6.0 + rng.random(shape), 0.0)
    o, d = torch.from_numpy(o_np), torch.from_numpy(d_np)
    mg = synth._FaceMultigrid(o, d, beta=1.7, coarse_max=1)
    assert len(mg.levels) >= 3
    for lvl in range(len(mg.levels) - 1):
        fo, fd, fc, _ = mg.levels[lvl]
        co, cd, cc, _ = mg.levels[lvl + 1]
        fo, fd = fo.numpy(), fd.numpy()
        fc = [x.numpy() for x in fc]
        nf = fo.size
        A = sp.lil_matrix((nf, nf))
        P = sp.lil_matrix((nf, co.numel()))
        cshape = tuple(co.shape)
        for k, j, i in np.ndindex(fo.shape):
            f = np.ravel_multi_index((k, j, i), fo.shape)
            A[f, f] = fd[k, j, i]
            for a, nb in enumerate(((k + 1, j, i), (k, j + 1, i), (k, j, i + 1))):
                if nb[a] < fo.shape[a] and fc[a][k, j, i] != 0.0:
                    g = np.ravel_multi_index(nb, fo.shape)
                    A[f, g] = A[g, f] = fc[a][k, j, i]
            if fo[k, j, i]:
                P[f, np.ravel_multi_index((k // 2, j // 2, i // 2), cshape)] = 1.0
        G = (P.T @ A.tocsr() @ P).toarray() / 1.7
        co_np = co.numpy()
        assert np.array_equal(co_np.reshape(-1), np.asarray(P.sum(axis=0)).reshape(-1) > 0)
        want_d = np.diag(G).reshape(cshape)
        assert np.allclose(cd.numpy(), np.where(co_np, want_d, 0.0), rtol=1e-14, atol=1e-14)
        for a in range(3):
            got = cc[a].numpy()
            for idx in np.ndindex(cshape):
                nb = list(idx)
                nb[a] += 1
                want = (G[np.ravel_multi_index(idx, cshape), np.ravel_multi_index(nb, cshape)]
                        if nb[a] < cshape[a] else 0.0)
                assert abs(got[idx] - want) <= 1e-14, (lvl, a, idx)


def test_multigrid_cycle_is_a_symmetric_positive_definite_preconditioner():
    """MINRES needs a symmetric positive definite preconditioner: the V-cycle's matrix,
    taken column by column on the open faces of a fiber-like mask with three levels, is
    symmetric, and its product with A has a positive spectrum with a small spread."""
    torch = pytest.importorskip("torch")
    solid = np.zeros((8, 7, 9), dtype=bool)
    solid[2:6, 2:4, :] = True
    solid[:, 5, 3:6] = True
    oU, oV, oW = synth._open_faces(~solid)
    o = torch.from_numpy(oW)
    # the W component's diagonal as stokes_flow_minres builds it
    ones = torch.ones(o.shape, dtype=torch.bool)
    d = torch.zeros(o.shape, dtype=torch.float64)
    for axis in range(3):
        for step in (-1, 1):
            nb = synth._shift(o, axis, step)
            inside = synth._shift(ones, axis, step)
            wall = 1.0 if axis == 0 else 2.0
            d += 1.0 * nb + wall * (inside & ~nb)
            if axis != 0:
                d += wall * ~inside
    d = d * o
    mg = synth._FaceMultigrid(o, d, coarse_max=20)
    assert len(mg.levels) >= 3
    fo, fd, fc, _ = mg.levels[0]
    cols = torch.nonzero(o.reshape(-1)).reshape(-1)
    n = cols.numel()
    B = np.zeros((n, n))
    A = np.zeros((n, n))
    for m, c in enumerate(cols.tolist()):
        e = torch.zeros(o.numel(), dtype=torch.float64)
        e[c] = 1.0
        e = e.view(o.shape)
        B[:, m] = mg.vcycle(e).reshape(-1)[cols].numpy()
        A[:, m] = synth._stencil_apply(fd, fc, e).reshape(-1)[cols].numpy()
    assert np.abs(A - A.T).max() == 0.0
    assert np.abs(B - B.T).max() <= 1e-13 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0.0
    ev = np.sort(np.linalg.eigvals(B @ A).real)
    assert ev[0] > 0.0 and ev[-1] / ev[0] < 20.0, (ev[0], ev[-1])


@pytest.mark.parametrize("solid", [_obstacle(), np.zeros((6, 12, 12), dtype=bool)],
                         ids=["obstacle", "duct"])
def test_jacobi_preconditioned_minres_matches_the_sparse_lu_fixture(solid):
    a = synth.stokes_flow(solid, 1e-6, dp=2.0)
    b = synth.stokes_flow_minres(solid, 1e-6, dp=2.0, tol=1e-12, precond="jacobi")
    scale = np.abs(a[2]).max()
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-10 * scale
    assert b[3]["precond"] == "jacobi"


def test_multigrid_keeps_minres_iterations_nearly_flat_under_refinement():
    """A channel with a bar across it and a post beside it, the same geometry at cell sizes
    h, h/2 and h/4: halving h multiplies the Jacobi-preconditioned MINRES iteration count
    by more than two (the Laplacian's condition number grows like h^-2), the
    multigrid-preconditioned one by much less, and both give the same flow."""
    its, q = {}, {}
    for r in (1, 2, 4):
        solid = np.zeros((12 * r, 9 * r, 10 * r), dtype=bool)
        solid[4 * r:8 * r, 3 * r:6 * r, :] = True
        solid[:, 7 * r:8 * r, 2 * r:4 * r] = True
        for pc in ("mg", "jacobi"):
            *_, info = synth.stokes_flow_minres(solid, 1e-6 / r, dp=1.0, tol=1e-10, precond=pc)
            its[pc, r] = info["minres_iters"]
            q[pc, r] = info["q_m3_s"]
        assert abs(q["mg", r] / q["jacobi", r] - 1.0) < 1e-9
    for r in (2, 4):
        growth_mg = its["mg", r] / its["mg", r // 2]
        growth_j = its["jacobi", r] / its["jacobi", r // 2]
        assert growth_j > 2.0 and growth_mg < 0.75 * growth_j, its
    assert its["mg", 4] * 5 < its["jacobi", 4], its


@pytest.mark.parametrize("shape", [(6, 5, 1), (6, 1, 5), (8, 1, 1), (3, 4, 4)])
def test_multigrid_minres_on_degenerate_lattices(shape):
    """One cell across in x and/or y leaves a velocity component with no open face (an
    empty multigrid level) and coarsening stops at extents of one; the flow still matches
    the sparse-LU fixture."""
    s = np.zeros(shape, dtype=bool)
    a = synth.stokes_flow(s, 1e-6, dp=1.0)
    b = synth.stokes_flow_minres(s, 1e-6, dp=1.0, tol=1e-12)
    assert abs(b[3]["q_m3_s"] / a[3]["q_m3_s"] - 1.0) <= 1e-12
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-10 * np.abs(a[2]).max()
