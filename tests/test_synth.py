"""The seeded input recipe (no GPU): the project-written SplitMix64 against the reference
generator's published output, the fiber rasteriser against a cell-by-cell distance test,
the stopping rule of the fiber generator, the flood fill that removes fluid pockets not
connected to the inlet, and the host potential-flow solver against its discrete problem
written out and solved by sparse LU."""
import math

import numpy as np
import pytest

from paper_2502_08034_gb300 import synth


def test_splitmix64_matches_the_reference_output():
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the first five outputs of the
    reference implementation seeded with 1234567, as its published test vector lists
    them."""
    r = synth.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_uniform_uses_the_top_53_bits():
    a, b = synth.SplitMix64(99), synth.SplitMix64(99)
    for _ in range(100):
        u = a.uniform(-2.0, 3.0)
        assert u == -2.0 + 5.0 * ((b.next_u64() >> 11) / 2.0 ** 53)
        assert -2.0 <= u < 3.0


def test_rasterised_fiber_is_the_set_of_cell_centres_within_its_radius():
    f = synth.Fiber(z0=5.3, x0=6.1, y0=3.7, theta=0.7, d=4.5)
    dims = (13, 9, 11)
    solid = synth.rasterise([f], dims)
    nx, ny, nz = dims
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                x, y, z = i + 0.5, j + 0.5, k + 0.5
                # distance from the axis: the in-plane offset across the axis direction
                # (cos theta, sin theta, 0) and the height above the plane z = z0
                across = (x - f.x0) * math.sin(f.theta) - (y - f.y0) * math.cos(f.theta)
                inside = across ** 2 + (z - f.z0) ** 2 <= (f.d / 2) ** 2
                assert solid[k, j, i] == inside, (i, j, k)


def test_fibers_are_added_until_the_porosity_is_first_reached():
    dims = (24, 20, 40)
    fibers, solid = synth.generate_fibers(7, dims, 0.8, (3.0, 5.0))
    n = np.prod(dims)
    assert 1.0 - solid.sum() / n <= 0.8
    before = synth.rasterise(fibers[:-1], dims)
    assert 1.0 - before.sum() / n > 0.8
    assert np.array_equal(synth.rasterise(fibers, dims), solid)
    assert all(3.0 <= f.d <= 5.0 and 0.0 <= f.theta < math.pi for f in fibers)


def test_unconnected_fluid_is_made_solid():
    solid = np.zeros((7, 5, 5), dtype=bool)
    solid[2] = True                 # a wall across the channel at k = 2 ...
    solid[2, 0, 0] = False          # ... with one hole: everything stays connected
    assert np.array_equal(synth.remove_unconnected(solid), solid)
    sealed = solid.copy()
    sealed[3:6, 1:4, 1:4] = True    # a solid block downstream of the wall ...
    sealed[4, 2, 2] = False         # ... enclosing one fluid cell on all six sides
    out = synth.remove_unconnected(sealed)
    want = sealed.copy()
    want[4, 2, 2] = True
    assert np.array_equal(out, want)
    blocked = solid.copy()
    blocked[2, 0, 0] = True         # no path from the inlet plane to the outlet plane
    with pytest.raises(ValueError):
        synth.remove_unconnected(blocked)


def _potential_flow_direct(solid, u_mean):
    """The potential-flow fixture's discrete problem written out and solved by sparse LU:
    cell-centred phi on fluid cells, conductance 1 between fluid neighbours, 2 to the inlet
    face (phi = 1) and the outlet face (phi = 0) of the first and last plane, none through
    solid cells or side walls; face velocities -grad phi, scaled so that the mean of W over
    fluid z-faces (inlet and outlet faces included) is u_mean."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nz, ny, nx = solid.shape
    fl = ~solid.astype(bool)
    idx = -np.ones(solid.shape, dtype=np.int64)
    idx[fl] = np.arange(int(fl.sum()))
    rows, cols, vals = [], [], []
    diag = np.zeros(int(fl.sum()))
    b = np.zeros_like(diag)
    for k, j, i in zip(*np.nonzero(fl)):
        c = idx[k, j, i]
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            kk, jj, ii = k + dk, j + dj, i + di
            if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx and fl[kk, jj, ii]:
                diag[c] += 1.0
                rows.append(c); cols.append(idx[kk, jj, ii]); vals.append(-1.0)
        if k == 0:
            diag[c] += 2.0
            b[c] += 2.0
        if k == nz - 1:
            diag[c] += 2.0
    A = sp.csr_matrix((vals, (rows, cols)), shape=(diag.size, diag.size)) + sp.diags(diag)
    phi = np.zeros(solid.shape)
    phi[fl] = spla.spsolve(A.tocsc(), b)
    U = np.zeros((nz, ny, nx + 1))
    V = np.zeros((nz, ny + 1, nx))
    W = np.zeros((nz + 1, ny, nx))
    U[:, :, 1:nx] = np.where(fl[:, :, 1:] & fl[:, :, :-1], phi[:, :, :-1] - phi[:, :, 1:], 0.0)
    V[:, 1:ny, :] = np.where(fl[:, 1:] & fl[:, :-1], phi[:, :-1] - phi[:, 1:], 0.0)
    W[1:nz] = np.where(fl[1:] & fl[:-1], phi[:-1] - phi[1:], 0.0)
    W[0] = np.where(fl[0], 2.0 * (1.0 - phi[0]), 0.0)
    W[nz] = np.where(fl[-1], 2.0 * phi[-1], 0.0)
    zf = np.concatenate([fl[:1], fl[1:] & fl[:-1], fl[-1:]])
    f = u_mean / W[zf].mean()
    return U * f, V * f, W * f


def test_host_potential_flow_is_the_discrete_potential_problem():
    _, solid = synth.generate_fibers(3, (14, 12, 20), 0.8, 3.0)
    solid = synth.remove_unconnected(solid)
    got = synth.potential_flow(solid, 1e-6, 0.004)
    want = _potential_flow_direct(solid, 0.004)
    for g, w in zip(got[:3], want):
        assert np.abs(g - w).max() <= 1e-10 * 0.004


def test_batched_workload_recipe():
    """The 48-lattice batch: lattice 0 is 64^3 and lattice 1 192x192x384; the others have
    nx = ny in {64, 80, ..., 192} and nz a multiple of 16 between nx and 2 nx (inside the
    clipping range [64, 384]); porosity, mean velocity (log-uniform), s_in and eta
    lie in their ranges; 187M cells in all."""
    qs = [synth.batch_instance_params(i) for i in range(48)]
    assert qs[0]["dims"] == (64, 64, 64) and qs[1]["dims"] == (192, 192, 384)
    for q in qs[2:]:
        nx, ny, nz = q["dims"]
        assert nx == ny and nx in range(64, 193, 16)
        assert nz % 16 == 0 and 64 <= nz <= 384
        assert nx <= nz <= 2 * nx                       # 16 round(nx U[1, 2] / 16)
    for i, q in enumerate(qs):
        assert q["seed"] == 3000 + i
        assert 0.75 <= q["porosity"] <= 0.90
        assert 0.001 <= q["u_mean"] <= 0.05
        assert 0.1 <= q["s_in"] <= 0.9 and -0.2 <= q["eta"] <= -0.02
    cells = sum(np.prod(q["dims"]) for q in qs)
    assert 180e6 < cells < 195e6, cells
    assert len({q["dims"] for q in qs}) > 20            # uneven sizes
    us = np.log10([q["u_mean"] for q in qs])
    assert us.min() < -2.5 and us.max() > -1.6        # spread over the log range


def test_multilevel_lattices_rasterise_the_same_fibers():
    """Every level of an upsampling chain rasterises the fibers drawn once at the finest
    level: a coarse cell is solid exactly when its centre, in finest-level units, lies
    within a fiber's radius (before the flood fill), and the cell size doubles per level."""
    fine = (32, 24, 48)
    fibers, solid_f = synth.generate_fibers(9, fine, 0.85, 4.0)
    cases = synth.multilevel_cases(fine, 3, 0.85, 4.0, 9, 0.01, -0.1, 0.5, 1e-8,
                                   h_fine=1e-6)
    assert [c.dims for c in cases] == [(8, 6, 12), (16, 12, 24), (32, 24, 48)]
    assert [c.h for c in cases] == [4e-6, 2e-6, 1e-6]
    assert np.array_equal(cases[-1].solid.astype(bool), synth.remove_unconnected(solid_f))
    for c, f in zip(cases[:2], (4, 2)):
        nx, ny, nz = c.dims
        raw = np.zeros((nz, ny, nx), dtype=bool)
        for fb in fibers:
            for k in range(nz):
                z = (k + 0.5) * f - fb.z0
                for j in range(ny):
                    y = (j + 0.5) * f
                    x = (np.arange(nx) + 0.5) * f
                    across = (x - fb.x0) * math.sin(fb.theta) - (y - fb.y0) * math.cos(fb.theta)
                    raw[k, j] |= across ** 2 + z ** 2 <= (fb.d / 2) ** 2
        assert np.array_equal(c.solid.astype(bool), synth.remove_unconnected(raw))


def test_area_multipliers_are_lognormal_on_wall_cells_only():
    _, solid = synth.generate_fibers(4, (40, 40, 60), 0.8, 8.0)
    m = synth.lognormal_area_mult(solid, sigma=0.3, seed=40)
    s = solid.astype(bool)
    pad = np.pad(s, 1)
    touch = (pad[1:-1, 1:-1, :-2] | pad[1:-1, 1:-1, 2:] | pad[1:-1, :-2, 1:-1] |
             pad[1:-1, 2:, 1:-1] | pad[:-2, 1:-1, 1:-1] | pad[2:, 1:-1, 1:-1])
    wall = touch & ~s
    assert np.all(m[~wall] == 1.0)
    z = np.log(m[wall]) / 0.3
    assert z.size > 5000
    assert np.array_equal(z, np.log(np.exp(0.3 * np.random.default_rng(40).standard_normal(
        z.size))) / 0.3)
    assert abs(np.median(z)) < 0.05 and abs(z.std() - 1.0) < 0.03
