"""The seeded input recipe (no GPU): the project-written SplitMix64 against the reference
generator's published output, the fiber rasteriser against a cell-by-cell distance test,
the stopping rule of the fiber generator, and the flood fill that removes fluid pockets
not connected to the inlet."""
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
