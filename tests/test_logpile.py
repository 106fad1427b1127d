"""The logpile lattice of the paper's benchmarks (Sec. IV) as a synthetic input (no GPU):
the rod layout the paper describes, the voxel porosity converging to the continuous
value, the box's mirror symmetries, and a flow field that carries the requested flow rate
through every plane without crossing a rod."""
import math

import numpy as np
import pytest

from paper_2502_08034_gb300 import synth


def test_rod_layout_is_the_papers():
    """43 rods of 20 um in seven layers at heights 20, 40, ..., 140 um; the odd layers
    along the flow (four rods 128 um apart across the 640 um width), the even layers
    across it (nine rods 128 um apart along the 1280 um length)."""
    rods = synth.logpile_rods()
    assert len(rods) == 43
    assert sorted({r[2] for r in rods}) == [20.0 * k for k in range(1, 8)]
    for layer, along, height, pos in rods:
        assert height == 20.0 * layer
        assert along == ("z" if layer % 2 else "y")
    along = [r for r in rods if r[1] == "z"]
    across = [r for r in rods if r[1] == "y"]
    assert len(along) == 16 and len(across) == 27
    assert sorted({r[3] for r in along}) == [128.0, 256.0, 384.0, 512.0]
    assert sorted({r[3] for r in across}) == [128.0 * m for m in range(1, 10)]
    # adjacent layers are one diameter apart: crossing rods touch
    assert synth.LOGPILE_LAYER_UM == synth.LOGPILE_ROD_D_UM
    assert synth.logpile_dims(1.25e-6) == (128, 512, 1024)      # 2^26 cells, as printed


def test_voxel_porosity_converges_to_the_continuous_value():
    """The continuous fluid fraction is 1 - pi r^2 (16 x 1280 + 27 x 640) / (1280 x 640 x
    160) = 0.90950; the voxel fraction approaches it as h shrinks."""
    exact = synth.logpile_porosity_exact()
    r = 10.0
    assert abs(exact - (1 - math.pi * r * r * (16 * 1280 + 27 * 640) / (1280 * 640 * 160))) < 1e-15
    errs = [abs((1.0 - synth.logpile_solid(h).mean()) - exact) for h in (5e-6, 2.5e-6, 1.25e-6)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-3


def test_mirror_symmetries_of_the_box():
    """The rods are placed symmetrically about the middle of the box's length, width and
    height, so the voxel mask equals each of its three mirror images."""
    s = synth.logpile_solid(2.5e-6)
    assert np.array_equal(s, s[::-1]) and np.array_equal(s, s[:, ::-1])
    assert np.array_equal(s, s[:, :, ::-1])


def test_rod_axes_are_solid_and_the_gaps_fluid():
    h = 2.5e-6
    s = synth.logpile_solid(h)
    um = h * 1e6
    for _, along, height, pos in synth.logpile_rods():
        i = int(height / um)
        if along == "z":
            j = int(pos / um)
            assert s[:, j, i].all()                      # the rod spans the whole length
        else:
            k = int(pos / um)
            assert s[k, :, i].all()                      # and the whole width
    # half-way between two rods of layer 1 (along the flow, height 20 um), at that
    # height: 64 um from both rods, and 20 um below the layer-2 axes (radius 10 um)
    assert not s[:, int(192.0 / um), int(20.0 / um)].any()


def test_flow_rate_and_no_flux_through_rods():
    c = synth.logpile_case(10e-6)
    h, q = c.h, synth.LOGPILE_Q_10PA
    fl = c.solid == 0
    nz = c.dims[2]
    for k in range(nz + 1):
        open_ = fl[min(k, nz - 1)] & fl[max(k - 1, 0)]
        assert abs(h * h * float(c.W[k][open_].sum()) - q) <= 1e-9 * q, k
        assert np.all(c.W[k][~open_] == 0.0)
    assert np.all(c.W[0] >= 0.0) and np.all(c.W[-1] >= 0.0)
    sol = c.solid.astype(bool)
    # no face velocity on a face of a rod or of a side wall
    assert np.all(c.U[:, :, 1:-1][sol[:, :, 1:] | sol[:, :, :-1]] == 0.0)
    assert np.all(c.U[:, :, [0, -1]] == 0.0) and np.all(c.V[:, [0, -1], :] == 0.0)
    assert np.all(c.V[:, 1:-1, :][sol[:, 1:, :] | sol[:, :-1, :]] == 0.0)
    assert c.info["max_div_rel"] < 1e-11
    assert c.eta == 0.0 and c.k0 == 7.2e-5 and c.s_in == pytest.approx(1.73e-7)


def test_box_must_be_divisible():
    with pytest.raises(ValueError):
        synth.logpile_dims(3e-6)
