"""Batched solves (one persistent launch per sweep over every lattice, CUDA-graph cycles
driven from the device, autotuned work items) against the oracle and against one-lattice
solves."""
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
def _small_batch(n=6):
    from paper_2502_08034_gb300 import synth
    return synth.batch_cases(n, scale=4, tol=1e-10)


def test_small_batch_matches_oracle_and_single_solves():
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()
    solvers = [rfb.Solver.from_case(c) for c in cases]
    try:
        with rfb.Batch(solvers) as b:
            res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                [1e-10] * len(cases))
        states = [s.get_state() for s in solvers]
        assert info["n_items"] > 0 and info["kchunk"] in (8, 16, 32, 64)
        assert info["sweeps_per_cycle"] % 2 == 0
        for c, r, s, sv in zip(cases, res, states, solvers):
            assert r["residual"] <= 1e-10
            ref = soc.steady_state(soc.assemble(problem_from_case(c, soc)))
            assert np.abs(s - ref).max() < 1e-6, c.name
            sv.reset_state()
            r1 = sv.solve(c.s_in, c.eta, 1e-10, precision="mixed")
            assert np.abs(sv.get_state() - ref).max() < 1e-6
            assert abs(r["I_tot"] - r1["I_tot"]) <= 1e-6 * abs(r1["I_tot"])
        # lattices converge at different sweep counts (uneven sizes / operating points)
        assert len({r["sweeps"] for r in res}) > 1
    finally:
        for s in solvers:
            s.close()


def test_device_driven_loop_equals_the_host_driven_cycles():
    """Without a timeout the cycles run in the device-driven loop (a conditional while
    node; a graph launch per 64 cycles of each check precision); with one, one captured cycle per
    launch with the host in between. Both run the same cycles: bitwise the same states,
    sweep counts and residuals."""
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()
    out = []
    for timeout in (0, 600000):
        solvers = [rfb.Solver.from_case(c) for c in cases]
        try:
            with rfb.Batch(solvers) as b:
                res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                    [1e-10] * len(cases), check_every=40, timeout_ms=timeout)
            out.append(([s.get_state() for s in solvers], res, info))
        finally:
            for s in solvers:
                s.close()
    (sa, ra, ia), (sb, rb, ib) = out
    assert ia["cycles"] == ib["cycles"] and ib["graph_launches"] == ib["cycles"]
    # the double-float cycles, then (for lattices whose tol lies below the double-float
    # floor) the FP64 ones: one device-driven launch per 64 cycles of each
    assert ia["graph_launches"] <= -(-ia["cycles"] // 64) + 1 and ia["graph_launches"] < ia["cycles"]
    assert ia["df_cycles"] == ib["df_cycles"] > 0
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    for x, y in zip(ra, rb):
        assert x["sweeps"] == y["sweeps"] and x["residual"] == y["residual"]


def test_batched_two_sweep_pass_and_one_sweep_kernel_reach_the_oracle():
    """The batched two-sweep TMA pass (per-lattice tensor maps in global memory, items of
    every lattice in one launch) and the one-sweep kernel over every lattice both reach
    the oracle's steady states."""
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()
    refs = [soc.steady_state(soc.assemble(problem_from_case(c, soc))) for c in cases]
    for kernel in ("blocked", "plain"):
        solvers = [rfb.Solver.from_case(c) for c in cases]
        try:
            with rfb.Batch(solvers) as b:
                res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                    [1e-10] * len(cases), fp32_kernel=kernel)
            if kernel == "blocked":
                assert info["sweeps_per_cycle"] % 4 == 0
            assert 0 < info["df_cycles"] <= info["cycles"]
            for c, r, sv, ref in zip(cases, res, solvers, refs):
                assert r["residual"] <= 1e-10
                assert np.abs(sv.get_state() - ref).max() < 1e-6, (kernel, c.name)
        finally:
            for s in solvers:
                s.close()


def test_batch_second_solve_reuses_tuning_and_warm_starts():
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()[:3]
    solvers = [rfb.Solver.from_case(c) for c in cases]
    try:
        with rfb.Batch(solvers) as b:
            args = ([c.s_in for c in cases], [c.eta for c in cases], [1e-9] * 3)
            r1, i1 = b.solve(*args)
            r2, i2 = b.solve(*args)       # warm start from the converged states
            assert i2["kchunk"] == i1["kchunk"]
            assert all(r["sweeps"] == 0 for r in r2)
            assert all(abs(a["I_tot"] - c["I_tot"]) <= 1e-9 * abs(a["I_tot"])
                       for a, c in zip(r1, r2))
    finally:
        for s in solvers:
            s.close()


def test_batch_rejects_fp64_and_bad_lattices():
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()[:2]
    solvers = [rfb.Solver.from_case(c) for c in cases]
    try:
        with rfb.Batch(solvers) as b:
            with pytest.raises(rfb.RfbError) as e:
                b.solve([0.5, 0.5], [-0.1, -0.1], [1e-8, 1e-8], precision="fp64")
            assert e.value.status == rfb.RFB_ERR_UNSUPPORTED
            with pytest.raises(rfb.RfbError):
                b.solve([1.5, 0.5], [-0.1, -0.1], [1e-8, 1e-8])
        with pytest.raises(rfb.RfbError):
            rfb.Batch([solvers[0], solvers[0]])
    finally:
        for s in solvers:
            s.close()


def test_batched_workload_48_lattices_full_size():
    """The batched workload at full size: 48 lattices from 64^3 to 192x192x384 (187M
    cells), porosity U[0.75, 0.9], log-uniform flow, uniform s_in and eta, residual
    1e-8, in one batch. Every lattice converges with a consistent mass balance; the 64^3
    lattice matches the oracle element by element (1e-6 max-abs)."""
    from paper_2502_08034_gb300 import rfb, synth
    cases = synth.batch_cases(48, flow_device="cuda", tol=1e-8)
    solvers = [rfb.Solver.from_case(c, device_inputs=True) for c in cases]
    try:
        with rfb.Batch(solvers) as b:
            res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                [1e-8] * len(cases))
        cells = sum(c.n * r["sweeps"] for c, r in zip(cases, res))
        print("batch: %d lattices, %.1f M cells, %.3f s until the last converged, "
              "%.1f GCell-updates/s, kchunk %d, %d sweeps/cycle, sweep %.3f ms, check %.3f ms"
              % (len(cases), sum(c.n for c in cases) / 1e6, info["time_ms"] / 1e3,
                 cells / info["time_ms"] / 1e6, info["kchunk"], info["sweeps_per_cycle"],
                 info["sweep_ms"], info["check_ms"]))
        for c, r in zip(cases, res):
            assert r["residual"] <= 1e-8, c.name
            assert r["mass_balance_rel"] < 1e-4, (c.name, r["mass_balance_rel"])
        s0 = solvers[0].get_state()
    finally:
        for s in solvers:
            s.close()
    ref = soc.steady_state(soc.assemble(problem_from_case(cases[0], soc)))
    assert np.abs(s0 - ref).max() < 1e-6


def test_batched_pass_64_and_128_column_tiles_are_the_same_sweeps():
    """The batched two-sweep pass with 64-column tiles (two CTAs per SM) and with
    128-column tiles, on lattices several narrow tiles wide with ragged last tiles in x and
    y: the same bits for the same cycles, and the oracle's steady states."""
    from paper_2502_08034_gb300 import rfb, synth
    dims = [(100, 28, 20), (148, 16, 24), (68, 30, 18)]
    cases = [synth.build_case("bt%dx%dx%d" % d, d, 0.8, 4.0, 11 + q, 0.01, -0.1, 0.4, 1e-10)
             for q, d in enumerate(dims)]
    refs = [soc.steady_state(soc.assemble(problem_from_case(c, soc))) for c in cases]
    out = []
    for kernel in (3, 7):                   # 128-column tiles, 64-column tiles
        solvers = [rfb.Solver.from_case(c) for c in cases]
        try:
            with rfb.Batch(solvers) as b:
                res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                    [1e-10] * len(cases), fp32_kernel=kernel, check_every=40)
            assert info["pass_tile_cols"] == (128 if kernel == 3 else 64)
            assert info["pass_stages"] > 0
            out.append(([s.get_state() for s in solvers], [r["sweeps"] for r in res]))
            for c, r, sv, ref in zip(cases, res, solvers, refs):
                assert r["residual"] <= 1e-10
                assert np.abs(sv.get_state() - ref).max() < 1e-7, (kernel, c.name)
        finally:
            for s in solvers:
                s.close()
    (sa, na), (sb, nb) = out
    assert na == nb
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


def test_batch_below_the_double_float_floor_finishes_with_fp64_checks():
    """A tolerance below what double-float defects resolve (10 x tau 2^-44 max_c d_c): the
    batch leaves the double-float cycles at that level and finishes with FP64 checks, at
    the oracle's steady states."""
    from paper_2502_08034_gb300 import rfb
    cases = _small_batch()[:2]
    refs = [soc.steady_state(soc.assemble(problem_from_case(c, soc))) for c in cases]
    solvers = [rfb.Solver.from_case(c) for c in cases]
    try:
        with rfb.Batch(solvers) as b:
            res, info = b.solve([c.s_in for c in cases], [c.eta for c in cases],
                                [1e-12] * len(cases))
        assert 0 < info["df_cycles"] < info["cycles"]
        for r, sv, ref in zip(res, solvers, refs):
            assert r["residual"] <= 1e-12
            assert np.abs(sv.get_state() - ref).max() < 1e-9
    finally:
        for s in solvers:
            s.close()
