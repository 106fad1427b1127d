"""The temporally blocked, TMA-staged FP32 correction passes (two sweeps, and with local
steps three sweeps with tensor-memory coefficients) are bitwise the same number of
one-sweep launches, on lattices with several tiles, ragged tile edges in y, odd z extents
and both pseudo-time step modes, for the operator and its transpose; and mixed-precision
solves with them match the oracle."""
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


# the step-field pass variants (local steps only)
THREE_AND_FOUR = ["blocked4_persistent", "blocked4_chunked", "three_sweep_persistent",
                  "three_sweep_chunked", "three_sweep5_persistent", "three_sweep5_chunked"]


@functools.lru_cache(maxsize=None)
def _case(dims, seed=7, d=4.0):
    from paper_2502_08034_gb300 import synth
    return synth.build_case("tb%dx%dx%d" % dims, dims, 0.82, d, seed, 0.01, -0.10, 0.4, 1e-10)


@pytest.mark.parametrize("dims", [(48, 48, 96), (64, 40, 37), (144, 30, 21), (256, 32, 16)])
@pytest.mark.parametrize("dt_mode", ["local", "global"])
def test_two_sweep_pass_is_bitwise_two_sweeps(dims, dt_mode):
    """Both launch shapes (persistent shares that cross tiles and chunked items with a
    padded last chunk) give the same bits as one-sweep launches."""
    from paper_2502_08034_gb300 import rfb
    case = _case(dims)
    states = []
    kernels = ["plain", "blocked_persistent", "blocked_chunked", "blocked"]
    if dt_mode == "local":      # the step-field passes: four TMA stages, three sweeps
        kernels += THREE_AND_FOUR
    for kernel in kernels:
        with rfb.Solver.from_case(case) as sv:
            for n in (6, 10, 4):      # several correction cycles
                sv.step(case.s_in, case.eta, n, precision="mixed", dt_mode=dt_mode,
                        fp32_kernel=kernel)
            states.append(sv.get_state())
    for st in states[1:]:
        assert np.array_equal(states[0], st)


def test_two_sweep_pass_odd_count():
    """An odd sweep count ends with one one-sweep launch."""
    from paper_2502_08034_gb300 import rfb
    case = _case((64, 40, 37))
    out = []
    for kernel in ("plain", "blocked_persistent", "blocked_chunked"):
        with rfb.Solver.from_case(case) as sv:
            sv.step(case.s_in, case.eta, 7, precision="mixed", fp32_kernel=kernel)
            out.append(sv.get_state())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_umt_with_two_sweep_passes_matches_oracle():
    from paper_2502_08034_gb300 import rfb
    case = _case((48, 48, 96))
    ref = soc.umt(problem_from_case(case, soc))
    with rfb.Solver.from_case(case) as sv:
        u, _ = sv.umt(1e-11, precision="mixed", fp32_kernel="blocked")
    assert abs(u - ref) < 1e-7


@pytest.mark.parametrize("dims", [(48, 48, 96), (64, 40, 37)])
def test_mixed_solve_with_two_sweep_passes_matches_oracle(dims):
    from paper_2502_08034_gb300 import rfb
    case = _case(dims)
    ref = soc.steady_state(soc.assemble(problem_from_case(case, soc)))
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-11, precision="mixed", fp32_kernel="blocked")
        s = sv.get_state()
    assert r["residual"] <= 1e-11
    assert np.abs(s - ref).max() < 1e-7


def test_two_sweep_pass_eligibility():
    """Local steps: the step-field pass takes nx % 4 == 0 and area multipliers (they enter
    through the step only); the global step keeps the mask-byte pass's nx % 16 == 0 and
    no multiplier; lattices outside that fall back to one-sweep launches under auto."""
    from paper_2502_08034_gb300 import rfb, synth
    case = _case((36, 20, 24))
    with rfb.Solver.from_case(case) as sv:
        sv.solve(case.s_in, case.eta, 1e-8, precision="mixed", fp32_kernel="blocked")
        with pytest.raises(rfb.RfbError) as e:
            sv.solve(case.s_in, case.eta, 1e-8, precision="mixed", fp32_kernel="blocked",
                     dt_mode="global")
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
    c2 = _case((48, 48, 96))
    m = synth.lognormal_area_mult(c2.solid)
    with rfb.Solver.from_case(c2, area_mult=m) as sv:
        sv.solve(c2.s_in, c2.eta, 1e-8, precision="mixed", fp32_kernel="blocked")
        with pytest.raises(rfb.RfbError):
            sv.solve(c2.s_in, c2.eta, 1e-8, precision="mixed", fp32_kernel="blocked",
                     dt_mode="global")
        sv.solve(c2.s_in, c2.eta, 1e-8, precision="mixed", dt_mode="global")   # auto


@pytest.mark.parametrize("dims", [(36, 20, 24), (52, 44, 30)])
def test_step_field_pass_is_bitwise_with_area_multipliers_and_nx_multiple_of_4(dims):
    """The step-field pass (local steps) on lattices whose nx is a multiple of 4 but not
    of 16, with lognormal area multipliers: both launch shapes give the bits of one-sweep
    launches."""
    from paper_2502_08034_gb300 import rfb, synth
    case = _case(dims)
    m = synth.lognormal_area_mult(case.solid, 0.3, 40)
    states = []
    for kernel in ["plain", "blocked_persistent", "blocked_chunked"] + THREE_AND_FOUR:
        with rfb.Solver.from_case(case, area_mult=m) as sv:
            for n in (6, 9):
                sv.step(case.s_in, case.eta, n, precision="mixed", fp32_kernel=kernel)
            states.append(sv.get_state())
    for st in states[1:]:
        assert np.array_equal(states[0], st)


@pytest.mark.parametrize("dims", [(48, 48, 96), (64, 40, 37), (144, 30, 21)])
def test_transposed_passes_are_bitwise_the_same_sweeps(dims):
    """Mixed adjoint corrections (transposed operator) through the two-sweep and the
    three-sweep passes: with 12 sweeps per cycle (whole passes of either) the adjoint and
    its gradients are the same bits."""
    from paper_2502_08034_gb300 import rfb, synth
    case = _case(dims)
    m = synth.lognormal_area_mult(case.solid, 0.3, 40)
    outs = []
    for kernel in ["blocked_chunked"] + THREE_AND_FOUR:
        with rfb.Solver.from_case(case, area_mult=m) as sv:
            # 6 mixed sweeps choose the pass variant (the same bits for every variant)
            sv.step(case.s_in, case.eta, 6, precision="mixed", fp32_kernel=kernel)
            sv.solve(case.s_in, case.eta, 1e-13, precision="fp64", max_sweeps=400000)
            dm, db, r = sv.adjoint("I_tot", 1e-11, precision="mixed", check_every=12)
            outs.append((dm.copy(), db, r["sweeps"]))
    for dm, db, n in outs[1:]:
        assert n == outs[0][2] and db == outs[0][1] and np.array_equal(dm, outs[0][0])


def test_three_sweep_pass_mixed_solve_matches_oracle():
    """A mixed solve through the three-sweep pass reaches the oracle's steady state."""
    from paper_2502_08034_gb300 import rfb
    case = _case((64, 40, 37))
    ref = soc.steady_state(soc.assemble(problem_from_case(case, soc)))
    for kernel in ("three_sweep_persistent", "three_sweep_chunked"):
        with rfb.Solver.from_case(case) as sv:
            r = sv.solve(case.s_in, case.eta, 1e-11, precision="mixed", fp32_kernel=kernel)
            assert sv.tuned_fp32_kernel()[0] == kernel
            s = sv.get_state()
        assert r["residual"] <= 1e-11
        assert np.abs(s - ref).max() < 1e-7
