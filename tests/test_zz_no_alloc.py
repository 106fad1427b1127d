"""rfb_soc_current_noalloc: outputs evaluated with a static device scratch array instead
of allocated memory, for callers that cannot allocate device memory when they need the
outputs (an external caching allocator owns the device, or cudaMalloc's implicit
synchronisation is not acceptable on their path).

Checked through the C ABI against rfb_soc_current on two calls in a row (the second call
finds the previous call's contents in the shared array), on two different lattices, and
for the size limit. This file is collected last so that a failure here comes after every
other test has run.
"""
import ctypes

import numpy as np
import pytest

from tests._cases import fiber_case, mixed_case_small

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-12   # matrix-free vs assembled FP64 check, same reduction order: equal up to
              # rounding


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


def _compare(a, b):
    for k in ("residual", "I_tot", "F_in", "F_out", "F_in_adv", "U", "outlet_mean"):
        assert a[k] == pytest.approx(b[k], rel=REL, abs=0.0), k
    assert a["nonfinite"] == b["nonfinite"] == 0


def _raw_noalloc(sv):
    from paper_2502_08034_gb300 import rfb
    r = rfb.SolveResult()
    st = rfb.lib().rfb_soc_current_noalloc(sv.h, ctypes.byref(r))
    assert st == rfb.RFB_OK, rfb.lib().rfb_soc_last_error(sv.h)
    return r.as_dict()


def test_noalloc_matches_current_on_consecutive_calls():
    from paper_2502_08034_gb300 import rfb
    a_case = fiber_case((16, 16, 32))
    b_case = mixed_case_small((32, 32, 64))
    with rfb.Solver.from_case(a_case) as a, rfb.Solver.from_case(b_case) as b:
        a.step(a_case.s_in, a_case.eta, 150)
        b.step(b_case.s_in, b_case.eta, 90, precision="mixed")
        ref_a, ref_b = a.current(), b.current()
        first = _raw_noalloc(a)
        second = _raw_noalloc(a)
        _compare(first, ref_a)
        _compare(second, ref_a)
        # another lattice in between: the scratch then holds b's partial sums
        _compare(_raw_noalloc(b), ref_b)
        _compare(_raw_noalloc(a), ref_a)


def test_noalloc_on_a_converged_state():
    """Near steady state the residual is a sum of cancelling terms, so the matrix-free
    check (this entry point) and the assembled-operator check (rfb_soc_current) differ by
    rounding relative to the terms, not to the residual: a cell's RHS combines terms up
    to max_c d_c |s| ~ 1e4 s^-1 here, so the two residuals may differ by about
    tau * 1e4 * 1e-15; the other outputs are sums of large terms and agree to 1e-12."""
    from paper_2502_08034_gb300 import rfb
    case = fiber_case((16, 16, 32))
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-11, precision="fp64")
        ref = sv.current()
        for _ in range(2):
            got = _raw_noalloc(sv)
            assert got["residual"] <= 1e-11
            assert abs(got["residual"] - ref["residual"]) <= ref["tau"] * 1e-11
            for k in ("I_tot", "F_in", "F_out", "F_in_adv", "U", "outlet_mean"):
                assert got[k] == pytest.approx(ref[k], rel=REL, abs=0.0), k
    assert r["residual"] <= 1e-11


def test_noalloc_after_a_umt_solve_at_another_velocity_scale():
    """The outputs belong to the last solve's operating point, velocity scale included,
    after a U_mt solve at another scale (which rescales the shared velocity copies)."""
    from paper_2502_08034_gb300 import rfb
    case = fiber_case((16, 16, 32))
    with rfb.Solver.from_case(case) as sv:
        sv.step(case.s_in, case.eta, 150, velocity_scale=1.0)
        before = _raw_noalloc(sv)
        sv.umt(1e-10, precision="fp64", velocity_scale=2.0)
        _compare(_raw_noalloc(sv), before)
        _compare(sv.current(), before)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_2502_08034_gb300 import rfb
    nx = ny = 2048
    nz = 2
    solid = np.zeros((nz, ny, nx), np.uint8)
    U = np.zeros((nz, ny, nx + 1))
    V = np.zeros((nz, ny + 1, nx))
    W = np.zeros((nz + 1, ny, nx))
    with rfb.Solver((nx, ny, nz), 1e-6, solid, U, V, W, 4e-10, 1e-7) as sv:
        sv.step(0.5, -0.05, 1)
        with pytest.raises(rfb.RfbError) as e:
            sv.current_noalloc()
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
        assert "static scratch" in str(e.value)
        sv.current()   # the allocated path still serves this lattice
