"""The 256x256x512 mixed-precision workload at full size, in the launch configuration the
benchmark times (autotuned FP32 kernel, local steps, residual 1e-8). The oracle cannot
solve 33.5M cells directly, so it is checked where it can compute outputs one by one: on
sampled interior z-planes the oracle assembles the operator of a 3-plane slab from the
same inputs, and its RHS on the GPU state at the middle plane (exactly the full
operator's rows there) must be at the tolerance's level. Properties that hold at any size
complete it: the mixed state within 1e-6 of the FP64 path after the same number of
sweeps (restarting the correction iteration each check cycle follows the trajectory of
the plain iteration, so the two differ by FP32 rounding only), mass balance, bounds. The
element-wise comparison with the oracle's steady state at this size is in
test_gpu_fullsize_golden.py."""
import functools

import numpy as np
import pytest

from oracle import soc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


@functools.lru_cache(maxsize=None)
def _case():
    from paper_2502_08034_gb300 import synth
    return synth.large_mixed_case(flow_device="cuda")


def _slab_rhs(case, s3, k):
    """Oracle RHS at plane k (1 <= k <= nz - 2) from the slab of planes k-1 .. k+1."""
    sl = slice(k - 1, k + 2)
    p = soc.Problem(case.solid[sl], case.U[sl], case.V[sl], case.W[k - 1:k + 3], case.h,
                    case.D, case.s_in, k0=case.k0, eta=case.eta)
    op = soc.assemble(p)
    r = (op.L @ s3[sl].ravel() + op.b).reshape(3, case.solid.shape[1], case.solid.shape[2])
    fluid = case.solid[k] == 0
    return r[1][fluid]


def test_mixed_workload_256x256x512_full_size():
    from paper_2502_08034_gb300 import rfb
    case = _case()
    nz = case.solid.shape[0]
    with rfb.Solver.from_case(case, device_inputs=True) as sv:
        r = sv.solve(case.s_in, case.eta, case.tol, precision="mixed")
        s_mixed = sv.get_state()
        kname, _, _ = sv.tuned_fp32_kernel()
        sv.reset_state()
        r64 = sv.step(case.s_in, case.eta, r["sweeps"], precision="fp64")
        s64 = sv.get_state()
    assert kname is not None and r["residual"] <= case.tol
    fluid = case.solid.ravel() == 0
    # the FP32-corrected state against the FP64 path after the same sweeps (the
    # mixed-precision target: 1e-6)
    diff = float(np.abs(s_mixed[fluid] - s64[fluid]).max())
    print("256x256x512 %s: %d sweeps, mixed - FP64 max %.2e" % (kname, r["sweeps"], diff))
    assert diff <= 1e-6
    assert abs(r["I_tot"] - r64["I_tot"]) <= 1e-6 * abs(r64["I_tot"])
    # conservation and the maximum principle at full size
    assert r["mass_balance_rel"] <= 1e-6
    kin = soc.kinetics(case.eta)
    lo, hi = min(case.s_in, kin.s_eq), max(case.s_in, kin.s_eq)
    assert s_mixed[fluid].min() >= lo - 1e-7 and s_mixed[fluid].max() <= hi + 1e-7
    # the oracle's own rows on sampled planes: tau RMS(RHS) at the tolerance's level
    s3 = s_mixed.reshape(case.solid.shape)
    rng = np.random.default_rng(17)
    planes = sorted(set(rng.integers(1, nz - 1, 6).tolist()) | {1, nz // 2, nz - 2})
    rhs = np.concatenate([_slab_rhs(case, s3, k) for k in planes])
    assert r["tau"] * np.sqrt(np.mean(rhs ** 2)) <= 10 * case.tol
