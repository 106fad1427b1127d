"""Failure detection on the GPU without a fault: the bounded mbarrier wait of the
two-sweep pass gives up on a barrier that nothing completes, records the error and lets
its kernel finish, and the context stays usable for the next solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_08034_gb300 import _build
    _build.build()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    from paper_2502_08034_gb300 import rfb, synth
    assert rfb.selftest_bounded_wait(1 << 12)
    assert rfb.selftest_bounded_wait(1)
    case = synth.fiber_channel_case(dims=(16, 16, 32), diameter=4.0)
    with rfb.Solver.from_case(case) as sv:
        r = sv.solve(case.s_in, case.eta, 1e-10, precision="mixed", fp32_kernel="blocked")
        assert r["residual"] <= 1e-10 and np.all(np.isfinite(sv.get_state()))


def test_bounded_wait_arguments():
    from paper_2502_08034_gb300 import rfb
    for bad in (0, -5, (1 << 26) + 1):
        with pytest.raises(rfb.RfbError) as e:
            rfb.selftest_bounded_wait(bad)
        assert e.value.status == rfb.RFB_ERR_INVALID_ARG
