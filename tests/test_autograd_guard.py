"""The autograd bridge's backward differentiates the solver handle's current states, so it
must refuse to run once the solver has been used again after its forward (no GPU: the C
library is replaced by a stand-in that returns success, and the solver by a duck-typed
stand-in where the bridge itself is tested)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2502_08034_gb300 import rfb  # noqa: E402
from paper_2502_08034_gb300.autograd import soc_objective  # noqa: E402


class _OkLib:
    """Every entry point returns RFB_OK and leaves its outputs as they are."""

    def rfb_soc_last_error(self, h):
        return b""

    def __getattr__(self, name):
        return lambda *a: rfb.RFB_OK


def test_every_state_changing_call_advances_the_generation(monkeypatch):
    monkeypatch.setattr(rfb, "lib", lambda: _OkLib())
    sv = object.__new__(rfb.Solver)
    sv.h, sv.n_cells, sv.state_generation = None, 8, 0
    other = object.__new__(rfb.Solver)
    other.h, other.n_cells, other.state_generation = None, 1, 0
    changing = [
        lambda: sv.solve(0.5, -0.1, 1e-8),
        lambda: sv.step(0.5, -0.1, 4),
        lambda: sv.solve_nernst(0.5, -0.1, 1e-8),
        lambda: sv.solve_bv(0.5, -0.1, 1e-8),
        lambda: sv.umt(1e-8),
        lambda: sv.set_state(np.zeros(8)),
        lambda: sv.set_area_mult(np.ones(8)),
        lambda: sv.set_area_mult(None),
        lambda: sv.upsample_from(other),
        lambda: sv.reset_state(),
    ]
    for k, call in enumerate(changing, start=1):
        call()
        assert sv.state_generation == k
    # reading the state or outputs, and the adjoint itself, change nothing
    sv.current()
    sv.current_noalloc()
    sv.get_state()
    sv.adjoint("I_tot", 1e-8)
    assert sv.state_generation == len(changing)
    b = object.__new__(rfb.Batch)
    b.b, b.solvers = None, [sv, other]
    b.solve([0.5, 0.5], [-0.1, -0.1], [1e-8, 1e-8])
    assert sv.state_generation == len(changing) + 1 and other.state_generation == 1
    sv.h = other.h = None


class _FakeSolver:
    """Duck-typed solver: I_tot = 1, U = 0.5, U_mt = 0.9; the adjoint of objective j is
    the constant field j (1, 2, 3) with dJ/dbeta = 0.25 j."""

    def __init__(self, n):
        self.n, self.state_generation, self.adjoints = n, 0, []

    def set_area_mult(self, m):
        self.state_generation += 1

    def solve(self, s_in, eta, tol, **kw):
        self.state_generation += 1
        return {"I_tot": 1.0, "U": 0.5}

    def umt(self, tol, **kw):
        self.state_generation += 1
        return 0.9, {}

    def adjoint(self, obj, tol, out=None, **kw):
        j = {"I_tot": 1.0, "U": 2.0, "U_mt": 3.0}[obj]
        self.adjoints.append(obj)
        return np.full(self.n, j), 0.25 * j, {}


def test_backward_is_the_weighted_sum_of_the_adjoints():
    sv = _FakeSolver(6)
    m = torch.ones(6, dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    I, U, Umt = soc_objective(sv, m, beta, 0.5, -0.1, 1e-8)
    (3.0 * I + 0.5 * U).backward()
    assert sv.adjoints == ["I_tot", "U"]               # no adjoint for a zero gradient
    assert torch.equal(m.grad, torch.full((6,), 3.0 * 1.0 + 0.5 * 2.0, dtype=torch.float64))
    assert float(beta.grad) == 3.0 * 0.25 + 0.5 * 0.5


def test_backward_refuses_after_the_solver_was_used_again():
    sv = _FakeSolver(4)
    m1 = torch.ones(4, dtype=torch.float64, requires_grad=True)
    m2 = torch.full((4,), 2.0, dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(1.0, dtype=torch.float64)
    I1, _, _ = soc_objective(sv, m1, beta, 0.5, -0.1, 1e-8)
    I2, _, _ = soc_objective(sv, m2, beta, 0.5, -0.1, 1e-8)
    with pytest.raises(RuntimeError, match="used again after this forward"):
        I1.backward()
    assert sv.adjoints == []
    I2.backward()                                       # the latest forward still works
    assert sv.adjoints == ["I_tot"]
