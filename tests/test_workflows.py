"""Host logic of the upsampling chain (Sec. III.A), without a GPU: the coarsest level
starts cold, every finer level is prolonged from the one before it and solved warm, and
U_mt is taken on the finest level only."""
from types import SimpleNamespace

from paper_2502_08034_gb300 import workflows


class _Level:
    def __init__(self, name, log):
        self.name, self.log = name, log

    def reset_state(self):
        self.log.append(("reset", self.name))

    def upsample_from(self, coarse):
        self.log.append(("upsample", coarse.name, self.name))

    def solve(self, s_in, eta, tol, precision):
        self.log.append(("solve", self.name, s_in, eta, tol, precision))
        return {"level": self.name}

    def umt(self, tol, precision):
        self.log.append(("umt", self.name, tol, precision))
        return 0.75, {}


def test_chain_order_and_outputs():
    log = []
    levels = [_Level(n, log) for n in ("128", "256", "512")]
    cases = [SimpleNamespace(s_in=0.5, eta=-0.1) for _ in levels]
    out, u = workflows.upsample_chain(levels, cases, 1e-8, precision="mixed")
    assert [r["level"] for r in out] == ["128", "256", "512"]
    assert u == (0.75, {})
    assert log == [
        ("reset", "128"), ("solve", "128", 0.5, -0.1, 1e-8, "mixed"),
        ("upsample", "128", "256"), ("solve", "256", 0.5, -0.1, 1e-8, "mixed"),
        ("upsample", "256", "512"), ("solve", "512", 0.5, -0.1, 1e-8, "mixed"),
        ("umt", "512", 1e-8, "mixed"),
    ]


def test_chain_without_umt():
    log = []
    levels = [_Level("a", log), _Level("b", log)]
    cases = [SimpleNamespace(s_in=0.3, eta=-0.05)] * 2
    out, u = workflows.upsample_chain(levels, cases, 1e-6, umt=False, precision="fp64")
    assert u is None and len(out) == 2
    assert not any(e[0] == "umt" for e in log)
