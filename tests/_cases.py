"""Small seeded workloads shared by the tests (built once per process)."""
import functools

import numpy as np

from paper_2502_08034_gb300 import synth


@functools.lru_cache(maxsize=None)
def fiber_case(dims=(16, 16, 32), seed=1, porosity=0.80, diameter=8.0, u_mean=0.01,
               eta=-0.10, s_in=0.5):
    return synth.fiber_channel_case(dims=dims, seed=seed, porosity=porosity,
                                    diameter=diameter, u_mean=u_mean, eta=eta, s_in=s_in)


@functools.lru_cache(maxsize=None)
def mixed_case_small(dims=(32, 32, 64), seed=2):
    return synth.large_mixed_case(dims=dims, seed=seed)


def channel_1d(n=40, w=0.01, h=1.25e-6):
    """3 x 3 x n lattice whose outer ring is fiber: the centre column is a 1D channel
    with uniform velocity w and four fiber neighbours in every cell."""
    nx = ny = 3
    solid = np.ones((n, ny, nx), dtype=np.uint8)
    solid[:, 1, 1] = 0
    U = np.zeros((n, ny, nx + 1))
    V = np.zeros((n, ny + 1, nx))
    W = np.zeros((n + 1, ny, nx))
    W[:, 1, 1] = w
    return solid, U, V, W, h


def problem_from_case(case, soc, **over):
    kw = dict(solid=case.solid, U=case.U, V=case.V, W=case.W, h=case.h, D=case.D,
              s_in=case.s_in, k0=case.k0, alpha=case.alpha, n_e=case.n_e, T=case.T,
              c0=case.c0, eta=case.eta)
    kw.update(over)
    return soc.Problem(**kw)
