"""Pins of the Butler-Volmer oracle (oracle/bv.py; no GPU): what the paper and the
mathematics fix, independently of the oracle's own code paths.

- The source equals the Butler-Volmer rate of Eq. source-term-bv1 with the overpotential
  of Eq. etat-from-s-bv (and the sinh form of Eq. source-term-bv at alpha = 1/2).
- With the potential held at 0 the first fixed-point step is the SBV model exactly
  (Sec. II.D: SBV disregards phi_L): C_O + C_R = c0 everywhere and C_R / c0 is the SBV
  steady state.
- At the fixed point every species balance holds, and so does the counter-ion's, which
  the model never solves for: the potential equation is the discrete charge balance and
  electroneutrality closes it.
- Summed over the lattice, the potential equation telescopes: the protons' migration
  current through the membrane equals I_tot minus the diffusion current at the inlet.
- C_O + C_R has no source: its inflow equals its outflow.
- A stronger supporting electrolyte (more protons, larger kappa_L) shrinks phi_L like
  1 / kappa and brings the state to the SBV one (Sec. II.C: with a strong supporting
  electrolyte kappa_L is large and phi_L small).
"""
import dataclasses
import functools
import math

import numpy as np
import pytest

from oracle import bv, soc
from tests._cases import fiber_case, problem_from_case


@functools.lru_cache(maxsize=None)
def _problem(dims=(8, 8, 12), k0=2e-5, eta=-0.10, s_in=0.2):
    return problem_from_case(fiber_case(dims, diameter=4.0, u_mean=0.002), soc, k0=k0,
                             eta=eta, s_in=s_in)


@functools.lru_cache(maxsize=None)
def _solved(dims=(8, 8, 12), c_H_in=None):
    p = _problem(dims)
    q = bv.BVParams(c_H_in=c_H_in)
    s0 = soc.steady_state(soc.assemble(p))
    C, phi, it = bv.solve(p, q, s0=s0, tol=1e-12)
    return p, q, s0, C, phi, it


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_source_is_the_butler_volmer_rate(alpha):
    p = dataclasses.replace(_problem(), alpha=alpha)
    rng = np.random.default_rng(1)
    N = p.solid.size
    phi = rng.uniform(-2e-3, 2e-3, N)
    CO = rng.uniform(1.0, 19.0, N)
    CR = rng.uniform(1.0, 19.0, N)
    kf, kb = bv.rate_coefficients(p, phi)
    S = kf * CO - kb * CR
    V_T = soc.R_GAS * p.T / soc.FARADAY
    Vt = p.n_e * (-p.eta) / V_T
    phit = -p.n_e * phi / V_T
    etat = Vt - phit - np.log(CR / CO)               # Eq. etat-from-s-bv
    nw = soc.n_wall(p.solid.astype(bool)).ravel()
    a = np.where(p.solid.ravel() == 0, nw / p.h, 0.0)
    ref = a * p.k0 * CO ** (1 - alpha) * CR ** alpha * (np.exp(alpha * etat) -
                                                        np.exp((alpha - 1) * etat))
    assert np.allclose(S, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    if alpha == 0.5:
        CT = CO + CR
        s = CR / CT
        sinh_form = 2 * a * p.k0 * CT * np.sqrt(s * (1 - s)) * np.sinh(etat / 2)
        assert np.allclose(S, sinh_form, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_zero_potential_step_is_the_sbv_model():
    p = _problem()
    q = bv.BVParams()
    s_sbv = soc.steady_state(soc.assemble(p))
    C, _ = bv.fixed_point_step(p, q, np.zeros(p.solid.size))
    fl = p.solid.ravel() == 0
    assert np.abs(C["O"][fl] + C["R"][fl] - p.c0).max() <= 1e-12 * p.c0
    assert np.abs(C["R"][fl] / p.c0 - s_sbv[fl]).max() <= 1e-12


def test_fixed_point_balances_every_species_and_the_counter_ion():
    p, q, _, C, phi, _ = _solved()
    r = bv.species_rhs(p, q, C, phi)
    Dk = bv.diffusivities(p, q)
    for k in ("O", "R", "H", "X"):
        scale = Dk[k] / p.h ** 2 * np.abs(C[k]).max()     # size of one diffusion term
        assert np.abs(r[k]).max() <= 1e-10 * scale, k
    pr = bv.potential_residual(p, q, C, phi)
    scale = p.n_e * soc.FARADAY * float(np.abs(bv.rate_coefficients(p, phi)[0]).max()) * p.c0
    assert np.abs(pr).max() <= 1e-10 * scale
    fl = p.solid.ravel() == 0
    assert np.all(bv.counter_ion(C)[fl] > 0)


def test_membrane_current_balances_the_reaction_current():
    p, q, _, C, phi, _ = _solved()
    o = bv.outputs(p, q, C, phi)
    cin = bv.inlet(p, q)
    Dk = bv.diffusivities(p, q)
    fin = p.solid[0] == 0
    nxny = p.solid.shape[1] * p.solid.shape[2]
    inlet_diff = 0.0
    for k in ("O", "R", "H", "X"):
        ck = C[k][:nxny].reshape(p.solid.shape[1:])
        inlet_diff += bv.Z[k] * Dk[k] * float(np.sum(np.where(fin, 2 * (cin[k] - ck) / p.h, 0.0)))
    inlet_current = soc.FARADAY * inlet_diff * p.h * p.h
    assert abs(o["I_membrane"] - (o["I_tot"] - inlet_current)) <= 1e-9 * abs(o["I_tot"])
    assert o["I_tot"] > 0


def test_quinone_total_is_conserved():
    p, q, _, C, phi, _ = _solved()
    nz, ny, nx = p.solid.shape
    CT = (C["O"] + C["R"]).reshape(nz, ny, nx)
    cin = bv.inlet(p, q)
    fin, fout = p.solid[0] == 0, p.solid[-1] == 0
    w_in, w_out = p.W[0], p.W[-1]
    inflow = float(np.sum(np.where(fin, w_in * (cin["O"] + cin["R"]) +
                                   2 * p.D / p.h * (cin["O"] + cin["R"] - CT[0]), 0.0)))
    outflow = float(np.sum(np.where(fout, w_out * CT[-1], 0.0)))
    assert abs(inflow - outflow) <= 1e-11 * abs(inflow)


def test_strong_supporting_electrolyte_reaches_the_sbv_state():
    fl = _problem().solid.ravel() == 0
    d, phis = [], []
    for ratio in (50.0, 500.0, 5000.0):
        p, q, s0, C, phi, _ = _solved(c_H_in=ratio * 20.0)
        o = bv.outputs(p, q, C, phi)
        d.append(float(np.abs(o["s"][fl] - s0[fl]).max()))
        phis.append(float(np.abs(phi[fl]).max()))
    assert d[0] > 0 and phis[0] > 0
    # phi ~ 1 / kappa, and the state difference with it
    assert 5 < phis[0] / phis[1] < 15 and 5 < phis[1] / phis[2] < 15
    assert d[1] < 0.2 * d[0] and d[2] < 0.2 * d[1]
