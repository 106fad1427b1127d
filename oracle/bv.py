"""CPU oracle of the Butler-Volmer model with electromigration (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module. The product path (the CUDA library behind ``include/rfb_soc.h``)
shares no code with it.

What it computes, in FP64, following the paper (arXiv 2502.08034), Sec. II.C and III.B:

* Species (Eq. nernst-planck): the oxidised and reduced quinone O, R (charge -2, the same
  diffusivity D) and protons H (charge +1, D_H) are solved for; the counter-ion
  HSO4- (X, charge -1, D_X) follows from electroneutrality (Eq. electroneutrality),
  C_X = C_H - 2 (C_O + C_R). The reaction O + 2 H+ + 2 e- -> R has stoichiometric numbers
  n_O = -1, n_R = +1, n_H = -2.
* Source (Eqs. source-term-bv1 and etat-from-s-bv): with eta~ = V~ - phi~_L - logit(s),
  phi~_L = -n_e phi_L / V_T, the Butler-Volmer rate per volume is
  S = a k0 C_O^(1-alpha) C_R^alpha (e^{alpha eta~} - e^{(alpha-1) eta~})
    = a k0 (C_O e^{alpha V~_c} - C_R e^{(alpha-1) V~_c}),  V~_c = V~ + n_e phi_L / V_T,
  linear in the concentrations at a given potential (a = m n_wall / h as in soc.py).
* Potential (Eq. poisson-phi with Eq. kappa, in the form div(kappa grad phi) that
  Algorithm 2 solves): div(kappa_L grad phi_L) = n_e F S - F sum_k z_k D_k lap C_k, over
  all four species.

Discretisation (readings stated once; the transport stencil is soc.py's):
* advection first-order upwind, diffusion the 7-point stencil, inlet value imposed on the
  inlet face (2 D/h^2), zero-gradient outlet, no flux through side walls and fibers;
* migration through a face between fluid cells c, n:
  (z D F / (R T h^2)) (C_c + C_n)/2 (phi_n - phi_c) added to cell c (and the mirror term
  to n); no migration through the inlet, outlet, side walls or fibers (zero normal
  electric field there, Sec. II.A boundary conditions);
* the membrane (phi_L = 0, Sec. II.A) is the low-x face of the cells i = 0 (the
  logpile's stacking-height axis is x): a cation exchange membrane, so only protons cross
  it, by migration with the face value C_H,c and the potential difference (0 - phi_c)
  over half a cell; the other species have no flux there (zero concentration gradient);
* potential: face conductance kappa_f = (F^2 / R T) sum_k z_k^2 D_k (C_k,c + C_k,n)/2
  (all four species), membrane conductance (F^2 / R T) D_H C_H,c over half a cell,
  lap C_k the diffusion stencil above (inlet face term included, so the sum of z_k F
  times the species fluxes over a cell's faces is exactly the potential equation's
  divergence: the discrete equation is charge conservation, and with the three species
  equations it implies the counter-ion's own balance);
* inlet: C_O = (1 - s_in) c0, C_R = s_in c0, C_H = 50 c0 (1 M sulfuric acid against
  20 mM quinone, Sec. II.B), C_X by electroneutrality; D = 4e-10, D_H = 9.3e-9,
  D_X = 1.38e-9 m^2/s (parameter table; its second proton row is read as HSO4-).

Steady state: the fixed-point iteration of Algorithm 2 with the time step taken to
infinity (the paper runs its steps to steady state): given phi, the linear O-R system
(transport, migration, source) and then the proton system are solved; then the potential
equation with the new concentrations and the source of the previous potential; repeated
until phi and the concentrations stop changing. Model refinement (Sec. III.C): the
iteration starts from the SBV steady state (C_O = (1 - s) c0, C_R = s c0, C_H from the
protons the SBV reaction consumed, phi = 0).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import soc

Z = {"O": -2, "R": -2, "H": 1, "X": -1}
N_STOICH = {"O": -1.0, "R": 1.0, "H": -2.0}
D_H = 9.3e-9
D_X = 1.38e-9
H_RATIO = 50.0            # inlet proton concentration / c0


@dataclasses.dataclass
class BVParams:
    D_H: float = D_H
    D_X: float = D_X
    c_H_in: Optional[float] = None   # None: H_RATIO * c0


def inlet(p: soc.Problem, q: BVParams) -> dict:
    cH = H_RATIO * p.c0 if q.c_H_in is None else q.c_H_in
    cO, cR = (1.0 - p.s_in) * p.c0, p.s_in * p.c0
    return {"O": cO, "R": cR, "H": cH, "X": cH - 2.0 * (cO + cR)}


def diffusivities(p: soc.Problem, q: BVParams) -> dict:
    return {"O": p.D, "R": p.D, "H": q.D_H, "X": q.D_X}


def transport(p: soc.Problem, D: float, c_in: float):
    """Advection and diffusion of one species (soc.py's operator with diffusivity D and
    inlet value c_in, no reaction): (L, b) with L C + b the net inflow rate per volume."""
    op = soc.assemble(dataclasses.replace(p, D=D, s_in=c_in, k0=0.0))
    return op.L, op.b


def laplacian(p: soc.Problem, c_in: float):
    """The diffusion stencil with unit diffusivity and inlet face value c_in: (L, b) with
    L C + b = lap_h C (no advection)."""
    op = soc.assemble(dataclasses.replace(p, D=1.0, beta=0.0, s_in=c_in, k0=0.0))
    return op.L, op.b


def _faces(p: soc.Problem):
    """Interior faces between fluid cells: (c, n) index arrays over the three axes."""
    fluid = ~p.solid.astype(bool)
    nz, ny, nx = fluid.shape
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    cs, ns = [], []
    for a, b, both in ((idx[:, :, :-1], idx[:, :, 1:], fluid[:, :, :-1] & fluid[:, :, 1:]),
                       (idx[:, :-1, :], idx[:, 1:, :], fluid[:, :-1, :] & fluid[:, 1:, :]),
                       (idx[:-1], idx[1:], fluid[:-1] & fluid[1:])):
        cs.append(a[both]); ns.append(b[both])
    return np.concatenate(cs), np.concatenate(ns)


def membrane_cells(p: soc.Problem) -> np.ndarray:
    """Fluid cells whose low-x face is the membrane (i = 0)."""
    fluid = ~p.solid.astype(bool)
    nz, ny, nx = fluid.shape
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    return idx[:, :, 0][fluid[:, :, 0]]


def migration(p: soc.Problem, z: int, D: float, phi: np.ndarray, membrane: bool) -> sp.csr_matrix:
    """Matrix M with (M C)_c = (z D F / (R T h^2)) [sum_n (C_c + C_n)/2 (phi_n - phi_c)
    (+ 2 C_c (0 - phi_c) through the membrane)]."""
    N = p.solid.size
    g = z * D * soc.FARADAY / (soc.R_GAS * p.T * p.h * p.h)
    c, n = _faces(p)
    dphi = phi[n] - phi[c]
    rows = np.concatenate([c, c, n, n])
    cols = np.concatenate([c, n, n, c])
    vals = np.concatenate([0.5 * g * dphi, 0.5 * g * dphi, -0.5 * g * dphi, -0.5 * g * dphi])
    if membrane:
        m = membrane_cells(p)
        rows = np.concatenate([rows, m]); cols = np.concatenate([cols, m])
        vals = np.concatenate([vals, -2.0 * g * phi[m]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def rate_coefficients(p: soc.Problem, phi: np.ndarray):
    """(kf, kb): S = kf C_O - kb C_R per cell, kf = a k0 e^{alpha V~_c},
    kb = a k0 e^{(alpha-1) V~_c}, V~_c = V~ + n_e phi_c / V_T (zero off the electrode)."""
    kin = soc.kinetics(p.eta, p.alpha, p.n_e, p.T)
    fl = p.solid.ravel() == 0
    nw = soc.n_wall(p.solid.astype(bool)).ravel()
    m = np.ones(p.solid.size) if p.area_mult is None else \
        np.asarray(p.area_mult, np.float64).ravel()
    kap = np.where(fl, p.k0 * m * nw / p.h, 0.0)
    vc = kin.Vt + p.n_e * phi / kin.V_T
    return kap * np.exp(p.alpha * vc), kap * np.exp((p.alpha - 1.0) * vc)


def conductance(p: soc.Problem, q: BVParams, C: dict, phi_free=None):
    """Potential operator K with (K phi)_c = (1/h^2) [sum_n kappa_f (phi_n - phi_c)
    - 2 kappa_m,c phi_c (membrane)], kappa from Eq. kappa."""
    N = p.solid.size
    Dk = diffusivities(p, q)
    pre = soc.FARADAY ** 2 / (soc.R_GAS * p.T)
    kcell = pre * sum(Z[k] ** 2 * Dk[k] * C[k] for k in ("O", "R", "H", "X"))
    c, n = _faces(p)
    kf = 0.5 * (kcell[c] + kcell[n]) / (p.h * p.h)
    rows = np.concatenate([c, c, n, n])
    cols = np.concatenate([c, n, n, c])
    vals = np.concatenate([-kf, kf, -kf, kf])
    m = membrane_cells(p)
    km = pre * Dk["H"] * C["H"][m] / (p.h * p.h)
    rows = np.concatenate([rows, m]); cols = np.concatenate([cols, m])
    vals = np.concatenate([vals, -2.0 * km])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def counter_ion(C: dict) -> np.ndarray:
    """C_X from electroneutrality: -2 C_O - 2 C_R + C_H - C_X = 0."""
    return C["H"] - 2.0 * (C["O"] + C["R"])


def potential_rhs(p: soc.Problem, q: BVParams, C: dict, S: np.ndarray) -> np.ndarray:
    """n_e F S - F sum_k z_k D_k lap_h C_k (Eq. poisson-phi)."""
    cin = inlet(p, q)
    Dk = diffusivities(p, q)
    acc = p.n_e * soc.FARADAY * S
    for k in ("O", "R", "H", "X"):
        L, b = laplacian(p, cin[k])
        acc = acc - soc.FARADAY * Z[k] * Dk[k] * (L @ C[k] + b)
    return np.where(p.solid.ravel() == 0, acc, 0.0)


def species_rhs(p: soc.Problem, q: BVParams, C: dict, phi: np.ndarray) -> dict:
    """Net rate of change per volume of every species (O, R, H, and the counter-ion X,
    whose balance is implied) at (C, phi); zero at steady state."""
    cin = inlet(p, q)
    Dk = diffusivities(p, q)
    kf, kb = rate_coefficients(p, phi)
    S = kf * C["O"] - kb * C["R"]
    out = {}
    for k in ("O", "R", "H", "X"):
        L, b = transport(p, Dk[k], cin[k])
        M = migration(p, Z[k], Dk[k], phi, membrane=(k == "H"))
        out[k] = L @ C[k] + b + M @ C[k] + N_STOICH.get(k, 0.0) * S
        out[k] = np.where(p.solid.ravel() == 0, out[k], 0.0)
    return out


def potential_residual(p: soc.Problem, q: BVParams, C: dict, phi: np.ndarray) -> np.ndarray:
    kf, kb = rate_coefficients(p, phi)
    S = kf * C["O"] - kb * C["R"]
    K = conductance(p, q, C)
    r = K @ phi - potential_rhs(p, q, C, S)
    return np.where(p.solid.ravel() == 0, r, 0.0)


def initial_from_sbv(p: soc.Problem, q: BVParams, s: np.ndarray) -> tuple:
    """Model refinement: concentrations from an SBV state s (C_T = c0), protons reduced by
    the two consumed per converted quinone, phi = 0."""
    cin = inlet(p, q)
    fl = p.solid.ravel() == 0
    C = {"O": np.where(fl, (1.0 - s) * p.c0, 0.0), "R": np.where(fl, s * p.c0, 0.0)}
    C["H"] = np.where(fl, cin["H"] - 2.0 * (C["R"] - cin["R"]), 0.0)
    C["X"] = counter_ion(C)
    return C, np.zeros(p.solid.size)


def _solve_fluid(A: sp.spmatrix, rhs: np.ndarray, fl: np.ndarray) -> np.ndarray:
    x = np.zeros(rhs.size)
    x[fl] = spla.spsolve(A[fl][:, fl].tocsc(), rhs[fl])
    return x


def fixed_point_step(p: soc.Problem, q: BVParams, phi: np.ndarray):
    """One step of Algorithm 2's fixed-point iteration in steady form: the O-R system
    (transport, migration, source) and then the proton system at the potential phi, then
    the potential equation with the new concentrations and source. Returns (C, phi_new)."""
    fl = p.solid.ravel() == 0
    N = p.solid.size
    cin = inlet(p, q)
    Dk = diffusivities(p, q)
    LO, bO = transport(p, Dk["O"], cin["O"])
    LR, bR = transport(p, Dk["R"], cin["R"])
    LH, bH = transport(p, Dk["H"], cin["H"])
    kf, kb = rate_coefficients(p, phi)
    AO = LO + migration(p, Z["O"], Dk["O"], phi, False)
    AR = LR + migration(p, Z["R"], Dk["R"], phi, False)
    A = sp.bmat([[AO - sp.diags(kf), sp.diags(kb)],
                 [sp.diags(kf), AR - sp.diags(kb)]]).tocsr()
    x = _solve_fluid(A, -np.concatenate([bO, bR]), np.concatenate([fl, fl]))
    C = {"O": x[:N], "R": x[N:]}
    S = kf * C["O"] - kb * C["R"]
    AH = LH + migration(p, Z["H"], Dk["H"], phi, True)
    C["H"] = _solve_fluid(AH, -(bH + N_STOICH["H"] * S), fl)
    C["X"] = counter_ion(C)
    K = conductance(p, q, C)
    return C, _solve_fluid(K, potential_rhs(p, q, C, S), fl)


def solve(p: soc.Problem, q: Optional[BVParams] = None, s0: Optional[np.ndarray] = None,
          tol: float = 1e-13, max_iter: int = 200):
    """Steady state of the Butler-Volmer model by the fixed-point iteration of
    Algorithm 2 (steady form), from the SBV state s0 (solved here if None): model
    refinement. Stops once the largest change of phi is <= tol (V_T / n_e) and that of
    every concentration <= tol times its largest value. Returns (C, phi, iterations)."""
    q = q or BVParams()
    if s0 is None:
        s0 = soc.steady_state(soc.assemble(p))
    C, phi = initial_from_sbv(p, q, s0)
    kin = soc.kinetics(p.eta, p.alpha, p.n_e, p.T)
    for it in range(1, max_iter + 1):
        Cn, phin = fixed_point_step(p, q, phi)
        dphi = float(np.abs(phin - phi).max())
        dc = max(float(np.abs(Cn[k] - C[k]).max() / np.abs(Cn[k]).max())
                 for k in ("O", "R", "H"))
        C, phi = Cn, phin
        if dphi <= tol * kin.V_T / p.n_e and dc <= tol:
            return C, phi, it
    raise RuntimeError("BV fixed-point iteration did not converge")


def outputs(p: soc.Problem, q: BVParams, C: dict, phi: np.ndarray) -> dict:
    """I_tot (Eq. I-tot-def), s = C_R / (C_O + C_R), utilisation from I_tot (Eq.
    utilization-def, first form), the outlet's flow-weighted mean s, the membrane current
    (protons' migration through the membrane) and potential statistics over fluid cells."""
    fl = p.solid.ravel() == 0
    kf, kb = rate_coefficients(p, phi)
    S = kf * C["O"] - kb * C["R"]
    h = p.h
    I_tot = p.n_e * soc.FARADAY * h ** 3 * float(S.sum())
    CT = C["O"] + C["R"]
    s = np.where(fl, C["R"] / np.where(fl, CT, 1.0), 0.0)
    nz, ny, nx = p.solid.shape
    Q = h * h * p.beta * float(np.sum(np.where(p.solid[0] == 0, p.W[0], 0.0)))
    U = I_tot / (p.n_e * soc.FARADAY * p.c0 * Q * (1.0 - p.s_in))
    w = np.where(p.solid[-1] == 0, p.beta * p.W[-1], 0.0).ravel()
    s_out = float(np.sum(w * s.reshape(nz, ny, nx)[-1].ravel())) / float(w.sum())
    m = membrane_cells(p)
    pre = soc.FARADAY ** 2 / (soc.R_GAS * p.T)
    I_mem = float(np.sum(pre * q.D_H * C["H"][m] * 2.0 * (0.0 - phi[m]) / h)) * h * h
    return {"I_tot": I_tot, "U": U, "s": s, "s_out": s_out, "I_membrane": I_mem,
            "phi_mean": float(phi[fl].mean()), "phi_max": float(phi[fl].max()),
            "phi_min": float(phi[fl].min()), "CT_min": float(CT[fl].min()),
            "CT_max": float(CT[fl].max())}
