"""CPU oracle for the steady state-of-charge problem (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module. The product path (the CUDA library behind ``include/rfb_soc.h``)
shares no code with it.

What it computes, in FP64, following the paper (arXiv 2502.08034):

* Kinetics: V_T = RT/F; applied reducing voltage V_ar = -eta (eta = overpotential at
  s = 1/2 with phi_L = 0, Eq. etat-from-s with s = 1/2); V~ = n_e V_ar / V_T
  (Eq. Vart-def); s_eq = sigma(V~) (Eq. seq-from-Var); affine rate law
  R~(s) = e^{alpha V~} (1 - (1 + e^{-V~}) s) (Eq. rate-from-soc-gen).
* The steady form of Eq. nernst-planck-soc on a voxel lattice, assembled face by face
  as explicit sparse matrices, the way the paper's explicit proof of concept holds its
  advection and diffusion operators as assembled sparse matrices (Sec. III.C):
  first-order upwind advection by the given face velocities,
  7-point diffusion, a Dirichlet inlet, zero-gradient outlet, no flux through side walls
  and fiber faces, and the Butler-Volmer source k0 a_c R~(s_c) with a_c = m_c n_wall/h
  (n_wall = number of fiber 6-neighbours; the paper's a = A/V of a cut cell).
  RHS(s) = L s + b.
* Kinetics mode 1 (the literal uniform activation overpotential): the source is the
  Butler-Volmer rate at a fixed eta~ = -n_e eta / V_T (Eqs. etat-def,
  source-term-bv-gen), k0 a_c s^alpha (1-s)^(1-alpha) (e^{alpha eta~} - e^{(alpha-1) eta~}),
  nonlinear in s; its steady state is found by Newton's method with the exact Jacobian.
* The steady state is the solution of RHS(s) = 0 (a sparse direct solve; the affine rate
  law makes the problem linear). ``explicit_iterate`` runs the paper's pseudo-time loop
  s <- s + dt RHS(s) (Algorithm 7's two-buffer loop with F = I + dt(A + D + R)).
* U_mt (Eq. umt-def): reaction off, s = 0 at the inlet, fluid cells touching a fiber
  held at 1 (Eq. np-fast-boundary; Algorithm 7 resets s[elec] := 1 every step).
* Outputs: I_tot (Eq. I-tot-def), F_in / F_out (Eq. electron-flow), mass-balance error
  (Eq. convergence-bv-flow), utilisation U (Eq. utilization-def, first form), residual
  (tau/dt)||ds||_RMS = tau RMS(RHS) (Eq. convergence-bv-change) with tau = V_f/Q.

Readings where the paper is silent (stated here once, used throughout):
* inlet diffusion: the value s_in is imposed on the inlet face, half a cell from the
  cell centre, so the diffusive term is (2D/h^2)(s_in - s_c); ``inlet_bc='ghost'``
  gives the alternative (D/h^2)(s_in - s_c);
* dt = C_CFL / max_c d_c with d_c = -L_cc (the diagonal of -L), so every explicit
  update is a convex combination for C_CFL <= 1; ``local_dt`` uses dt_c = C_CFL / d_c;
* tau = V_f / Q with V_f the fluid volume and Q = sum over inlet faces of W h^2;
* F_in includes the inlet diffusive flux so that I_tot = F_out - F_in holds exactly.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

R_GAS = 8.314462618      # J/(mol K)
FARADAY = 96485.33212    # C/mol


# --------------------------------------------------------------------------------------
# Kinetics (Sec. II.B-II.D)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Kinetics:
    V_T: float        # thermal voltage RT/F
    V_ar: float       # applied reducing voltage
    Vt: float         # n_e V_ar / V_T
    s_eq: float       # sigma(Vt)
    A: float          # intercept of R~(s): e^{alpha Vt}
    B: float          # -slope of R~(s): e^{alpha Vt} (1 + e^{-Vt})
    alpha: float = 0.5
    K1: float = 0.0   # e^{alpha eta~} - e^{(alpha-1) eta~} at eta~ = Vt (kinetics mode 1)


def kinetics(eta: float, alpha: float = 0.5, n_e: int = 2, T: float = 298.0) -> Kinetics:
    V_T = R_GAS * T / FARADAY
    V_ar = -eta
    Vt = n_e * V_ar / V_T
    A = math.exp(alpha * Vt)
    B = A * (1.0 + math.exp(-Vt))
    s_eq = 1.0 / (1.0 + math.exp(-Vt))
    K1 = math.exp(alpha * Vt) - math.exp((alpha - 1.0) * Vt)
    return Kinetics(V_T, V_ar, Vt, s_eq, A, B, alpha, K1)


def rate_affine(s, kin: Kinetics):
    """R~(s) by Eq. rate-from-soc-gen."""
    return kin.A * (1.0 - (1.0 + math.exp(-kin.Vt)) * np.asarray(s, dtype=np.float64))


def rate_bv(s, Vt: float, alpha: float = 0.5):
    """R~(s) by Eq. source-term-bv-gen divided by a k0 C_T, with eta~ from
    Eq. etat-from-s (phi_L = 0)."""
    s = np.asarray(s, dtype=np.float64)
    etat = Vt - np.log(s / (1.0 - s))
    return s ** alpha * (1.0 - s) ** (1.0 - alpha) * (np.exp(alpha * etat) -
                                                     np.exp((alpha - 1.0) * etat))


def rate_uniform(s, etat: float, alpha: float = 0.5):
    """R~(s) = S / (a k0 C_T) at a fixed dimensionless overpotential eta~ (Eq. etat-def):
    s^alpha (1 - s)^(1 - alpha) (e^{alpha eta~} - e^{(alpha - 1) eta~})
    (Eq. source-term-bv-gen; Eq. source-term-bv at alpha = 1/2). Kinetics mode 1, the
    literal uniform activation overpotential."""
    s = np.asarray(s, dtype=np.float64)
    return s ** alpha * (1.0 - s) ** (1.0 - alpha) * (math.exp(alpha * etat) -
                                                     math.exp((alpha - 1.0) * etat))


def rate_uniform_slope(s, etat: float, alpha: float = 0.5):
    """d R~/ds of ``rate_uniform`` for 0 < s < 1:
    (e^{alpha eta~} - e^{(alpha-1) eta~}) s^(alpha-1) (1-s)^(-alpha) (alpha - s)."""
    s = np.asarray(s, dtype=np.float64)
    return (math.exp(alpha * etat) - math.exp((alpha - 1.0) * etat)) * \
        s ** (alpha - 1.0) * (1.0 - s) ** (-alpha) * (alpha - s)


# --------------------------------------------------------------------------------------
# Operator assembly
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Everything the discrete operator depends on. Arrays in (nz, ny, nx) layout."""
    solid: np.ndarray
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    h: float
    D: float
    s_in: float
    k0: float = 0.0
    alpha: float = 0.5
    n_e: int = 2
    T: float = 298.0
    c0: float = 20.0
    eta: float = 0.0
    beta: float = 1.0
    area_mult: Optional[np.ndarray] = None
    inlet_bc: str = "face"
    kinetics_mode: int = 0    # 0 affine (Eq. rate-from-soc-gen), 1 uniform eta_act

    @property
    def dims(self):
        nz, ny, nx = self.solid.shape
        return nx, ny, nz


@dataclasses.dataclass
class Operator:
    L: sp.csr_matrix          # N x N, rows of solid cells empty
    b: np.ndarray             # N
    unknown: np.ndarray       # N bool: cells whose value is solved for
    fixed: np.ndarray         # N float: values of the non-unknown cells (0 on solid)
    kappa: np.ndarray         # N: k0 a_c (zero in U_mt mode)
    kin: Kinetics
    Q: float                  # volumetric flow rate through the inlet
    tau: float                # V_f / Q
    n_fluid: int
    nonlinear: bool = False   # kinetics mode 1: L, b hold transport only and the source
                              # kappa_c R~(s_c) is rate_uniform at eta~ = kin.Vt
    s_in: float = 0.0         # inlet value the operator was assembled with


def n_wall(solid: np.ndarray) -> np.ndarray:
    """Number of in-domain solid 6-neighbours of each cell (nz, ny, nx)."""
    s = solid.astype(np.int32)
    n = np.zeros_like(s)
    n[:, :, 1:] += s[:, :, :-1]
    n[:, :, :-1] += s[:, :, 1:]
    n[:, 1:, :] += s[:, :-1, :]
    n[:, :-1, :] += s[:, 1:, :]
    n[1:] += s[:-1]
    n[:-1] += s[1:]
    return n


def assemble(p: Problem, mode: str = "sbv") -> Operator:
    """Build RHS(s) = L s + b for every fluid cell.

    mode 'sbv': Eq. nernst-planck-soc with the affine source (Eq. rate-from-soc-gen); with
    ``p.kinetics_mode == 1`` the source is the Butler-Volmer rate at a uniform activation
    overpotential (Eq. source-term-bv-gen, eta~ = -n_e eta / V_T by Eq. etat-def), which is
    nonlinear in s: L and b then hold advection and diffusion only and ``rhs`` adds
    kappa_c R~(s_c).
    mode 'umt': Eqs. np-fast-interior/np-fast-boundary with s_in = 0 and the cells that
    touch a fiber held at 1 (Eq. umt-def)."""
    solid = p.solid.astype(bool)
    nz, ny, nx = solid.shape
    N = nx * ny * nz
    h, D = p.h, p.D
    beta = p.beta
    s_in = 0.0 if mode == "umt" else p.s_in
    idx = np.arange(N).reshape(nz, ny, nx)
    fluid = ~solid
    rows, cols, vals = [], [], []
    b = np.zeros(N)

    def add(r, c, v):
        rows.append(r); cols.append(c); vals.append(v)

    def interior_faces(a, c, u, both):
        # face between cell a (low side) and c (high side), velocity u along +axis.
        a, c, u, both = a.ravel(), c.ravel(), u.ravel() * beta, both.ravel()
        pos = np.maximum(u, 0.0) / h      # flux a -> c carries s_a
        neg = np.maximum(-u, 0.0) / h     # flux c -> a carries s_c
        add(a, a, -pos); add(c, a, pos)
        add(c, c, -neg); add(a, c, neg)
        dd = np.where(both, D / (h * h), 0.0)
        add(a, a, -dd); add(a, c, dd)
        add(c, c, -dd); add(c, a, dd)

    interior_faces(idx[:, :, :-1], idx[:, :, 1:], p.U[:, :, 1:-1],
                   fluid[:, :, :-1] & fluid[:, :, 1:])
    interior_faces(idx[:, :-1, :], idx[:, 1:, :], p.V[:, 1:-1, :],
                   fluid[:, :-1, :] & fluid[:, 1:, :])
    interior_faces(idx[:-1], idx[1:], p.W[1:-1], fluid[:-1] & fluid[1:])

    # inlet: faces W[0] below plane k = 0 (Dirichlet s_in on the face)
    cin = idx[0].ravel()
    fin = fluid[0].ravel()
    w = p.W[0].ravel() * beta
    add(cin, cin, -np.maximum(-w, 0.0) / h)
    np.add.at(b, cin, np.maximum(w, 0.0) / h * s_in)
    g = 2.0 if p.inlet_bc == "face" else 1.0
    gd = np.where(fin, g * D / (h * h), 0.0)
    add(cin, cin, -gd)
    np.add.at(b, cin, gd * s_in)
    # outlet: faces W[nz] above plane nz-1, zero-gradient (flux w s_c)
    cout = idx[-1].ravel()
    w = p.W[-1].ravel() * beta
    add(cout, cout, -w / h)

    kin = kinetics(p.eta, p.alpha, p.n_e, p.T)
    kappa = np.zeros(N)
    nw = n_wall(solid)
    nonlinear = mode == "sbv" and p.kinetics_mode == 1
    if mode == "sbv":
        m = np.ones(N) if p.area_mult is None else np.asarray(p.area_mult, np.float64).ravel()
        kappa = np.where(fluid.ravel(), p.k0 * m * nw.ravel() / h, 0.0)
        if not nonlinear:
            add(idx.ravel(), idx.ravel(), -kappa * kin.B)
            b += kappa * kin.A

    L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    L.sum_duplicates()
    fl = fluid.ravel()
    # rows and columns of solid cells carry only zero velocities: drop them entirely
    L = sp.diags(fl.astype(np.float64)) @ L @ sp.diags(fl.astype(np.float64))
    L = L.tocsr()
    L.eliminate_zeros()
    b = np.where(fl, b, 0.0)

    unknown = fl.copy()
    fixed = np.zeros(N)
    if mode == "umt":
        elec = fl & (nw.ravel() > 0)
        unknown = fl & ~elec
        fixed[elec] = 1.0
    Q = h * h * beta * float(np.sum(np.where(fin, p.W[0].ravel(), 0.0)))
    nf = int(fl.sum())
    Vf = nf * h ** 3
    tau = Vf / Q if Q > 0 else (nz * h) ** 2 / D
    return Operator(L, b, unknown, fixed, kappa, kin, Q, tau, nf, nonlinear, s_in)


# --------------------------------------------------------------------------------------
# Steady state, iteration, outputs
# --------------------------------------------------------------------------------------

def source(op: Operator, s: np.ndarray) -> np.ndarray:
    """k0 a_c R~(s_c) per cell (s^-1), for either kinetics mode."""
    if op.nonlinear:
        return op.kappa * rate_uniform(np.clip(s, 0.0, 1.0), op.kin.Vt, op.kin.alpha)
    return op.kappa * rate_affine(s, op.kin)


def rhs(op: Operator, s: np.ndarray) -> np.ndarray:
    """RHS(s) = L s + b (+ the nonlinear source in kinetics mode 1), zero on solid cells."""
    r = op.L @ s + op.b
    if op.nonlinear:
        r = r + source(op, s)
    return r


def jacobian(op: Operator, s: np.ndarray) -> sp.csr_matrix:
    """d RHS / ds at s: L itself for the affine law; L + diag(kappa R~'(s)) in mode 1."""
    if not op.nonlinear:
        return op.L
    d = np.zeros(s.size)
    k = op.kappa != 0
    d[k] = op.kappa[k] * rate_uniform_slope(s[k], op.kin.Vt, op.kin.alpha)
    return (op.L + sp.diags(d)).tocsr()


def step_diagonal(op: Operator) -> np.ndarray:
    """d_c of the pseudo-time step: the diagonal of -L plus, in kinetics mode 1, the
    affine law's reaction slope k0 a_c (e^{alpha V~} + e^{(alpha-1) V~}) at the same
    dimensionless voltage (the step does not depend on the state)."""
    d = -op.L.diagonal()
    if op.nonlinear:
        d = d + op.kappa * op.kin.B
    return d


def residual(op: Operator, s: np.ndarray) -> float:
    """tau * RMS of RHS over the unknown cells (Eq. convergence-bv-change)."""
    r = rhs(op, s)[op.unknown]
    return op.tau * math.sqrt(float(np.mean(r * r))) if r.size else 0.0


def steady_state(op: Operator, direct_max: int = 40000, rtol: float = 1e-14) -> np.ndarray:
    """Solve RHS(s) = 0 for the unknown cells; other cells take their fixed values.

    Up to ``direct_max`` unknowns: sparse LU (SuperLU). Larger systems: GMRES on the
    row-scaled system D^{-1} L (D = diag L) with an incomplete-LU preconditioner, to a
    relative residual of ``rtol``; both are library linear solvers of the same system."""
    if op.nonlinear:
        return newton_steady_state(op, direct_max=direct_max, rtol=rtol)
    u = op.unknown
    s = op.fixed.copy()
    Luu = op.L[u][:, u].tocsc()
    rhs_u = -(op.b[u] + op.L[u] @ op.fixed)
    s[u] = _linear_solve(Luu, rhs_u, direct_max, rtol)
    return s


def _linear_solve(A: sp.spmatrix, r: np.ndarray, direct_max: int, rtol: float) -> np.ndarray:
    if A.shape[0] <= direct_max:
        return spla.spsolve(A.tocsc(), r)
    dinv = sp.diags(1.0 / A.diagonal())
    As = (dinv @ A).tocsc()
    rs = dinv @ r
    ilu = spla.spilu(As, drop_tol=1e-5, fill_factor=10)
    M = spla.LinearOperator(As.shape, ilu.solve)
    x, info = spla.gmres(As, rs, M=M, rtol=rtol, atol=0.0, restart=200, maxiter=20)
    if info != 0:
        raise RuntimeError("oracle GMRES did not reach rtol=%g (info=%d)" % (rtol, info))
    return x


def newton_steady_state(op: Operator, s0: Optional[np.ndarray] = None, direct_max: int = 40000,
                        rtol: float = 1e-14, max_iter: int = 400) -> np.ndarray:
    """RHS(s) = 0 for kinetics mode 1 by Newton's method globalised with pseudo-transient
    continuation (Kelley and Keyes, SIAM J. Numer. Anal. 35, 1998): on the unknown cells
    (D/delta - J(s)) ds = RHS(s), with J = L + diag(kappa R~'(s)) the exact Jacobian and D
    the pseudo-time step diagonal (``step_diagonal``); delta starts at 0.4 (one implicit
    step of the explicit loop's size) and grows by switched evolution relaxation,
    delta <- delta ||RHS_prev|| / ||RHS||, so the iteration turns into Newton's method near
    the solution. Steps are halved while they would leave (0, 1). Starts from s = s_in
    (clamped into (0, 1)) unless s0 is given; stops once delta >= 1e8 and the step is
    below rtol max|s|, or below 1e-9 max|s| and no smaller than half the previous one (the
    rounding floor of the linear solves). At delta >= 1e8 the pseudo-time term D/delta is
    at most 1e-8 of the diagonal, so the step solves Newton's equation to that accuracy
    and these tests are as valid as for Newton's method itself; delta cannot be required
    to grow further, since near the rounding floor ||RHS|| only jitters and the update
    above stalls."""
    u = op.unknown
    s = initial_state(op, op.s_in) if s0 is None else np.array(s0, dtype=np.float64)
    s[u] = np.clip(s[u], 1e-12, 1.0 - 1e-12)
    d = step_diagonal(op)[u]
    delta = 0.4
    r = rhs(op, s)[u]
    rn = float(np.linalg.norm(r))
    prev = math.inf
    for _ in range(max_iter):
        J = jacobian(op, s)[u][:, u]
        A = (sp.diags(d / delta) - J).tocsr() if delta < 1e15 else -J
        ds = _linear_solve(A, r, direct_max, rtol)
        lam = 1.0
        while True:
            t_ = s[u] + lam * ds
            if np.all(t_ > 0.0) and np.all(t_ < 1.0):
                break
            lam *= 0.5
        s[u] = t_
        r = rhs(op, s)[u]
        rn_new = float(np.linalg.norm(r))
        step = float(np.max(np.abs(ds))) if ds.size else 0.0
        scale = max(1.0, float(np.max(np.abs(s))))
        newton = delta >= 1e8
        if newton and lam == 1.0 and (step <= rtol * scale or
                                      (step <= 1e-9 * scale and step >= 0.5 * prev)):
            return s
        prev = step if (newton and lam == 1.0) else math.inf
        if rn_new == 0.0:
            return s
        delta = min(delta * rn / rn_new, 1e16) if lam == 1.0 else max(delta * 0.5, 1e-3)
        rn = rn_new
    raise RuntimeError("oracle pseudo-transient Newton iteration did not converge")


def nonlinear_step_cap(op: Operator, s: np.ndarray, cfl: float) -> np.ndarray:
    """Kinetics mode 1: cfl / (d_T,c + kappa_c max(0, -R~'(s_c))) per cell, d_T the
    transport diagonal of -L. Near s = 1 the rate's slope grows like (1-s)^(-alpha), and
    the explicit update stays stable only with a step below the inverse of that local
    stiffness; the slope is taken at min(s, 1 - 2^-40) so the cap never reaches 0."""
    d = -op.L.diagonal()
    sh = np.minimum(s, 1.0 - 2.0 ** -40)
    sl = np.zeros(s.size)
    k = (op.kappa != 0) & (sh > op.kin.alpha)
    sl[k] = -rate_uniform_slope(sh[k], op.kin.Vt, op.kin.alpha)
    den = d + op.kappa * sl
    return np.where(den > 0, cfl / np.where(den > 0, den, 1.0), np.inf)


def dt_global(op: Operator, cfl: float) -> float:
    d = step_diagonal(op)[op.unknown]
    return cfl / float(d.max())


def explicit_iterate(op: Operator, cfl: float, tol: float, s0: Optional[np.ndarray] = None,
                     max_steps: int = 10_000_000, check_every: int = 1, local_dt: bool = False):
    """Explicit pseudo-time stepping to tau*RMS(RHS) < tol, two buffers as in Algorithm 7.

    In kinetics mode 1 each cell's step is also capped by ``nonlinear_step_cap`` (the
    fixed point does not depend on the step) and the update is clipped into [0, 1] (a
    guard of Sec. III.B; at a converged state it does not bind, since there RHS = 0 with
    s inside the interval).
    Returns (s, steps)."""
    u = op.unknown
    d = step_diagonal(op)
    if local_dt:
        dt = np.where(u, cfl / np.where(d > 0, d, 1.0), 0.0)
    else:
        dt = np.where(u, dt_global(op, cfl), 0.0)
    s = [op.fixed.copy() if s0 is None else np.array(s0, dtype=np.float64), None]
    if s0 is None:
        s[0][u] = 0.0
    n = 0
    while n < max_steps:
        i, j = n % 2, (n + 1) % 2
        if op.nonlinear:
            dtn = np.minimum(dt, nonlinear_step_cap(op, s[i], cfl))
            s[j] = np.clip(s[i] + dtn * rhs(op, s[i]), 0.0, 1.0)
        else:
            s[j] = s[i] + dt * rhs(op, s[i])
        s[j][~u] = op.fixed[~u]
        n += 1
        if n % check_every == 0 and residual(op, s[j]) < tol:
            break
    return s[n % 2], n


def initial_state(op: Operator, s_in: float) -> np.ndarray:
    """Cold start: s = s_in on unknown fluid cells (the paper initialises from the inlet
    value), fixed values elsewhere."""
    s = op.fixed.copy()
    s[op.unknown] = s_in
    return s


@dataclasses.dataclass
class Outputs:
    I_tot: float
    F_in: float
    F_out: float
    F_in_adv: float
    mass_balance_rel: float
    U: float
    U_outlet_form: float
    residual: float


def outputs(p: Problem, op: Operator, s: np.ndarray) -> Outputs:
    """Currents, mass balance and utilisation of state s (Sec. II.C)."""
    solid = p.solid.astype(bool)
    nz, ny, nx = solid.shape
    h = p.h
    scale = p.n_e * FARADAY * p.c0
    I_tot = scale * h ** 3 * float(np.sum(source(op, s)))
    s3 = s.reshape(nz, ny, nx)
    fin = ~solid[0]
    fout = ~solid[-1]
    g = 2.0 if p.inlet_bc == "face" else 1.0
    w_in = p.beta * p.W[0]
    w_out = p.beta * p.W[-1]
    adv_in = float(np.sum(np.where(fin, w_in * p.s_in, 0.0)))
    dif_in = float(np.sum(np.where(fin, g * p.D / h * (p.s_in - s3[0]), 0.0)))
    F_in_adv = scale * h * h * adv_in
    F_in = scale * h * h * (adv_in + dif_in)
    F_out = scale * h * h * float(np.sum(np.where(fout, w_out * s3[-1], 0.0)))
    mb = abs(I_tot - (F_out - F_in)) / abs(I_tot) if I_tot != 0 else abs(F_out - F_in)
    denom = scale * op.Q * (1.0 - p.s_in)
    U = I_tot / denom if denom != 0 else float("nan")
    sw = float(np.sum(np.where(fout, w_out, 0.0)))
    s_out_mean = float(np.sum(np.where(fout, w_out * s3[-1], 0.0))) / sw if sw else float("nan")
    U_out = (s_out_mean - p.s_in) / (1.0 - p.s_in)
    return Outputs(I_tot, F_in, F_out, F_in_adv, mb, U, U_out, residual(op, s))


def umt(p: Problem, s: Optional[np.ndarray] = None) -> float:
    """U_mt = sum_out W s_mt / sum_out W (Eq. umt-def) of the U_mt steady state."""
    op = assemble(p, mode="umt")
    if s is None:
        s = steady_state(op)
    solid = p.solid.astype(bool)
    nz, ny, nx = solid.shape
    s3 = s.reshape(nz, ny, nx)
    fout = ~solid[-1]
    w = p.W[-1]
    return float(np.sum(np.where(fout, w * s3[-1], 0.0))) / float(np.sum(np.where(fout, w, 0.0)))


# --------------------------------------------------------------------------------------
# Discrete adjoint of the steady state
# --------------------------------------------------------------------------------------
#
# The steady state solves RHS(s; m, beta) = L(m, beta) s + b(m, beta) = 0 (linear in s,
# Eq. rate-from-soc-gen). For an objective J(s, m, beta):
#   L^T lam = -dJ/ds,   dJ/dp = dJ/dp|explicit + lam . dRHS/dp
# In kinetics mode 1 (nonlinear source) L is the Jacobian dRHS/ds at the steady state,
# L + diag(kappa R~'(s)), and R~ below is the mode-1 rate.
# with dRHS_c/dm_c = k0 n_wall(c)/h R~(s_c) (only row c) and dRHS/dbeta = the advective
# part of RHS divided by beta (every face velocity carries beta). Objectives:
#   'I_tot' : J = n_e F c0 h^3 sum_c k0 m_c n_wall/h R~(s_c)              (Eq. I-tot-def)
#   'U'     : J = I_tot / (n_e F c0 Q (1 - s_in)), Q = beta h^2 sum_in W  (Eq. utilization-def)
#   'U_mt'  : J = sum_out W s / sum_out W on the U_mt state (Eq. umt-def); independent of m.

def _advection_only(p: Problem, mode: str) -> Operator:
    """Operator with D = 0 and no reaction: L_adv s + b_adv is the advective part."""
    q = dataclasses.replace(p, D=0.0, k0=0.0)
    return assemble(q, mode=mode)


def transposed_iterate(A: sp.spmatrix, g: np.ndarray, cfl: float, tol: float,
                       max_steps: int = 10_000_000, check_every: int = 100):
    """Explicit pseudo-time iteration of A^T lam + g = 0 with the local step
    dt_c = cfl / d_c, d_c = -A_cc (A and A^T share their diagonal): lam <- lam +
    dt (A^T lam + g), from lam = 0, the forward loop of Algorithm 7 applied to the
    transposed operator, until ||A^T lam + g||_2 <= tol ||g||_2. Returns (lam, steps)."""
    At = A.T.tocsr()
    d = -A.diagonal()
    dt = cfl / d
    lam = np.zeros(A.shape[0])
    gn = float(np.linalg.norm(g))
    n = 0
    while n < max_steps:
        lam = lam + dt * (At @ lam + g)
        n += 1
        if n % check_every == 0 and float(np.linalg.norm(At @ lam + g)) <= tol * gn:
            break
    return lam, n


def adjoint(p: Problem, s: np.ndarray, objective: str = "I_tot", direct_max: int = 40000,
            rtol: float = 1e-14, iter_tol: float = 1e-13) -> dict:
    """Adjoint state and gradients at the steady state s (solved here if None).

    L^T lam = -dJ/ds: sparse LU up to ``direct_max`` unknowns; larger affine problems
    (kinetics mode 0) by the explicit transposed iteration ``transposed_iterate`` to a
    relative residual of ``iter_tol`` (the forward pseudo-time loop applied to L^T)."""
    mode = "umt" if objective == "U_mt" else "sbv"
    op = assemble(p, mode)
    if s is None:
        s = steady_state(op)
    u = op.unknown
    N = s.size
    h = p.h
    scale = p.n_e * FARADAY * p.c0 * h ** 3
    nw = n_wall(p.solid.astype(bool)).ravel().astype(np.float64)
    m = np.ones(N) if p.area_mult is None else np.asarray(p.area_mult, np.float64).ravel()
    fl = p.solid.ravel() == 0
    kap0 = np.where(fl, p.k0 * nw / h, 0.0)             # dkappa/dm
    g = np.zeros(N)
    if op.nonlinear:
        slope = np.zeros(N)
        k = kap0 != 0
        slope[k] = rate_uniform_slope(s[k], op.kin.Vt, op.kin.alpha)
        R = rate_uniform(s, op.kin.Vt, op.kin.alpha)
    else:
        slope = np.full(N, -op.kin.B)
        R = rate_affine(s, op.kin)
    if objective in ("I_tot", "U"):
        g = scale * kap0 * m * slope                    # dI_tot/ds
        denom = p.n_e * FARADAY * p.c0 * op.Q * (1.0 - p.s_in)
        if objective == "U":
            g = g / denom
    elif objective == "U_mt":
        nz, ny, nx = p.solid.shape
        w_out = np.zeros(N)
        w_out[(nz - 1) * nx * ny:] = np.where(fl[(nz - 1) * nx * ny:], p.beta * p.W[-1].ravel(),
                                              0.0)
        g = np.where(u, w_out / w_out.sum(), 0.0)
    else:
        raise ValueError(objective)
    Luu = jacobian(op, s)[u][:, u]
    lam = np.zeros(N)
    if Luu.shape[0] <= direct_max:
        lam[u] = spla.spsolve(Luu.T.tocsc(), -g[u])
    elif not op.nonlinear:
        lam[u], _ = transposed_iterate(Luu, g[u], 0.4, iter_tol)
    else:
        raise ValueError("the oracle's kinetics-mode-1 adjoint is direct only (<= %d unknowns)"
                         % direct_max)
    # gradients
    dm = np.zeros(N)
    if objective == "I_tot":
        dm = (scale + lam) * kap0 * R
    elif objective == "U":
        dm = (scale / denom + lam) * kap0 * R
    dm = np.where(fl, dm, 0.0)
    adv = _advection_only(p, mode)
    adv_rhs = (adv.L @ s + adv.b)
    dbeta = float(np.dot(lam[u], adv_rhs[u])) / p.beta if p.beta != 0 else float("nan")
    if objective == "U":
        J = outputs(p, op, s).U
        dbeta -= J / p.beta
    return {"lam": lam, "d_area_mult": dm, "d_beta": dbeta, "g": g, "s": s}


# --------------------------------------------------------------------------------------
# Iterative upsampling (Sec. III.A)
# --------------------------------------------------------------------------------------

def prolong(s_coarse: np.ndarray, solid_coarse: np.ndarray, solid_fine: np.ndarray,
            s_in: float) -> np.ndarray:
    """2x injection: s_f(i,j,k) = s_c(i//2, j//2, k//2). A fine fluid cell whose parent is
    solid takes the mean over the parent's fluid 6-neighbours, else s_in. Solid -> 0."""
    sc = s_coarse.reshape(solid_coarse.shape)
    cfluid = ~solid_coarse.astype(bool)
    nzc, nyc, nxc = sc.shape
    acc = np.zeros_like(sc)
    cnt = np.zeros_like(sc)
    for axis in range(3):
        for sh in (-1, 1):
            vals = np.where(cfluid, sc, 0.0)
            f = cfluid.astype(np.float64)
            sl_src = [slice(None)] * 3
            sl_dst = [slice(None)] * 3
            if sh == 1:   # neighbour at +1 along axis
                sl_src[axis] = slice(1, None); sl_dst[axis] = slice(0, -1)
            else:
                sl_src[axis] = slice(0, -1); sl_dst[axis] = slice(1, None)
            acc[tuple(sl_dst)] += vals[tuple(sl_src)]
            cnt[tuple(sl_dst)] += f[tuple(sl_src)]
    fill = np.where(cnt > 0, acc / np.where(cnt > 0, cnt, 1.0), s_in)
    parent = np.where(cfluid, sc, fill)
    fine = parent.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)
    fine = np.where(solid_fine.astype(bool), 0.0, fine)
    return fine.ravel()


# --------------------------------------------------------------------------------------
# Nernst model (Sec. II.D, Eqs. nernst-eta-inst-def, nernst-model-eta-update,
# nernst-model-s-update; explicit form Algorithm 8)
# --------------------------------------------------------------------------------------

def nernst_iterate(p: Problem, omega: float, tol: float, cfl: float = 0.4,
                   local_dt: bool = True, max_steps: int = 2_000_000, check_every: int = 10):
    """The explicit Nernst model for the affine-kinetics problem p (alpha = 1/2).

    Electrode cells (fluid cells with k0 a_c > 0) are Dirichlet cells holding
    s = sigma(V~ - eta~) (Eq. nernst-model-s-update); every step applies the transport
    operator (advection + diffusion, the SBV operator without its source) to the current
    state, the electrode cells' transport rate T_c = (L_T s + b_T)_c plays the part of
    Delta s_elec / Delta t in Eq. nernst-eta-inst-def,
        eta~_I = 2 asinh( -T_c / (2 k0 a_c sqrt(s_c (1 - s_c))) ),
    eta~ <- (1 - w_c) eta~ + w_c eta~_I (Eq. nernst-model-eta-update), and the other fluid
    cells take the explicit step s <- s + dt T. The paper leaves the relaxation open; the
    update is a fixed-point map of eta~ whose slope at a cell is
        G_c = (-d_c sqrt(s(1-s)) / (k0 a_c) + (1 - 2s) sinh(eta~/2)) / cosh(eta~/2)
    (d_c the transport diagonal), so one global weight must stay below 2 / (1 + |G_c|) at
    every electrode cell, about 1e-3 for slow kinetics. Each cell therefore uses
    w_c = omega / (1 + |G_c|) at the current state: stable for omega in (0, 1], the
    local Newton step at omega = 1. Start: s = s_in, eta~ = 0, electrode
    cells at sigma(V~). Stops when the SBV residual tau RMS(RHS_SBV(s)) < tol, the steady
    state of both models (Sec. III.C: they converge to the same solution).
    Returns (s, eta_t, steps); eta_t is 0 off the electrode cells."""
    if abs(p.alpha - 0.5) > 1e-15:
        raise ValueError("the Nernst model is derived for alpha = 1/2 (Eq. source-term-bv)")
    sbv = assemble(p)                                   # residual of the SBV problem
    tr = assemble(dataclasses.replace(p, k0=0.0))       # transport only
    kin = sbv.kin
    kappa = sbv.kappa                                   # k0 a_c
    elec = sbv.unknown & (kappa > 0)
    inner = sbv.unknown & ~elec
    d = step_diagonal(sbv)
    d_t = -tr.L.diagonal()                              # transport diagonal
    if local_dt:
        dt = np.where(inner, cfl / np.where(d > 0, d, 1.0), 0.0)
    else:
        dt = np.where(inner, dt_global(sbv, cfl), 0.0)
    s = initial_state(sbv, p.s_in)
    eta_t = np.zeros(s.size)
    s[elec] = 1.0 / (1.0 + np.exp(-(kin.Vt - eta_t[elec])))
    n = 0
    while n < max_steps:
        T = tr.L @ s + tr.b
        se = s[elec]
        root = np.sqrt(se * (1.0 - se))
        eta_i = 2.0 * np.arcsinh(-T[elec] / (2.0 * kappa[elec] * root))
        e = eta_t[elec]
        G = (-d_t[elec] * root / kappa[elec] + (1.0 - 2.0 * se) * np.sinh(e / 2.0)) / \
            np.cosh(e / 2.0)
        w = omega / (1.0 + np.abs(G))
        eta_t[elec] = (1.0 - w) * e + w * eta_i
        s_new = s + dt * T
        s_new[elec] = 1.0 / (1.0 + np.exp(-(kin.Vt - eta_t[elec])))
        s = s_new
        n += 1
        if n % check_every == 0 and residual(sbv, s) < tol:
            break
    return s, eta_t, n
