"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks oracle/soc.py against something other than itself: numbers the paper
prints, closed forms, exact discrete identities, symmetries, bounds, limits and brute
force, chosen so that a dropped term, a wrong sign or index, or a transposed operand in
the oracle fails at least one of them.
"""
import dataclasses
import math
import os

import numpy as np
import scipy.sparse.linalg as spla
import pytest

from oracle import soc
from tests._cases import channel_1d, fiber_case, problem_from_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[parts[0]] = (float(parts[1]), float(parts[2]))
    return out


# ---------------------------------------------------------------- kinetics (Sec. II.B-D)

def test_kinetics_values_printed_in_paper():
    g = _golden("kinetics_paper.txt")
    kin = soc.kinetics(0.0, 0.5, 2, 298.0)
    v, tol = g["V_T_volts"]
    assert abs(kin.V_T - v) < tol
    # Nernst overpotential (V_T/n_e) logit(s) at s = 0.99: invert s_eq(V_ar) = 0.99
    v, tol = g["nernst_overpotential_s099_V"]
    # s_eq = sigma(n_e V_ar / V_T) -> V_ar = V_T/n_e * logit(s_eq); check via kinetics()
    var = kin.V_T / 2 * math.log(0.99 / 0.01)
    assert abs(soc.kinetics(-var).s_eq - 0.99) < 1e-12
    assert abs(var - v) < tol
    v, tol = g["s_eq_at_Var_0"]
    assert abs(kin.s_eq - v) <= tol


@pytest.mark.parametrize("eta", [-0.2, -0.1, -0.05, -0.02, 0.0, 0.03])
@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_affine_rate_law_matches_butler_volmer_form(eta, alpha):
    """Eq. rate-from-soc-gen equals Eq. source-term-bv-gen / (a k0 C_T) with eta~ from
    Eq. etat-from-s, pointwise in s."""
    kin = soc.kinetics(eta, alpha)
    s = np.linspace(1e-3, 1 - 1e-3, 201)
    a = soc.rate_affine(s, kin)
    b = soc.rate_bv(s, kin.Vt, alpha)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * kin.A)
    # zero at s_eq = sigma(V~) (Eq. seq-from-Var)
    assert abs(soc.rate_affine(kin.s_eq, kin)) < 1e-12 * kin.A


def test_alpha_half_reduces_to_cosh_form():
    """Eq. rate-from-soc: R~ = e^{V~/2} - 2 cosh(V~/2) s at alpha = 1/2."""
    for eta in (-0.1, -0.05, 0.02):
        kin = soc.kinetics(eta, 0.5)
        s = np.linspace(0, 1, 11)
        ref = math.exp(kin.Vt / 2) - 2 * math.cosh(kin.Vt / 2) * s
        assert np.allclose(soc.rate_affine(s, kin), ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------- exact 1D discrete closed form

def _closed_form_1d(n, a, d, K, g, E_in):
    """e_k = s_k - s* of the 1D channel: rows
    k=0:   (a + d + g d + K) e0 - d e1 = (a + g d) E_in
    0<k<n-1: a(e_{k-1}-e_k) + d(e_{k+1} - 2e_k + e_{k-1}) - K e_k = 0
    k=n-1: -(a + d) e_{n-2} + (a + d + K) e_{n-1} = 0,
    solved through the roots of d r^2 - (a + 2d + K) r + (a + d) = 0."""
    k = np.arange(n, dtype=np.float64)
    if d == 0.0:
        return E_in * (a / (a + K)) ** (k + 1)
    disc = math.sqrt((a + K) ** 2 + 4 * d * K)
    rs = ((a + 2 * d + K) - disc) / (2 * d)   # small root
    rl = ((a + 2 * d + K) + disc) / (2 * d)   # large root, normalised at the outlet
    phi_s = rs ** k
    phi_l = rl ** (k - (n - 1))

    def row0(v):
        return (a + d + g * d + K) * v[0] - d * v[1]

    def rowN(v):
        return -(a + d) * v[n - 2] + (a + d + K) * v[n - 1]

    M = np.array([[row0(phi_s), row0(phi_l)], [rowN(phi_s), rowN(phi_l)]])
    P, Q = np.linalg.solve(M, np.array([(a + g * d) * E_in, 0.0]))
    return P * phi_s + Q * phi_l


@pytest.mark.parametrize("D", [4e-10, 0.0, 4e-9])
@pytest.mark.parametrize("inlet_bc", ["face", "ghost"])
@pytest.mark.parametrize("k0,m", [(1e-7, 1.0), (1e-6, 0.7), (0.0, 1.0)])
@pytest.mark.parametrize("h", [1.25e-6, 5e-6])
def test_1d_channel_exact_discrete_closed_form(D, inlet_bc, k0, m, h):
    n, w = 40, 0.01
    solid, U, V, W, _ = channel_1d(n, w, h)
    eta, s_in = -0.08, 0.2
    area = np.full(solid.shape, m)
    p = soc.Problem(solid, U, V, W, h, D, s_in, k0=k0, eta=eta, area_mult=area,
                    inlet_bc=inlet_bc)
    op = soc.assemble(p)
    s = soc.steady_state(op).reshape(solid.shape)[:, 1, 1]
    kin = soc.kinetics(eta)
    K = k0 * m * 4 / h * kin.B
    s_star = kin.A / kin.B if K > 0 else s_in
    g = 2.0 if inlet_bc == "face" else 1.0
    e = _closed_form_1d(n, w / h, D / h ** 2, K, g, s_in - s_star)
    assert np.allclose(s - s_star, e, rtol=0, atol=1e-12 * max(abs(s_in - s_star), 0.1))
    if k0 == 0.0:
        assert np.allclose(s, s_in, atol=1e-13)


def test_residual_is_tau_times_rms_with_tau_the_residence_time():
    """Eq. convergence-bv-change on the 1D channel at s = s_in in every fluid cell: the
    advective and diffusive fluxes cancel (a uniform state, the inlet face at s_in), so
    RHS_c = k0 a R~(s_in) in each of the n cells, with a = 4/h (four fiber faces); and
    tau = V_f / Q = n h^3 / (w h^2) = n h / w, the time the flow takes to cross the
    channel. The residual is then tau k0 (4/h) |R~(s_in)|, up to the rounding of the
    transport terms that cancel (a few ulps of (w/h + 6 D/h^2) s_in per cell)."""
    n, w, h, D = 40, 0.01, 1.25e-6, 4e-10
    solid, U, V, W, _ = channel_1d(n, w, h)
    for s_in, eta, k0 in ((0.2, -0.08, 1e-6), (0.9, -0.02, 3e-7)):
        p = soc.Problem(solid, U, V, W, h, D, s_in, k0=k0, eta=eta)
        op = soc.assemble(p)
        assert abs(op.tau - n * h / w) <= 1e-15 * n * h / w
        s = soc.initial_state(op, s_in)
        r = soc.rhs(op, s)[op.unknown]
        want = k0 * 4.0 / h * float(soc.rate_bv(s_in, op.kin.Vt))
        ulp = 8 * np.finfo(np.float64).eps * (w / h + 6 * D / h ** 2) * s_in
        assert r.size == n and np.max(np.abs(r - want)) <= ulp
        assert abs(soc.residual(op, s) - n * h / w * abs(want)) <= n * h / w * ulp


def test_n_wall_brute_force():
    """n_wall(c) = number of solid cells among the six face neighbours inside the lattice,
    counted cell by cell with explicit neighbour offsets on a random mask."""
    rng = np.random.default_rng(9)
    solid = (rng.uniform(size=(5, 4, 3)) < 0.45).astype(np.uint8)
    got = soc.n_wall(solid.astype(bool))
    nz, ny, nx = solid.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                cnt = 0
                for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                   (0, 0, 1), (0, 0, -1)):
                    kk, jj, ii = k + dk, j + dj, i + di
                    if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx and solid[kk, jj, ii]:
                        cnt += 1
                assert got[k, j, i] == cnt, (k, j, i)


def test_plug_flow_continuum_limit_first_order():
    """With D = 0 and a fixed area per volume (a = 4/h0, via m = h/h0) the discrete
    solution approaches the plug-flow exponential s(z) = s_eq + (s_in - s_eq)
    exp(-K z / w) at first order in h (first-order upwinding)."""
    L, w, eta, s_in, k0, h0 = 50e-6, 0.01, -0.05, 0.1, 1e-5, 1.25e-6
    kin = soc.kinetics(eta)
    K = k0 * 4 / h0 * kin.B
    errs = []
    for n in (20, 40, 80, 160):
        h = L / n
        solid, U, V, W, _ = channel_1d(n, w, h)
        p = soc.Problem(solid, U, V, W, h, 0.0, s_in, k0=k0, eta=eta,
                        area_mult=np.full(solid.shape, h / h0))
        s = soc.steady_state(soc.assemble(p)).reshape(solid.shape)[:, 1, 1]
        z = (np.arange(n) + 1.0) * h     # outflow face of each cell
        exact = kin.s_eq + (s_in - kin.s_eq) * np.exp(-K * z / w)
        errs.append(np.max(np.abs(s - exact)))
    assert errs[0] > 1e-3
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), ratios


# --------------------------------------------------- structure of the 3D operator

def _p3(dims=(16, 16, 32), **over):
    return problem_from_case(fiber_case(dims), soc, **over)


def test_m_matrix_sign_structure_and_monotone_step():
    """Upwinding + diffusion + a decreasing source give an M-matrix: off-diagonals >= 0,
    diagonal < 0; I + dt L is non-negative for C_CFL <= 1 (monotone update)."""
    p = _p3()
    op = soc.assemble(p)
    L = op.L.tocoo()
    off = L.row != L.col
    assert np.all(L.data[off] >= 0.0)
    fl = p.solid.ravel() == 0
    assert np.all(op.L.diagonal()[fl] < 0.0)
    dt = soc.dt_global(op, 1.0)
    F = (dt * op.L).tocsr()
    F.setdiag(F.diagonal() + 1.0)
    Fd = F[fl][:, fl]
    assert Fd.min() >= -1e-15
    # the flow really has transverse components on this lattice
    assert np.abs(p.U).max() > 0.2 * np.abs(p.W).max()
    assert np.abs(p.V).max() > 0.2 * np.abs(p.W).max()


def test_uniform_state_is_steady_without_reaction():
    """k0 = 0 and s = s_in everywhere: every face flux balances for a divergence-free
    velocity field, so RHS vanishes (needs each face velocity on the right face)."""
    p = _p3(k0=0.0, s_in=0.37)
    op = soc.assemble(p)
    s = np.where(p.solid.ravel() == 0, 0.37, 0.0)
    r = soc.rhs(op, s)
    scale = 0.37 * np.abs(p.W).max() / p.h
    assert np.abs(r).max() < 1e-10 * scale


def test_conservation_identity_any_state():
    """sum_c h^3 RHS_c = (F_in - F_out + I_tot) / (n_e F c0) for any s (telescoping)."""
    p = _p3()
    op = soc.assemble(p)
    rng = np.random.default_rng(0)
    s = np.where(p.solid.ravel() == 0, rng.uniform(0, 1, p.solid.size), 0.0)
    o = soc.outputs(p, op, s)
    lhs = p.h ** 3 * float(np.sum(soc.rhs(op, s)))
    rhs_ = (o.F_in - o.F_out + o.I_tot) / (p.n_e * soc.FARADAY * p.c0)
    assert abs(lhs - rhs_) < 1e-11 * (o.F_in + o.F_out) / (p.n_e * soc.FARADAY * p.c0)


def test_steady_state_mass_balance_and_bounds():
    """At steady state I_tot = F_out - F_in (Eq. convergence-bv-flow) and
    min(s_in, s_eq) <= s <= max(s_in, s_eq) (discrete maximum principle)."""
    p = _p3()
    op = soc.assemble(p)
    s = soc.steady_state(op)
    o = soc.outputs(p, op, s)
    assert o.mass_balance_rel < 1e-9
    fl = p.solid.ravel() == 0
    lo, hi = min(p.s_in, op.kin.s_eq), max(p.s_in, op.kin.s_eq)
    assert s[fl].min() >= lo - 1e-11 and s[fl].max() <= hi + 1e-11
    assert o.residual < 1e-12
    # the two printed utilisation expressions agree once the second is corrected for
    # s_in != 0 and for the inlet diffusive flux
    U_corr = o.U_outlet_form - (o.F_in - o.F_in_adv) / (
        p.n_e * soc.FARADAY * p.c0 * op.Q * (1 - p.s_in))
    assert abs(o.U - U_corr) < 1e-9 * abs(o.U)


def test_inlet_at_equilibrium_is_steady():
    p = _p3()
    kin = soc.kinetics(p.eta)
    p2 = _p3(s_in=kin.s_eq)
    op = soc.assemble(p2)
    s = soc.steady_state(op)
    fl = p.solid.ravel() == 0
    assert np.allclose(s[fl], kin.s_eq, atol=1e-11)


def test_xy_transposition_symmetry():
    """Swapping the x and y axes of the geometry and the flow transposes the solution."""
    p = _p3()
    s = soc.steady_state(soc.assemble(p)).reshape(p.solid.shape)
    solid_t = np.ascontiguousarray(p.solid.transpose(0, 2, 1))
    U_t = np.ascontiguousarray(p.V.transpose(0, 2, 1))
    V_t = np.ascontiguousarray(p.U.transpose(0, 2, 1))
    W_t = np.ascontiguousarray(p.W.transpose(0, 2, 1))
    pt = soc.Problem(solid_t, U_t, V_t, W_t, p.h, p.D, p.s_in, k0=p.k0, eta=p.eta)
    st = soc.steady_state(soc.assemble(pt)).reshape(solid_t.shape)
    assert np.allclose(st, s.transpose(0, 2, 1), rtol=0, atol=1e-13)


def test_x_mirror_symmetry():
    """Mirroring x (i -> nx-1-i) with U negated on mirrored faces mirrors the solution."""
    p = _p3()
    s = soc.steady_state(soc.assemble(p)).reshape(p.solid.shape)
    pm = soc.Problem(p.solid[:, :, ::-1].copy(), -p.U[:, :, ::-1].copy(),
                     p.V[:, :, ::-1].copy(), p.W[:, :, ::-1].copy(), p.h, p.D, p.s_in,
                     k0=p.k0, eta=p.eta)
    sm = soc.steady_state(soc.assemble(pm)).reshape(p.solid.shape)
    assert np.allclose(sm, s[:, :, ::-1], rtol=0, atol=1e-13)


# --------------------------------------------- iteration and solver (brute force)

def test_dense_lu_brute_force_small_lattice():
    p = problem_from_case(fiber_case((6, 6, 10), diameter=2.0, porosity=0.8), soc)
    for mode in ("sbv", "umt"):
        op = soc.assemble(p, mode)
        u = op.unknown
        A = op.L[u][:, u].toarray()
        rhs_u = -(op.b[u] + op.L[u] @ op.fixed)
        x = np.linalg.solve(A, rhs_u)
        s = soc.steady_state(op)
        assert np.allclose(s[u], x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("local_dt", [False, True])
def test_explicit_iteration_reaches_the_steady_state(local_dt):
    """The paper's pseudo-time loop (Algorithm 7 with dt from a CFL bound) converges to
    the solution of RHS = 0; a per-cell dt changes only the path, not the fixed point."""
    p = problem_from_case(fiber_case((8, 8, 12), diameter=3.0), soc)
    op = soc.assemble(p)
    ref = soc.steady_state(op)
    s, n = soc.explicit_iterate(op, 0.4, 1e-13, s0=soc.initial_state(op, p.s_in),
                                check_every=50, local_dt=local_dt)
    assert n < 10_000_000
    assert np.abs(s - ref).max() < 1e-11


def test_grid_fits_gmres_matches_direct():
    """The large-system solver path agrees with SuperLU on a mid-size lattice."""
    p = _p3((16, 16, 32))
    op = soc.assemble(p)
    a = soc.steady_state(op, direct_max=10 ** 9)
    b = soc.steady_state(op, direct_max=0)
    assert np.abs(a - b).max() < 1e-12


# ------------------------------------------------------------------------- U_mt

def test_umt_bounds_and_upper_bound_on_utilisation():
    """0 <= U_mt <= 1 and U <= U_mt for s_in = 0 (Eq. umt-def and the text after it)."""
    for eta in (-0.2, -0.1, -0.02):
        p = _p3(s_in=0.0, eta=eta)
        op = soc.assemble(p)
        s = soc.steady_state(op)
        o = soc.outputs(p, op, s)
        u = soc.umt(p)
        assert 0.0 <= u <= 1.0
        assert o.U <= u + 1e-12


def test_umt_is_the_fast_kinetics_limit():
    """k0 -> infinity with s_eq -> 1 and s_in = 0 drives the SBV state to the U_mt state
    (Eqs. np-fast-interior/np-fast-boundary)."""
    p = _p3(s_in=0.0, eta=-0.35, k0=10.0)
    op = soc.assemble(p)
    s = soc.steady_state(op)
    o = soc.outputs(p, op, s)
    u = soc.umt(p)
    assert abs(o.U_outlet_form - u) < 1e-5
    s_mt = soc.steady_state(soc.assemble(p, "umt"))
    fl = p.solid.ravel() == 0
    assert np.abs(s[fl] - s_mt[fl]).max() < 1e-5


@pytest.mark.parametrize("inlet_bc", ["face", "ghost"])
def test_umt_closed_form_of_a_channel_inside_electrode_cells(inlet_bc):
    """5 x 5 x n lattice with a solid outer ring: the centre column touches no fiber; its
    four neighbours do, so in the U_mt problem (Eqs. np-fast-interior/np-fast-boundary)
    they are held at 1, and the inlet is at 0. With flow only in the centre column the
    centre's rows are the 1D channel's with K = 4 D / h^2 towards s* = 1 and E_in = -1, and
    U_mt (Eq. umt-def) is the centre's outlet value."""
    n, w, h, D = 30, 0.004, 1.25e-6, 4e-10
    solid = np.ones((n, 5, 5), dtype=np.uint8)
    solid[:, 1:4, 1:4] = 0
    U = np.zeros((n, 5, 6))
    V = np.zeros((n, 6, 5))
    W = np.zeros((n + 1, 5, 5))
    W[:, 2, 2] = w
    p = soc.Problem(solid, U, V, W, h, D, 0.7, k0=3e-6, eta=-0.1, inlet_bc=inlet_bc)
    g = 2.0 if inlet_bc == "face" else 1.0
    e = _closed_form_1d(n, w / h, D / h ** 2, 4 * D / h ** 2, g, -1.0)
    op = soc.assemble(p, "umt")
    s = soc.steady_state(op).reshape(solid.shape)
    assert np.allclose(s[:, 2, 2], 1.0 + e, rtol=0, atol=1e-12)
    ring = np.ones((5, 5), dtype=bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = ring[2, 2] = False
    assert np.all(s[:, ring] == 1.0)
    assert abs(soc.umt(p) - (1.0 + e[-1])) <= 1e-12


def test_umt_independent_of_kinetics_and_inlet():
    a = soc.umt(_p3(s_in=0.3, eta=-0.1, k0=1e-7))
    b = soc.umt(_p3(s_in=0.9, eta=-0.02, k0=5e-6))
    assert a == b


# ------------------------------------------------------------------ prolongation

def test_prolongation_injection():
    """Every fine cell of a non-cubic lattice against its parent, cell by cell: fine fluid
    cells under a fluid parent take the parent's value, a fine fluid cell under a solid
    parent the mean of the parent's fluid 6-neighbours, fine solid cells 0."""
    rng = np.random.default_rng(3)
    solid_c = np.zeros((4, 3, 5), dtype=np.uint8)
    solid_c[1, 1, 1] = 1
    solid_c[2, 0, 3] = 1
    sc = rng.uniform(size=solid_c.size) * (solid_c.ravel() == 0)
    solid_f = solid_c.repeat(2, 0).repeat(2, 1).repeat(2, 2).copy()
    solid_f[2, 2, 2] = 0   # fine fluid cell under the solid coarse parent (1, 1, 1)
    sf = soc.prolong(sc, solid_c, solid_f, 0.5).reshape(solid_f.shape)
    scr = sc.reshape(solid_c.shape)
    nz, ny, nx = solid_f.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                parent = (k // 2, j // 2, i // 2)
                if solid_f[k, j, i]:
                    assert sf[k, j, i] == 0.0
                elif not solid_c[parent]:
                    assert sf[k, j, i] == scr[parent], (k, j, i)
    nb = [scr[0, 1, 1], scr[2, 1, 1], scr[1, 0, 1], scr[1, 2, 1], scr[1, 1, 0], scr[1, 1, 2]]
    assert abs(sf[2, 2, 2] - np.mean(nb)) < 1e-15
    assert sf[3, 3, 3] == 0.0


# ---------------------------------------------------------------- adjoint (FD pinned)

def _fd_objective(p, objective):
    if objective == "U_mt":
        return soc.umt(p)
    op = soc.assemble(p)
    o = soc.outputs(p, op, soc.steady_state(op))
    return o.I_tot if objective == "I_tot" else o.U


@pytest.mark.parametrize("objective,kmode", [("I_tot", 0), ("U", 0), ("U_mt", 0),
                                            ("I_tot", 1), ("U", 1)])
def test_oracle_adjoint_matches_central_differences(objective, kmode):
    """The adjoint gradients equal central finite differences of the steady-state solve
    with respect to the per-voxel area multiplier and the velocity scale (kinetics mode 1:
    of Newton solves of the nonlinear problem, adjoint of the Jacobian at the solution)."""
    import dataclasses
    base = _p3((8, 8, 12), kinetics_mode=kmode)
    rng = np.random.default_rng(40)
    nw = soc.n_wall(base.solid.astype(bool)).ravel()
    fl = base.solid.ravel() == 0
    m = np.where(fl & (nw > 0), np.exp(0.3 * rng.standard_normal(base.solid.size)), 1.0)
    p = dataclasses.replace(base, area_mult=m.reshape(base.solid.shape), k0=2e-6)
    adj = soc.adjoint(p, None, objective)
    walls = np.flatnonzero(fl & (nw > 0))
    pick = rng.choice(walls, 5, replace=False)
    for c in pick:
        eps = 1e-6 * m[c]
        mp, mm = m.copy(), m.copy()
        mp[c] += eps
        mm[c] -= eps
        jp = _fd_objective(dataclasses.replace(p, area_mult=mp.reshape(p.solid.shape)), objective)
        jm = _fd_objective(dataclasses.replace(p, area_mult=mm.reshape(p.solid.shape)), objective)
        fd = (jp - jm) / (2 * eps)
        if objective == "U_mt":
            assert fd == 0.0 and adj["d_area_mult"][c] == 0.0
        else:
            assert abs(fd - adj["d_area_mult"][c]) <= 1e-5 * abs(fd), (c, fd, adj["d_area_mult"][c])
    eps = 1e-6
    jp = _fd_objective(dataclasses.replace(p, beta=1 + eps), objective)
    jm = _fd_objective(dataclasses.replace(p, beta=1 - eps), objective)
    fd = (jp - jm) / (2 * eps)
    assert abs(fd - adj["d_beta"]) <= 1e-6 * abs(fd), (fd, adj["d_beta"])


# ------------------------------------ kinetics mode 1: uniform activation overpotential

def test_uniform_eta_rate_is_the_butler_volmer_source():
    """Eq. source-term-bv (alpha = 1/2): R~ = 2 sqrt(s(1-s)) sinh(eta~/2); for any alpha,
    substituting eta~ = V~ - logit(s) (Eq. etat-from-s) gives the affine law
    (Eq. rate-from-soc-gen); R~ vanishes at s = 0 and s = 1 and is positive between them
    for a reducing eta~ > 0."""
    s = np.linspace(0.0, 1.0, 41)
    for etat in (0.3, 3.9, 7.79):
        ref = 2.0 * np.sqrt(s * (1.0 - s)) * math.sinh(etat / 2.0)
        assert np.allclose(soc.rate_uniform(s, etat, 0.5), ref, rtol=1e-13, atol=1e-13)
        r = soc.rate_uniform(s, etat, 0.5)
        assert r[0] == 0.0 and r[-1] == 0.0 and np.all(r[1:-1] > 0.0)
    si = np.linspace(0.01, 0.99, 33)
    for alpha in (0.3, 0.5, 0.7):
        for eta in (-0.1, -0.03, 0.02):
            kin = soc.kinetics(eta, alpha)
            etat = kin.Vt - np.log(si / (1.0 - si))
            got = np.array([soc.rate_uniform(x, e, alpha) for x, e in zip(si, etat)])
            assert np.allclose(got, soc.rate_affine(si, kin), rtol=1e-11, atol=1e-12)


def test_uniform_eta_slope_matches_central_differences():
    s = np.linspace(0.02, 0.98, 25)
    for alpha in (0.3, 0.5, 0.7):
        for etat in (0.5, 7.79):
            e = 1e-6
            fd = (soc.rate_uniform(s + e, etat, alpha) - soc.rate_uniform(s - e, etat, alpha)) / (2 * e)
            assert np.allclose(soc.rate_uniform_slope(s, etat, alpha), fd, rtol=1e-7, atol=1e-7)


def _bisect(f, lo, hi):
    flo = f(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("alpha", [0.5, 0.3])
def test_uniform_eta_channel_without_diffusion_is_solved_cell_by_cell(alpha):
    """With D = 0 the 1D channel's rows decouple downstream: cell k solves
    (w/h)(s_{k-1} - s_k) + kappa R~(s_k) = 0 (s_{-1} = s_in), a concave scalar equation
    with one root in [s_{k-1}, 1]; bisection cell by cell gives the exact discrete state
    that the oracle's Newton solve of the assembled system must reproduce."""
    n, w, h, k0, m, eta, s_in = 30, 0.004, 1.25e-6, 5e-6, 0.8, -0.06, 0.2
    solid, U, V, W, _ = channel_1d(n, w, h)
    p = soc.Problem(solid, U, V, W, h, 0.0, s_in, k0=k0, eta=eta, alpha=alpha,
                    area_mult=np.full(solid.shape, m), kinetics_mode=1)
    op = soc.assemble(p)
    s = soc.steady_state(op).reshape(solid.shape)[:, 1, 1]
    etat = soc.kinetics(eta, alpha).Vt
    kappa = k0 * m * 4 / h
    prev, ref = s_in, []
    for _ in range(n):
        f = lambda x, pr=prev: (w / h) * (pr - x) + kappa * float(soc.rate_uniform(x, etat, alpha))
        prev = _bisect(f, prev, 1.0)
        ref.append(prev)
    assert np.max(np.abs(s - np.array(ref))) < 1e-13
    assert ref[-1] > s_in + 0.05       # the reaction matters


def test_uniform_eta_plug_flow_closed_form_first_order():
    """alpha = 1/2, D = 0: ds/dz = (k0 a/w) 2 sqrt(s(1-s)) sinh(eta~/2) integrates with
    s = sin^2(theta) to s(z) = sin^2(asin(sqrt(s_in)) + (k0 a/w) sinh(eta~/2) z); the
    upwind solution approaches it at first order in h."""
    L, w, eta, s_in, k0, h0 = 50e-6, 0.01, -0.05, 0.1, 1e-5, 1.25e-6
    etat = soc.kinetics(eta).Vt
    c = k0 * 4 / h0 * math.sinh(etat / 2) / w
    assert math.asin(math.sqrt(s_in)) + c * L < math.pi / 2
    errs = []
    for n in (20, 40, 80, 160):
        h = L / n
        solid, U, V, W, _ = channel_1d(n, w, h)
        p = soc.Problem(solid, U, V, W, h, 0.0, s_in, k0=k0, eta=eta,
                        area_mult=np.full(solid.shape, h / h0), kinetics_mode=1)
        s = soc.steady_state(soc.assemble(p)).reshape(solid.shape)[:, 1, 1]
        z = (np.arange(n) + 1.0) * h
        exact = np.sin(math.asin(math.sqrt(s_in)) + c * z) ** 2
        errs.append(np.max(np.abs(s - exact)))
    assert errs[0] > 1e-3
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), ratios


@pytest.mark.parametrize("local_dt,k0", [(True, 2e-6), (False, 2e-6), (True, 6e-6),
                                         (False, 6e-6)])
def test_uniform_eta_3d_newton_explicit_and_balance(local_dt, k0):
    """On a fiber lattice: the Newton state has RHS = 0, the explicit pseudo-time loop
    (clip guard never active at the end) reaches it, I_tot = F_out - F_in holds, and
    s_in <= s <= 1 (the source is >= 0 for a reducing overpotential). k0 = 6e-6 drives
    wall cells to s > 0.9999, where the rate's slope is steep and the step cap acts."""
    p = _p3((12, 12, 24), kinetics_mode=1, k0=k0)
    op = soc.assemble(p)
    assert op.nonlinear
    s = soc.steady_state(op)
    assert soc.residual(op, s) < 1e-12
    o = soc.outputs(p, op, s)
    assert o.mass_balance_rel < 1e-10
    fl = p.solid.ravel() == 0
    assert np.all(s[fl] >= p.s_in - 1e-14) and np.all(s[fl] < 1.0)
    if k0 > 5e-6:
        assert s[fl].max() > 0.9999
        cap = soc.nonlinear_step_cap(op, s, 0.4)
        assert np.any(cap[op.unknown] < soc.dt_global(op, 0.4))
    se, n = soc.explicit_iterate(op, 0.4, 1e-12, s0=soc.initial_state(op, p.s_in),
                                 check_every=50, local_dt=local_dt)
    assert np.max(np.abs(se - s)) < 1e-10
    # mode 1 is a different problem from mode 0 at the same overpotential
    s0 = soc.steady_state(soc.assemble(_p3((12, 12, 24), k0=k0)))
    assert np.max(np.abs(s0 - s)) > 1e-4


def test_uniform_eta_zero_overpotential_is_inert():
    """eta = 0 gives eta~ = 0 and R~ = 0: with divergence-free faces s = s_in is steady."""
    p = _p3((12, 12, 24), kinetics_mode=1, k0=2e-6, eta=0.0)
    op = soc.assemble(p)
    s = soc.initial_state(op, p.s_in)
    assert np.max(np.abs(soc.rhs(op, s))) < 1e-9 * np.max(np.abs(op.L.diagonal()))


# ------------------------------------------------------------------ grid convergence

def _restrict_fluid_mean(s_f, fluid_f):
    """2x coarsening: the mean of a coarse cell's fluid children (Sec. IV compares levels
    by averaging the fine solution onto the coarse cells)."""
    nz, ny, nx = s_f.shape
    a = (s_f * fluid_f).reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
    n = fluid_f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
    return np.where(n > 0, a / np.maximum(n, 1), 0.0), n > 0


@pytest.mark.parametrize("seed", [5, 6])
def test_grid_convergence_same_fibers_three_levels(seed):
    """The same analytic fibers rasterised at h, h/2, h/4 (8x8x16 to 32x32x64, each level
    with its own flood fill and flow): the RMS difference between a level and the next
    finer one (restricted by fluid-cell averaging) falls, and so does the change in U."""
    from paper_2502_08034_gb300 import synth
    cases = synth.multilevel_cases((32, 32, 64), 3, 0.8, 8.0, seed, 0.01, -0.10, 0.5, 1e-10)
    sols = []
    for c in cases:
        p = problem_from_case(c, soc)
        op = soc.assemble(p)
        s = soc.steady_state(op)
        sols.append((s.reshape(c.solid.shape), c.solid == 0, soc.outputs(p, op, s).U))
    errs = []
    for lev in range(2):
        sc, fc, _ = sols[lev]
        r, has = _restrict_fluid_mean(*sols[lev + 1][:2])
        m = fc & has
        errs.append(float(np.sqrt(np.mean((r[m] - sc[m]) ** 2))))
    assert errs[1] < errs[0], errs
    dU = [abs(sols[1][2] - sols[0][2]), abs(sols[2][2] - sols[1][2])]
    assert dU[1] < dU[0], dU


# ------------------------------------------------------------------ Nernst model

def _nernst_problem(k0=7.2e-5, **over):
    return _p3((12, 12, 24), k0=k0, **over)


@pytest.mark.parametrize("local_dt", [True, False])
def test_nernst_model_reaches_the_sbv_steady_state(local_dt):
    """The Nernst model's fixed point is the SBV steady state (Sec. III.C: both models
    converge to the same solution), and there eta~ = V~ - logit(s) on electrode cells
    (Eq. s-from-etat) with the Butler-Volmer source of Eq. source-term-bv balancing
    transport (Eq. nernst-model-elec)."""
    p = _nernst_problem()
    ref = soc.steady_state(soc.assemble(p))
    s, eta_t, n = soc.nernst_iterate(p, 1.0 if local_dt else 0.5, 1e-12, local_dt=local_dt)
    assert np.max(np.abs(s - ref)) < 1e-10 * np.max(np.abs(ref))
    op = soc.assemble(p)
    elec = op.unknown & (op.kappa > 0)
    kin = op.kin
    assert np.max(np.abs(eta_t[elec] - (kin.Vt - np.log(s[elec] / (1 - s[elec]))))) < 1e-8
    tr = soc.assemble(dataclasses.replace(p, k0=0.0))
    T = (tr.L @ s + tr.b)[elec]
    src = op.kappa[elec] * 2 * np.sqrt(s[elec] * (1 - s[elec])) * np.sinh(eta_t[elec] / 2)
    assert np.max(np.abs(T + src)) < 1e-6 * np.max(np.abs(src))
    assert np.all(eta_t[~elec] == 0.0)


def test_nernst_model_fast_kinetics_limit():
    """k0 -> infinity: the electrode cells approach the Dirichlet value s_eq = sigma(V~) of
    Eq. np-fast-boundary at first order in 1/k0 (a 100x faster rate constant brings them
    about 100x closer), and eta~ falls towards 0."""
    errs, etas = [], []
    for k0 in (1e-2, 1.0):
        p = _nernst_problem(k0=k0)
        op = soc.assemble(p)
        elec = op.unknown & (op.kappa > 0)
        s, eta_t, _ = soc.nernst_iterate(p, 1.0, 1e-8)
        errs.append(np.max(np.abs(s[elec] - op.kin.s_eq)))
        etas.append(np.max(np.abs(eta_t[elec])))
    assert 80 < errs[0] / errs[1] < 120, errs
    assert etas[1] < etas[0] / 5, etas


def test_nernst_model_needs_alpha_one_half():
    with pytest.raises(ValueError):
        soc.nernst_iterate(_nernst_problem(alpha=0.3), 0.5, 1e-8)


@pytest.mark.parametrize("objective", ["I_tot", "U", "U_mt"])
def test_large_problem_adjoint_iteration_equals_the_direct_adjoint(objective):
    """The oracle's path for adjoints beyond its direct-solve size (the explicit
    transposed iteration with local steps) reaches the sparse-LU adjoint: forced here on
    a small lattice with area multipliers (direct_max = 0), to 1e-9 relative in lam and
    in both gradients."""
    import dataclasses
    base = _p3((12, 10, 20))
    rng = np.random.default_rng(3)
    nw = soc.n_wall(base.solid.astype(bool)).ravel()
    fl = base.solid.ravel() == 0
    m = np.where(fl & (nw > 0), np.exp(0.3 * rng.standard_normal(base.solid.size)), 1.0)
    p = dataclasses.replace(base, area_mult=m.reshape(base.solid.shape))
    mode = "umt" if objective == "U_mt" else "sbv"
    s = soc.steady_state(soc.assemble(p, mode))
    a = soc.adjoint(p, s, objective)
    b = soc.adjoint(p, s, objective, direct_max=0, iter_tol=1e-14)
    assert np.abs(b["lam"] - a["lam"]).max() <= 1e-9 * np.abs(a["lam"]).max()
    if objective != "U_mt":
        assert np.abs(b["d_area_mult"] - a["d_area_mult"]).max() <= \
            1e-9 * np.abs(a["d_area_mult"]).max()
    assert abs(b["d_beta"] - a["d_beta"]) <= 1e-9 * abs(a["d_beta"])


def test_transposed_iteration_is_the_transpose_solve():
    """transposed_iterate solves A^T x + g = 0 for a nonsymmetric M-matrix (upwind
    advection): the result satisfies the transposed system, and it differs from the
    solution of the untransposed one."""
    p = _p3((8, 8, 12))
    op = soc.assemble(p)
    u = op.unknown
    A = op.L[u][:, u].tocsr()
    g = np.random.default_rng(5).standard_normal(A.shape[0])
    x, n = soc.transposed_iterate(A, g, 0.4, 1e-13)
    assert n > 0
    assert np.linalg.norm(A.T @ x + g) <= 1e-12 * np.linalg.norm(g)
    y = spla.spsolve(A.tocsc(), -g)
    assert np.abs(x - y).max() > 1e-3 * np.abs(y).max()


def test_host_potential_flow_is_divergence_free_and_thread_independent():
    """The host potential-flow input generator: divergence-free to its tolerance, no flow
    through fibers or side walls, inflow only at the inlet and outflow only at the
    outlet, mean W over fluid z-faces equal to the requested value, and the same bits
    with one thread as with eight."""
    from paper_2502_08034_gb300 import synth
    _, solid = synth.generate_fibers(2, (24, 20, 40), 0.8, 4.0)
    solid = synth.remove_unconnected(solid)
    U1, V1, W1, i1 = synth.potential_flow(solid, 1e-6, 0.003, threads=1)
    U8, V8, W8, i8 = synth.potential_flow(solid, 1e-6, 0.003, threads=8)
    assert np.array_equal(U1, U8) and np.array_equal(V1, V8) and np.array_equal(W1, W8)
    assert i1["max_div_rel"] < 1e-11
    fl = solid == 0
    div = (U1[:, :, 1:] - U1[:, :, :-1]) + (V1[:, 1:, :] - V1[:, :-1, :]) + (W1[1:] - W1[:-1])
    assert np.abs(div[fl]).max() < 1e-11 * 0.003
    assert np.all(U1[:, :, 0] == 0) and np.all(U1[:, :, -1] == 0)
    assert np.all(V1[:, 0, :] == 0) and np.all(V1[:, -1, :] == 0)
    assert np.all(W1[0] >= 0) and np.all(W1[-1] >= 0)
    sx = solid.astype(bool)
    assert np.all(U1[:, :, 1:-1][sx[:, :, 1:] | sx[:, :, :-1]] == 0)
    assert np.all(W1[1:-1][sx[1:] | sx[:-1]] == 0)
    zf = np.concatenate([fl[:1], fl[1:] & fl[:-1], fl[-1:]])
    assert abs(W1[zf].mean() - 0.003) < 1e-15
