"""Seeded synthetic workloads: fiber voxel lattices and potential-flow face velocities.

This module only *produces inputs*. It holds none of the state-of-charge method's
arithmetic (no advection, diffusion, kinetics or sweep); both the CUDA library and the
CPU oracle consume what it returns. Random numbers come from a project-written
SplitMix64 generator (Steele, Lea & Flood 2014), so the same seed gives the same lattice
on every machine.

Geometry (the paper's electrodes are fibers of a few-micron diameter resolved at
h = 1.25 um, Sec. IV): straight cylinders whose axes lie in planes z = z0, at a uniform
random in-plane angle, added one at a time until the fluid fraction first drops to the
target porosity. Fluid that is not 6-connected to the inlet plane is then made solid, so
every fluid cell reaches the inlet Dirichlet condition.

Flow: the paper obtains u from a Navier-Stokes/Chorin solve (Sec. III.A, Algorithm 1).
Here a discrete potential flow stands in for it: phi = 1 on inlet faces, 0 on outlet
faces, no flux through fiber faces and side walls, solved by Jacobi-preconditioned FP64
CG; face velocities are -grad(phi), scaled so that the mean z-velocity over fluid
z-faces equals the requested mean. The result is discretely divergence-free (to the CG
tolerance), which the state-of-charge operator's maximum principle relies on.

Layout: arrays are C-ordered (nz, ny, nx), so the flat cell index is
c = i + nx*(j + ny*k). Face arrays: U (nz, ny, nx+1) with U[k,j,i] on the face between
cells i-1 and i; V (nz, ny+1, nx); W (nz+1, ny, nx) with W[0] the inlet plane and
W[nz] the outlet plane. Velocities are in m/s, positive along +x/+y/+z.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import Optional, Sequence

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) with 53-bit uniform doubles."""

    def __init__(self, seed: int):
        self.state = int(seed) & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def normal(self) -> float:
        """Box-Muller; returns one of the pair (the generator is cheap)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class Fiber:
    """Infinite cylinder, axis in the plane z = z0 through (x0, y0) at angle theta.

    Coordinates are in cell units of the lattice the fiber was drawn on (``unit``
    finest-level cells per unit)."""

    z0: float
    x0: float
    y0: float
    theta: float
    d: float


def rasterise(fibers: Sequence[Fiber], dims, scale: float = 1.0) -> np.ndarray:
    """Solid mask (nz, ny, nx) of the union of fibers; a cell is solid when its centre
    lies within d/2 of a fiber axis. ``scale`` = fiber-coordinate units per cell."""
    nx, ny, nz = dims
    solid = np.zeros((nz, ny, nx), dtype=bool)
    for f in fibers:
        _stamp(solid, f, scale)
    return solid


def _stamp(solid: np.ndarray, f: Fiber, scale: float) -> int:
    """OR one fiber into ``solid``; returns the number of newly solid cells."""
    nz, ny, nx = solid.shape
    r = 0.5 * f.d
    klo = max(0, int(math.floor((f.z0 - r) / scale - 0.5)) - 1)
    khi = min(nz - 1, int(math.ceil((f.z0 + r) / scale - 0.5)) + 1)
    if klo > khi:
        return 0
    x = (np.arange(nx) + 0.5) * scale
    y = (np.arange(ny) + 0.5) * scale
    st, ct = math.sin(f.theta), math.cos(f.theta)
    dperp = np.abs((x[None, :] - f.x0) * st - (y[:, None] - f.y0) * ct)  # (ny, nx)
    added = 0
    for k in range(klo, khi + 1):
        dz = (k + 0.5) * scale - f.z0
        inside = dz * dz + dperp * dperp <= r * r
        if inside.any():
            plane = solid[k]
            added += int(np.count_nonzero(inside & ~plane))
            plane |= inside
    return added


def generate_fibers(seed: int, dims, porosity: float, diameter, max_fibers: int = 1_000_000):
    """Draw fibers until the fluid fraction first reaches ``porosity`` or below.

    Per fiber the draws are z0 ~ U(0, nz), x0 ~ U(0, nx), y0 ~ U(0, ny),
    theta ~ U[0, pi) and, when ``diameter`` is a (lo, hi) pair, d ~ U[lo, hi].
    Returns (fibers, solid mask (nz, ny, nx) bool)."""
    nx, ny, nz = dims
    rng = SplitMix64(seed)
    n = nx * ny * nz
    target_solid = (1.0 - porosity) * n
    solid = np.zeros((nz, ny, nx), dtype=bool)
    nsolid = 0
    fibers = []
    while nsolid < target_solid and len(fibers) < max_fibers:
        z0 = rng.uniform(0.0, nz)
        x0 = rng.uniform(0.0, nx)
        y0 = rng.uniform(0.0, ny)
        th = rng.uniform(0.0, math.pi)
        if isinstance(diameter, (tuple, list)):
            d = rng.uniform(diameter[0], diameter[1])
        else:
            d = float(diameter)
        f = Fiber(z0, x0, y0, th, d)
        fibers.append(f)
        nsolid += _stamp(solid, f, 1.0)
    return fibers, solid


def remove_unconnected(solid: np.ndarray) -> np.ndarray:
    """Make solid every fluid cell not 6-connected to the inlet plane k = 0."""
    from scipy import ndimage

    fluid = ~solid
    lab, _ = ndimage.label(fluid)  # default structure = 6-connectivity in 3D
    keep = np.unique(lab[0])
    keep = keep[keep != 0]
    connected = np.isin(lab, keep)
    if not connected[-1].any():
        raise ValueError("fiber lattice blocks the channel: no fluid path from inlet to outlet")
    return solid | ~connected


# --------------------------------------------------------------------------------------
# Potential flow fixture
# --------------------------------------------------------------------------------------

def potential_flow(solid: np.ndarray, h: float, u_mean: float, tol: float = 1e-12,
                   device: str = "cpu", max_iter: int = 200000, check_every: int = 25,
                   threads: int = 0):
    """Discrete potential flow on the fluid cells of ``solid``.

    Returns (U, V, W, info) as float64 numpy arrays in the face layouts of this module;
    info holds the CG iteration count and the achieved max |div u| / u_mean.
    On a CUDA device the native fixture solver (librfbsynth.so) runs; on the CPU its host
    counterpart (librfbsynth_host.so, OpenMP, ``threads`` <= 0: the default count), the
    same equations and stopping rule, with results independent of the thread count."""
    if str(device).startswith("cuda"):
        return _potential_flow_native(solid, h, u_mean, tol, max_iter, device)
    return _potential_flow_host(solid, h, u_mean, tol, max_iter, max(check_every, 1) * 8,
                                threads)


def _potential_flow_host(solid, h, u_mean, tol, max_iter, check_every, threads):
    import ctypes

    from . import _build

    if not os.path.exists(_build.HOST_SYNTH_LIB):
        _build.build(targets=[_build.HOST_SYNTH_LIB])
    lib = ctypes.CDLL(_build.HOST_SYNTH_LIB)
    f = lib.rfb_synth_potential_flow_cpu
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [ctypes.c_int] * 2 + \
        [ctypes.c_void_p] * 5 + [ctypes.c_int]
    nz, ny, nx = solid.shape
    sol = np.ascontiguousarray(solid, dtype=np.uint8)
    U = np.empty((nz, ny, nx + 1))
    V = np.empty((nz, ny + 1, nx))
    W = np.empty((nz + 1, ny, nx))
    info = np.zeros(4)
    rc = f(nx, ny, nz, h, u_mean, tol, max_iter, check_every, sol.ctypes.data, U.ctypes.data,
           V.ctypes.data, W.ctypes.data, info.ctypes.data, int(threads))
    if rc not in (0, 3):
        raise RuntimeError("host potential-flow solver failed (code %d)" % rc)
    out = {"cg_iters": int(info[0]), "max_div_rel": float(info[1]),
           "true_residual_rel": float(info[2]), "superficial_q": float(info[3])}
    return U, V, W, out


def _potential_flow_native(solid, h, u_mean, tol, max_iter, device):
    import ctypes

    import torch

    from . import _build

    if not os.path.exists(_build.SYNTH_LIB):
        raise RuntimeError("librfbsynth.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(_build.SYNTH_LIB)
    f = lib.rfb_synth_potential_flow
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [ctypes.c_int] * 2 + \
        [ctypes.c_void_p] * 5 + [ctypes.c_void_p]
    nz, ny, nx = solid.shape
    dev = torch.device(device)
    d_solid = torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8)).to(dev)
    U = torch.empty((nz, ny, nx + 1), dtype=torch.float64, device=dev)
    V = torch.empty((nz, ny + 1, nx), dtype=torch.float64, device=dev)
    W = torch.empty((nz + 1, ny, nx), dtype=torch.float64, device=dev)
    info = (ctypes.c_double * 4)()
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = f(nx, ny, nz, h, u_mean, tol, max_iter, 200, d_solid.data_ptr(), U.data_ptr(),
           V.data_ptr(), W.data_ptr(), ctypes.cast(info, ctypes.c_void_p), stream)
    torch.cuda.synchronize(dev)
    if rc not in (0, 3):
        raise RuntimeError("native potential-flow solver failed (code %d)" % rc)
    out = {"cg_iters": int(info[0]), "max_div_rel": float(info[1]),
           "true_residual_rel": float(info[2]), "superficial_q": float(info[3])}
    return U.cpu().numpy(), V.cpu().numpy(), W.cpu().numpy(), out


# --------------------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------------------

H_PAPER = 1.25e-6          # m, the paper's finest resolution (Sec. IV)
D_SOC = 4e-10              # m^2/s, AQDS / H2AQDS diffusivity (parameter table)


@dataclasses.dataclass
class Case:
    name: str
    dims: tuple            # (nx, ny, nz)
    h: float
    solid: np.ndarray      # (nz, ny, nx) uint8, 1 = fiber
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    D: float
    k0: float
    alpha: float
    T: float
    n_e: int
    c0: float
    s_in: float
    eta: float             # overpotential in volts (negative = reducing)
    tol: float
    u_mean: float
    info: dict

    @property
    def n(self) -> int:
        return int(self.dims[0] * self.dims[1] * self.dims[2])

    @property
    def porosity(self) -> float:
        return 1.0 - float(self.solid.mean())


def build_case(name: str, dims, porosity: float, diameter, seed: int, u_mean: float,
               eta: float, s_in: float, tol: float, h: float = H_PAPER,
               flow_device: str = "cpu", k0: float = 1e-7, flow_tol: float = 1e-12) -> Case:
    fibers, solid = generate_fibers(seed, dims, porosity, diameter)
    solid = remove_unconnected(solid)
    U, V, W, info = potential_flow(solid, h, u_mean, tol=flow_tol, device=flow_device)
    info = dict(info)
    info["n_fibers"] = len(fibers)
    if not info["max_div_rel"] < 1e3 * flow_tol:
        raise RuntimeError("potential flow did not converge: %r" % (info,))
    return Case(name=name, dims=tuple(int(d) for d in dims), h=h,
                solid=solid.astype(np.uint8), U=U, V=V, W=W, D=D_SOC, k0=k0, alpha=0.5,
                T=298.0, n_e=2, c0=20.0, s_in=s_in, eta=eta, tol=tol, u_mean=u_mean,
                info=info)


def multilevel_cases(fine_dims, levels: int, porosity: float, diameter, seed: int,
                     u_mean: float, eta: float, s_in: float, tol: float,
                     h_fine: float = H_PAPER, flow_device: str = "cpu", k0: float = 1e-7,
                     name: str = "fiber", only_level=None):
    """The same analytic fibers rasterised at ``levels`` resolutions, coarsest first.

    Fibers are drawn once in finest-level cell units (porosity target at the finest
    level); level l has dims fine_dims / 2^(levels-1-l) and cell size h_fine times the
    same factor. Each level gets its own flood fill and potential flow. ``only_level``
    (an index) builds that level alone and returns a one-element list."""
    fibers, solid_f = generate_fibers(seed, fine_dims, porosity, diameter)
    out = []
    for lev in range(levels):
        if only_level is not None and lev != only_level:
            continue
        f = 2 ** (levels - 1 - lev)
        dims = tuple(int(d) // f for d in fine_dims)
        solid = solid_f if f == 1 else rasterise(fibers, dims, scale=float(f))
        solid = remove_unconnected(solid)
        U, V, W, info = potential_flow(solid, h_fine * f, u_mean, device=flow_device)
        info = dict(info)
        info["n_fibers"] = len(fibers)
        out.append(Case(name="%s%dx%dx%d" % ((name,) + dims), dims=dims, h=h_fine * f,
                        solid=solid.astype(np.uint8), U=U, V=V, W=W, D=D_SOC, k0=k0,
                        alpha=0.5, T=298.0, n_e=2, c0=20.0, s_in=s_in, eta=eta, tol=tol,
                        u_mean=u_mean, info=info))
    return out


def upsampling_cases(flow_device: str = "cpu", only_level=None):
    """The upsampling workload: 128x128x256 (h = 5 um) -> 256x256x512 -> 512x512x1024
    (h = 1.25 um), porosity 0.82 and d = 8 at the finest level, seed 5, 1 cm/s,
    eta = -0.10 V, s_in = 0.5, residual 1e-8 at each level."""
    return multilevel_cases((512, 512, 1024), 3, 0.82, 8.0, 5, 0.01, -0.10, 0.5, 1e-8,
                            flow_device=flow_device, only_level=only_level)


def lognormal_area_mult(solid: np.ndarray, sigma: float = 0.3, seed: int = 40) -> np.ndarray:
    """Per-cell reactive-area multiplier: exp(sigma Z), Z standard normal (numpy PCG64
    with ``seed``), on fluid cells with at least one fiber 6-neighbour (median 1); 1 on
    every other cell. Shape (nz, ny, nx)."""
    s = solid.astype(bool)
    touch = np.zeros_like(s)
    touch[:, :, 1:] |= s[:, :, :-1]
    touch[:, :, :-1] |= s[:, :, 1:]
    touch[:, 1:, :] |= s[:, :-1, :]
    touch[:, :-1, :] |= s[:, 1:, :]
    touch[1:] |= s[:-1]
    touch[:-1] |= s[1:]
    wall = touch & ~s
    z = np.random.default_rng(seed).standard_normal(int(wall.sum()))
    m = np.ones(s.shape)
    m[wall] = np.exp(sigma * z)
    return m


def adjoint_case(dims=(128, 128, 256), seed=4, **kw) -> Case:
    """Differentiation workload: 128x128x256, porosity 0.8, d = 8, 1 cm/s, -0.10 V,
    s_in = 0.5."""
    return build_case("fiber%dx%dx%d_adjoint" % tuple(dims), dims, 0.80, 8.0, seed, 0.01,
                      -0.10, 0.5, 1e-12, **kw)


def batch_instance_params(i: int, n_x_choices=tuple(range(64, 193, 16))):
    """Geometry and operating point of lattice i of the batched workload.

    Lattice 0 is 64^3 and lattice 1 is 192x192x384; others draw (SplitMix64, seed
    3000 + i, in this order) nx = ny uniform over {64, 80, ..., 192},
    nz = 16 round(nx U[1, 2] / 16) clipped to [64, 384], porosity U[0.75, 0.90]; then
    for every lattice the operating point: mean velocity log-uniform in [0.1, 5] cm/s,
    s_in U[0.1, 0.9], eta U[-0.2, -0.02] V. Fibers (d = 8 cells) use their own stream
    (generate_fibers with seed 3000 + i)."""
    rng = SplitMix64(3000 + i)
    if i == 0:
        nx, nz = 64, 64
        por = rng.uniform(0.75, 0.90)
    elif i == 1:
        nx, nz = 192, 384
        por = rng.uniform(0.75, 0.90)
    else:
        nx = n_x_choices[min(int(rng.uniform() * len(n_x_choices)), len(n_x_choices) - 1)]
        nz = int(16 * round(nx * rng.uniform(1.0, 2.0) / 16))
        nz = max(64, min(384, nz))
        por = rng.uniform(0.75, 0.90)
    u = 10 ** rng.uniform(math.log10(0.001), math.log10(0.05))
    s_in = rng.uniform(0.1, 0.9)
    eta = rng.uniform(-0.2, -0.02)
    return dict(dims=(nx, nx, nz), porosity=por, u_mean=u, s_in=s_in, eta=eta, seed=3000 + i)


def batch_cases(n: int = 48, flow_device: str = "cpu", tol: float = 1e-8, scale: int = 1):
    """The batched workload (``scale`` > 1 divides every dimension, for tests)."""
    out = []
    for i in range(n):
        q = batch_instance_params(i)
        dims = tuple(max(16, d // scale) for d in q["dims"])
        out.append(build_case("batch%02d_%dx%dx%d" % ((i,) + dims), dims, q["porosity"],
                              8.0 / scale if scale > 1 else 8.0, q["seed"], q["u_mean"],
                              q["eta"], q["s_in"], tol, flow_device=flow_device))
    return out


def fiber_channel_case(dims=(48, 48, 96), porosity=0.80, diameter=8.0, seed=1,
                       u_mean=0.01, eta=-0.10, s_in=0.5, tol=1e-10, **kw) -> Case:
    """Plain FP64 workload: 48x48x96, d = 8 cells, porosity 0.80, 1 cm/s, eta = -0.10 V,
    s_in = 0.5 (defaults); smaller dims give the same recipe at test size."""
    return build_case("fiber48x48x96" if tuple(dims) == (48, 48, 96) else
                      "fiber%dx%dx%d" % tuple(dims), dims, porosity, diameter, seed,
                      u_mean, eta, s_in, tol, **kw)


def large_mixed_case(dims=(256, 256, 512), seed=2, **kw) -> Case:
    """Mixed-precision workload: 256x256x512, porosity 0.85, d ~ U[6, 10] cells,
    0.5 cm/s, eta = -0.05 V, s_in = 0.3, residual 1e-8."""
    return build_case("fiber%dx%dx%d_mixed" % tuple(dims), dims, 0.85, (6.0, 10.0), seed,
                      0.005, -0.05, 0.3, 1e-8, **kw)


# --------------------------------------------------------------------------------------
# Logpile lattice (the paper's benchmark electrode, Sec. IV)
# --------------------------------------------------------------------------------------
#
# A box of 1280 x 640 x 160 um (the paper's flow length x width x height) holding 43 rods
# of diameter 20 um in seven layers whose axes lie at heights 20, 40, ..., 140 um. Layers
# 1, 3, 5 and 7 run along the flow, four rods each at widths 128, 256, 384 and 512 um;
# layers 2, 4 and 6 run across it, nine rods each at flow positions 128, 256, ..., 1152
# um. Adjacent layers are one diameter apart, so crossing rods touch. In this module's
# axes the flow runs along z (the paper's x), y is the paper's y and x the paper's z
# (the stacking height).

LOGPILE_BOX_UM = (1280.0, 640.0, 160.0)   # flow length, width, height
LOGPILE_ROD_D_UM = 20.0
LOGPILE_PITCH_UM = 128.0
LOGPILE_LAYER_UM = 20.0
LOGPILE_Q_10PA = 0.345e-6 / 3600.0        # m^3/s: 3.45 mL/h at 100 Pa, scaled to 10 Pa


def logpile_rods():
    """The 43 rods: (layer, along, c1_um, c2_um). along = 'z' (with the flow; axis at
    height c1 and width c2) or 'y' (across it; axis at height c1 and flow position c2)."""
    rods = []
    for layer in range(1, 8):
        height = LOGPILE_LAYER_UM * layer
        if layer % 2 == 1:
            for m in range(1, 5):
                rods.append((layer, "z", height, LOGPILE_PITCH_UM * m))
        else:
            for m in range(1, 10):
                rods.append((layer, "y", height, LOGPILE_PITCH_UM * m))
    return rods


def logpile_dims(h: float):
    """(nx, ny, nz) of the logpile box at cell size h (which must divide it)."""
    um = h * 1e6
    n = [L / um for L in (LOGPILE_BOX_UM[2], LOGPILE_BOX_UM[1], LOGPILE_BOX_UM[0])]
    dims = tuple(int(round(v)) for v in n)
    if any(abs(v - d) > 1e-9 * d for v, d in zip(n, dims)):
        raise ValueError("h = %g m does not divide the 1280 x 640 x 160 um box" % h)
    return dims


def logpile_solid(h: float) -> np.ndarray:
    """Solid mask (nz, ny, nx) of the logpile at cell size h: a cell is solid when its
    centre lies within a rod's radius of the rod's axis (distances in cell units)."""
    nx, ny, nz = logpile_dims(h)
    um = h * 1e6
    r = 0.5 * LOGPILE_ROD_D_UM / um
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    z = np.arange(nz) + 0.5
    solid = np.zeros((nz, ny, nx), dtype=bool)
    for _, along, c1, c2 in logpile_rods():
        a, b = c1 / um, c2 / um
        if along == "z":
            disk = (x[None, :] - a) ** 2 + (y[:, None] - b) ** 2 <= r * r     # (ny, nx)
            solid |= disk[None, :, :]
        else:
            disk = (x[None, :] - a) ** 2 + (z[:, None] - b) ** 2 <= r * r     # (nz, nx)
            solid |= disk[:, None, :]
    return solid


def logpile_porosity_exact() -> float:
    """Fluid fraction of the continuous logpile: the rods are tangent where they cross,
    so their volumes add: 1 - pi r^2 (16 x 1280 + 27 x 640) / (1280 x 640 x 160)."""
    r = 0.5 * LOGPILE_ROD_D_UM
    L, W, H = LOGPILE_BOX_UM
    n_along = sum(1 for rod in logpile_rods() if rod[1] == "z")
    n_across = len(logpile_rods()) - n_along
    return 1.0 - math.pi * r * r * (n_along * L + n_across * W) / (L * W * H)


def logpile_case(h: float = H_PAPER, q: float = LOGPILE_Q_10PA, eta: float = 0.0,
                 s_in: float = 1.73e-7, k0: float = 7.2e-5, tol: float = 1e-6,
                 flow_device: str = "cpu", flow_tol: float = 1e-12, flow: str = "potential",
                 dp: float = 10.0) -> Case:
    """The paper's reference reaction case on the logpile (Sec. IV): 10 Pa, applied
    reducing voltage 0 (eta = 0, s_eq = 1/2), the parameter table's k0 and inlet state
    of charge, tolerance 1e-6 on the residual.
    flow = 'potential': the potential flow of this module, rescaled so that the volumetric
    flow rate through the inlet is q (default: the paper's 3.45 mL/h at 100 Pa scaled
    linearly to 10 Pa). flow = 'stokes': the Stokes flow at the pressure drop dp (Pa)
    from ``stokes_flow_minres`` on ``flow_device``."""
    solid = remove_unconnected(logpile_solid(h))
    if flow == "stokes":
        # tol 1e-11: the multigrid-preconditioned norm weights the velocity residual by
        # about A^-1, so it starts larger than the diagonal-preconditioned one; at 1e-11 the
        # divergence stays below 1e-9 of the mean inlet-face flux
        U, V, W, info = stokes_flow_minres(solid, h, dp=dp, tol=1e-11, device=flow_device)
        q = info["q_m3_s"]
        f = 1.0
    elif flow == "potential":
        # solved at a mean z-velocity of 1 m/s over fluid z-faces, scaled to the rate q
        U, V, W, info = potential_flow(solid, h, 1.0, tol=flow_tol, device=flow_device)
        fin = ~solid[0]
        f = q / (h * h * float(np.sum(np.where(fin, W[0], 0.0))))
        U, V, W = U * f, V * f, W * f
    else:
        raise ValueError("flow must be 'potential' or 'stokes'")
    info = dict(info)
    info["flow"] = flow
    info["q_m3_s"] = q
    info["n_rods"] = len(logpile_rods())
    fz = np.zeros(W.shape, dtype=bool)
    fz[1:-1] = (solid[:-1] == 0) & (solid[1:] == 0)
    u_mean = float(W[fz].mean())                # mean z-velocity over fluid z-faces (m/s)
    dims = logpile_dims(h)
    return Case(name="logpile%dx%dx%d" % dims, dims=dims, h=h, solid=solid.astype(np.uint8),
                U=U, V=V, W=W, D=D_SOC, k0=k0, alpha=0.5, T=298.0, n_e=2, c0=20.0,
                s_in=s_in, eta=eta, tol=tol, u_mean=u_mean, info=info)


# --------------------------------------------------------------------------------------
# Stokes flow fixture (CPU, sparse LU; small lattices)
# --------------------------------------------------------------------------------------

MU_WATER = 8.8891e-4   # Pa s (parameter table)


def _face_laplacian(open_, along, h, mu):
    """A = -mu Lap on the open faces of one velocity component (face array ``open_``,
    component along array axis ``along``: 0 = z, 1 = y, 2 = x). Neighbour faces:
    open -> coupled; closed along the component's own axis -> a wall face with velocity 0
    one cell away; closed across it -> a wall half a cell away (ghost value -u);
    outside the lattice across z (inlet / outlet planes) -> zero normal gradient;
    outside across x or y (side walls) -> wall half a cell away."""
    import scipy.sparse as sp
    shape = open_.shape
    idx = -np.ones(shape, dtype=np.int64)
    idx[open_] = np.arange(int(open_.sum()))
    n = int(open_.sum())
    c = mu / (h * h)
    diag = np.zeros(n)
    rows, cols = [], []
    for axis in range(3):
        for step in (-1, 1):
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if step == 1:
                src[axis], dst[axis] = slice(0, shape[axis] - 1), slice(1, None)
            else:
                src[axis], dst[axis] = slice(1, None), slice(0, shape[axis] - 1)
            a = idx[tuple(src)]
            b = idx[tuple(dst)]
            have = a >= 0
            coupled = have & (b >= 0)
            rows.append(a[coupled]); cols.append(b[coupled])
            np.add.at(diag, a[coupled], c)
            closed = have & (b < 0)
            np.add.at(diag, a[closed], c if axis == along else 2 * c)
            # faces on the lattice's last layer along this direction have no neighbour
            edge = [slice(None)] * 3
            edge[axis] = shape[axis] - 1 if step == 1 else 0
            e = idx[tuple(edge)]
            e = e[e >= 0]
            if axis != 0:                       # side walls half a cell away
                np.add.at(diag, e, c if axis == along else 2 * c)
            # axis 0 (inlet / outlet): zero normal gradient, nothing added
    r = np.concatenate(rows)
    q = np.concatenate(cols)
    A = sp.csr_matrix((np.full(r.size, -c), (r, q)), shape=(n, n)) + sp.diags(diag)
    return A.tocsc(), idx


def stokes_flow(solid: np.ndarray, h: float, dp: float = 1.0, mu: float = MU_WATER,
                tol: float = 1e-13, max_iter: int = 5000):
    """Steady Stokes flow through the fluid cells of ``solid`` driven by the pressure drop
    ``dp`` (Pa) from the inlet to the outlet; at the paper's Reynolds numbers its
    incompressible Navier-Stokes solve (Sec. III.A, Algorithm 1) reaches this flow, which
    is linear in the pressure (Sec. IV scales flows between pressures). Staggered grid in
    this module's face layout: -mu Lap u + grad p = 0 on every open face and div u = 0 in
    every fluid cell; no slip on fiber faces and side walls (staircase walls), zero normal
    gradient of velocity at the inlet and outlet planes, and pressures dp and 0 on ghost
    cell centres one cell before the inlet and past the outlet.
    Solved by conjugate gradients on the pressure Schur complement S = D A^-1 D^T (SPD:
    the boundary pressures fix the constant), with sparse LU factors of the three velocity
    Laplacians A. Returns (U, V, W, info) in m/s."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    solid = solid.astype(bool)
    fluid = ~solid
    nz, ny, nx = solid.shape
    oU = np.zeros((nz, ny, nx + 1), dtype=bool)
    oU[:, :, 1:nx] = fluid[:, :, :-1] & fluid[:, :, 1:]
    oV = np.zeros((nz, ny + 1, nx), dtype=bool)
    oV[:, 1:ny, :] = fluid[:, :-1, :] & fluid[:, 1:, :]
    oW = np.zeros((nz + 1, ny, nx), dtype=bool)
    oW[1:nz] = fluid[:-1] & fluid[1:]
    oW[0] = fluid[0]
    oW[nz] = fluid[-1]
    cidx = -np.ones((nz, ny, nx), dtype=np.int64)
    nf = int(fluid.sum())
    cidx[fluid] = np.arange(nf)

    blocks, divs, rhs = [], [], []
    for open_, along in ((oU, 2), (oV, 1), (oW, 0)):
        A, fidx = _face_laplacian(open_, along, h, mu)
        n = A.shape[0]
        # divergence: a face is the high face of the cell below it along its axis (+1/h)
        # and the low face of the cell above it (-1/h)
        f_of = fidx[open_]
        pos = np.argwhere(open_)
        lo = pos.copy()
        lo[:, along] -= 1
        rows, cols, vals = [], [], []
        for cellpos, sign in ((lo, 1.0), (pos, -1.0)):
            ok = (cellpos[:, along] >= 0) & (cellpos[:, along] < (nz, ny, nx)[along])
            cp = cellpos[ok]
            rows.append(cidx[cp[:, 0], cp[:, 1], cp[:, 2]]); cols.append(f_of[ok])
            vals.append(np.full(int(ok.sum()), sign / h))
        D = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(nf, n))
        b = np.zeros(n)
        if along == 0:
            b[fidx[0][oW[0]]] = dp / h            # (p_0 - dp) / h on the inlet faces
        blocks.append(spla.splu(A))
        divs.append(D)
        rhs.append(b)

    def a_inv(vs):
        return [lu.solve(v) for lu, v in zip(blocks, vs)]

    def s_mul(p):
        u = a_inv([D.T @ p for D in divs])
        return sum(D @ x for D, x in zip(divs, u))

    S = spla.LinearOperator((nf, nf), matvec=s_mul, dtype=np.float64)
    g = -sum(D @ x for D, x in zip(divs, a_inv(rhs)))
    iters = [0]

    def count(_):
        iters[0] += 1

    p, info_cg = spla.cg(S, g, rtol=tol, atol=0.0, maxiter=max_iter, callback=count)
    if info_cg != 0:
        raise RuntimeError("Stokes pressure CG did not converge (info=%d)" % info_cg)
    u = a_inv([b + D.T @ p for b, D in zip(rhs, divs)])
    out = []
    for open_, x in zip((oU, oV, oW), u):
        f = np.zeros(open_.shape)
        f[open_] = x
        out.append(f)
    U, V, W = out
    div = sum(D @ x for D, x in zip(divs, u))
    q = h * h * float(W[0][oW[0]].sum())
    # a cell's net outflow (div u h^3) relative to the mean flux of an inlet face
    mean_face_q = q / max(int(oW[0].sum()), 1)
    info = {"cg_iters": iters[0], "q_m3_s": q,
            "max_div_rel": float(np.abs(div).max() * h ** 3 / max(abs(mean_face_q), 1e-300))}
    return U, V, W, info


def _open_faces(fluid):
    """Open-face masks (U, V, W) of a fluid mask (nz, ny, nx): faces between two fluid
    cells, plus the inlet and outlet faces of fluid cells."""
    nz, ny, nx = fluid.shape
    oU = np.zeros((nz, ny, nx + 1), dtype=bool)
    oU[:, :, 1:nx] = fluid[:, :, :-1] & fluid[:, :, 1:]
    oV = np.zeros((nz, ny + 1, nx), dtype=bool)
    oV[:, 1:ny, :] = fluid[:, :-1, :] & fluid[:, 1:, :]
    oW = np.zeros((nz + 1, ny, nx), dtype=bool)
    oW[1:nz] = fluid[:-1] & fluid[1:]
    oW[0] = fluid[0]
    oW[nz] = fluid[-1]
    return oU, oV, oW


def _shift(x, axis, step):
    """y[i] = x[i + step] along ``axis`` (zero where i + step leaves the array)."""
    import torch
    y = torch.zeros_like(x)
    n = x.shape[axis]
    if step == 1:
        y.narrow(axis, 0, n - 1).copy_(x.narrow(axis, 1, n - 1))
    else:
        y.narrow(axis, 1, n - 1).copy_(x.narrow(axis, 0, n - 1))
    return y


def _block_sum(x):
    """Sums over the 2 x 2 x 2 blocks of a (nz, ny, nx) array (odd extents padded with
    zeros): the block lattice of one multigrid coarsening."""
    import torch
    nz, ny, nx = x.shape
    x = torch.nn.functional.pad(x, (0, nx % 2, 0, ny % 2, 0, nz % 2))
    z, y, w = x.shape
    return x.reshape(z // 2, 2, y // 2, 2, w // 2, 2).sum(dim=(1, 3, 5))


def _parity(x, axis, r):
    """x where the index along ``axis`` is r modulo 2, zero elsewhere."""
    import torch
    y = torch.zeros_like(x)
    sl = [slice(None)] * 3
    sl[axis] = slice(r, None, 2)
    y[tuple(sl)] = x[tuple(sl)]
    return y


def _stencil_apply(d, c, x):
    """y = A x for a symmetric 7-point stencil stored as its diagonal d and the couplings
    c[a] of every entry to its high neighbour along axis a."""
    y = d * x
    for a in range(3):
        n = x.shape[a]
        if n == 1:
            continue
        ca = c[a].narrow(a, 0, n - 1)
        y.narrow(a, 0, n - 1).addcmul_(ca, x.narrow(a, 1, n - 1))
        y.narrow(a, 1, n - 1).addcmul_(ca, x.narrow(a, 0, n - 1))
    return y


class _FaceMultigrid:
    """Multigrid V-cycle for the unit-stencil negative Laplacian A of one velocity
    component of ``stokes_flow_minres`` (the open faces ``open_``, diagonal ``diag`` with
    the wall terms), used as that component's preconditioner.

    Coarsening by aggregation: the faces of each 2 x 2 x 2 block are one coarse unknown,
    prolongation P copies a coarse value onto the block's open faces and restriction is
    P^T. The Galerkin product P^T A P of a 7-point stencil is again a 7-point stencil on the
    block lattice (a coupling inside a block adds twice to the block's diagonal, one across
    two blocks becomes theirs), so every level is a diagonal and three coupling arrays and
    the geometry never has to be rasterised again. With piecewise-constant P the Galerkin
    operator rates a smooth error about twice as stiff as it is, because the staircase
    P e_c puts the whole jump between two blocks across a single face; the coarse operator
    is therefore divided by ``beta`` (the over-correction of unsmoothed aggregation:
    Braess 1995; Vanek, Mandel and Brezina 1996).
    Smoother: damped Jacobi with weight ``omega`` < 1, ``nu`` steps before and as many after
    the coarse correction. The stencils are weakly diagonally dominant M-matrices on every
    level, so 2 D / omega - A is positive definite and the cycle is a symmetric positive
    definite operator whatever the (SPD) coarse solve: what MINRES needs of a
    preconditioner. The coarsest level (at most ``coarse_max`` unknowns) is solved exactly
    with the inverse of its dense matrix."""

    def __init__(self, open_, diag, beta=2.0, omega=0.8, nu=2, coarse_max=2000):
        import torch
        self.omega, self.nu = omega, nu
        f64 = torch.float64
        o = open_
        d = diag * o
        c = [-(o & _shift(o, a, 1)).to(f64) for a in range(3)]
        self.levels = []
        while True:
            dinv = torch.where(o, 1.0 / torch.where(o, d, torch.ones_like(d)), torch.zeros_like(d))
            self.levels.append((o, d, c, dinv))
            if int(o.sum()) <= coarse_max or max(o.shape) == 1:
                break
            d, c = ((_block_sum(d) + 2.0 * sum(_block_sum(_parity(c[a], a, 0)) for a in range(3)))
                    / beta, [_block_sum(_parity(c[a], a, 1)) / beta for a in range(3)])
            o = _block_sum(o.to(f64)) > 0
            d = d * o
        # dense inverse of the coarsest level
        o, d, c, _ = self.levels[-1]
        idx = -torch.ones(o.shape, dtype=torch.int64, device=o.device)
        n = int(o.sum())
        idx[o] = torch.arange(n, device=o.device)
        m = torch.diag(d[o])
        for a in range(3):
            hi = _shift(idx, a, 1)
            both = o & (hi >= 0) & (c[a] != 0)
            i, j, v = idx[both], hi[both], c[a][both]
            m[i, j] = v
            m[j, i] = v
        self.coarse_inv = torch.cholesky_inverse(torch.linalg.cholesky(m))

    def vcycle(self, b, lvl=0):
        """One V-cycle from the zero guess for A x = b on level ``lvl`` (b zero off the
        level's open entries); returns x, zero off them."""
        o, d, c, dinv = self.levels[lvl]
        if lvl == len(self.levels) - 1:
            x = b.new_zeros(b.shape)
            x[o] = self.coarse_inv @ b[o]
            return x
        w = self.omega * dinv
        x = w * b
        for _ in range(self.nu - 1):
            x = x + w * (b - _stencil_apply(d, c, x))
        xc = self.vcycle(_block_sum(b - _stencil_apply(d, c, x)), lvl + 1)
        z, y, v = xc.shape
        x = x + xc[:, None, :, None, :, None].expand(z, 2, y, 2, v, 2).reshape(
            2 * z, 2 * y, 2 * v)[:o.shape[0], :o.shape[1], :o.shape[2]] * o
        for _ in range(self.nu):
            x = x + w * (b - _stencil_apply(d, c, x))
        return x


def stokes_flow_minres(solid: np.ndarray, h: float, dp: float = 1.0, mu: float = MU_WATER,
                       tol: float = 1e-10, max_iter: int = 200000, device: str = "cpu",
                       precond: str = "mg"):
    """The Stokes flow of ``stokes_flow`` (same staggered discretisation and boundary
    conditions), matrix-free in PyTorch on any device: preconditioned MINRES (Paige and
    Saunders, SIAM J. Numer. Anal. 12, 1975) on the symmetric saddle-point system
        [A  -D^T] [u]   [b]
        [-D   0 ] [p] = [0],
    in the scaled velocity u^ = (mu / h) u, where A is the unit-stencil negative Laplacian
    on the open faces, D the unit-stencil divergence and b = dp on the inlet faces: both
    unknowns are then of the size of dp. The preconditioner is block diagonal: the
    identity on the pressures (the Schur complement D A^-1 D^T of the scaled system is
    close to I) and, on each velocity component, either one symmetric multigrid V-cycle
    for A (precond='mg', ``_FaceMultigrid``: its iteration count barely grows as h
    shrinks) or the diagonal of A (precond='jacobi': iterations grow like 1/h). Stops
    when the preconditioned residual norm falls below tol times its initial value.
    Returns (U, V, W, info) in m/s."""
    import torch
    dev = torch.device(device)
    f64 = torch.float64
    solid = solid.astype(bool)
    fluid_np = ~solid
    nz, ny, nx = solid.shape
    opens = [torch.from_numpy(o).to(dev) for o in _open_faces(fluid_np)]
    fluid = torch.from_numpy(fluid_np).to(dev)
    c = 1.0
    along_of = (2, 1, 0)                      # U along x (axis 2), V along y, W along z
    diags = []
    for o, along in zip(opens, along_of):
        d = torch.zeros(o.shape, dtype=f64, device=dev)
        ones = torch.ones(o.shape, dtype=torch.bool, device=dev)
        for axis in range(3):
            for step in (-1, 1):
                nb = _shift(o, axis, step)
                inside = _shift(ones, axis, step)
                wall = c if axis == along else 2 * c
                d += c * nb + wall * (inside & ~nb)
                if axis != 0:                 # side walls half a cell away
                    d += wall * ~inside
        diags.append(d * o)
    sizes = [o.numel() for o in opens] + [fluid.numel()]
    shapes = [o.shape for o in opens] + [fluid.shape]
    offs = np.cumsum([0] + sizes)

    def views(x):
        return [x[offs[i]:offs[i + 1]].view(shapes[i]) for i in range(4)]

    def apply(x):
        U, V, W, P = views(x)
        y = torch.empty_like(x)
        yU, yV, yW, yP = views(y)
        for u, yu, o, d in ((U, yU, opens[0], diags[0]), (V, yV, opens[1], diags[1]),
                            (W, yW, opens[2], diags[2])):
            torch.mul(d, u, out=yu)
            for axis in range(3):
                n = u.shape[axis]
                if n > 1:
                    yu.narrow(axis, 0, n - 1).sub_(u.narrow(axis, 1, n - 1), alpha=c)
                    yu.narrow(axis, 1, n - 1).sub_(u.narrow(axis, 0, n - 1), alpha=c)
            yu.mul_(o)
        # -D^T p on the faces: p_high - p_low, with p = 0 outside the lattice
        Pz = torch.nn.functional.pad(P, (0, 0, 0, 0, 1, 1))
        yU[:, :, 1:nx] += (P[:, :, 1:] - P[:, :, :-1]) * opens[0][:, :, 1:nx]
        yV[:, 1:ny, :] += (P[:, 1:, :] - P[:, :-1, :]) * opens[1][:, 1:ny, :]
        yW += (Pz[1:] - Pz[:-1]) * opens[2]
        # -D u in the fluid cells
        div = U[:, :, 1:] - U[:, :, :-1] + V[:, 1:, :] - V[:, :-1, :] + W[1:] - W[:-1]
        yP.copy_(-div * fluid)
        return y

    if precond == "jacobi":
        minv = torch.cat([torch.where(o, 1.0 / torch.where(o, d, torch.ones_like(d)),
                                      torch.zeros_like(d)).reshape(-1)
                          for o, d in zip(opens, diags)] + [fluid.to(f64).reshape(-1)])

        def prec(r):
            return minv * r
    elif precond == "mg":
        mgs = [_FaceMultigrid(o, d) for o, d in zip(opens, diags)]
        fluid64 = fluid.to(f64)

        def prec(r):
            z = torch.empty_like(r)
            rv, zv = views(r), views(z)
            for i in range(3):
                zv[i].copy_(mgs[i].vcycle(rv[i]))
            zv[3].copy_(rv[3] * fluid64)
            return z
    else:
        raise ValueError("precond must be 'mg' or 'jacobi'")
    b = torch.zeros(int(offs[-1]), dtype=f64, device=dev)
    views(b)[2][0] = dp * opens[2][0]

    # preconditioned MINRES
    x = torch.zeros_like(b)
    r1 = b.clone()
    y = prec(r1)
    beta1 = float(torch.dot(r1, y)) ** 0.5
    beta, oldb, dbar, epsln, phibar, cs, sn = beta1, 0.0, 0.0, 0.0, beta1, -1.0, 0.0
    w = torch.zeros_like(b)
    w2 = torch.zeros_like(b)
    r2 = r1.clone()
    it = 0
    while it < max_iter and phibar > tol * beta1:
        it += 1
        v = y / beta
        y = apply(v)
        if it >= 2:
            y -= (beta / oldb) * r1
        alfa = float(torch.dot(v, y))
        y -= (alfa / beta) * r2
        r1, r2 = r2, y
        y = prec(r2)
        oldb, beta = beta, float(torch.dot(r2, y)) ** 0.5
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = max((gbar * gbar + beta * beta) ** 0.5, 1e-300)
        cs, sn = gbar / gamma, beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1, w2 = w2, w
        w = (v - oldeps * w1 - delta * w2) / gamma
        x += phi * w
    if phibar > tol * beta1:
        raise RuntimeError("Stokes MINRES did not converge in %d iterations" % it)
    oU, oV, oW = _open_faces(fluid_np)
    U, V, W = ((t.cpu().numpy() * (h / mu)) * o for t, o in zip(views(x)[:3], (oU, oV, oW)))
    q = h * h * float(W[0].sum())
    div = (U[:, :, 1:] - U[:, :, :-1] + V[:, 1:, :] - V[:, :-1, :] + W[1:] - W[:-1]) / h
    mean_face_q = q / max(int(fluid_np[0].sum()), 1)
    info = {"minres_iters": it, "precond": precond, "q_m3_s": q,
            "max_div_rel": float(np.abs(div[fluid_np]).max() * h ** 3 / max(abs(mean_face_q), 1e-300))}
    return U, V, W, info
