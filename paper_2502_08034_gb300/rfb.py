"""Python binding of the C ABI in include/rfb_soc.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library ``librfbsoc.so`` built in-tree by
``_build.build()``; if the library is missing this module raises instead of falling
back to anything else. Inputs may be numpy arrays (host memory) or CUDA torch tensors
(device memory, used in place for the copy into library-owned buffers).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p
from typing import Optional

import numpy as np

from . import _build

RFB_OK, RFB_ERR_INVALID_ARG, RFB_ERR_CUDA, RFB_ERR_OOM = 0, 1, 2, 3
RFB_ERR_NOT_CONVERGED, RFB_ERR_NONFINITE, RFB_ERR_STATE, RFB_ERR_UNSUPPORTED = 4, 5, 6, 7
MEM_HOST, MEM_DEVICE = 0, 1
PREC = {"fp64": 0, "mixed": 1}
KIN_AFFINE, KIN_UNIFORM_ETA = 0, 1
INLET = {"face": 0, "ghost": 1}
DT = {"global": 0, "local": 1}
OBJECTIVES = {"I_tot": 0, "U": 1, "U_mt": 2}


class Kinetics(ctypes.Structure):
    _fields_ = [("k0", c_double), ("alpha", c_double), ("n_e", c_int32), ("mode", c_int32),
                ("T", c_double), ("c0", c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("inlet_bc", c_int32), ("dt_mode", c_int32),
                ("check_every", c_int32), ("cfl", c_double), ("velocity_scale", c_double),
                ("max_sweeps", c_int64), ("fp32_kernel", c_int32), ("timeout_ms", c_int32),
                ("reserved", c_int32 * 6)]


class SolveResult(ctypes.Structure):
    _fields_ = [("sweeps", c_int64), ("checks", c_int64), ("residual", c_double),
                ("I_tot", c_double), ("F_in", c_double), ("F_out", c_double),
                ("F_in_adv", c_double), ("mass_balance_rel", c_double), ("U", c_double),
                ("outlet_mean", c_double), ("dt", c_double), ("tau", c_double),
                ("time_ms", c_double), ("nonfinite", c_int64), ("sweep_ms", c_double),
                ("check_ms", c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class BVParams(ctypes.Structure):
    _fields_ = [("D_H", c_double), ("D_X", c_double), ("c_H_in", c_double),
                ("cg_rtol", c_double), ("cycle", c_int32), ("max_cg", c_int32),
                ("start", c_int32), ("reserved", c_int32)]


class BVResult(ctypes.Structure):
    _fields_ = [("sweeps", c_int64), ("cycles", c_int64), ("cg_iterations", c_int64),
                ("residual", c_double), ("dphi", c_double), ("I_tot", c_double),
                ("U", c_double), ("s_out", c_double), ("I_membrane", c_double),
                ("phi_mean", c_double), ("phi_min", c_double), ("phi_max", c_double),
                ("time_ms", c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


BV_START = {"auto": 0, "sbv": 1, "cold": 2}

_LIB = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("librfbsoc.so is not built (run __graft_entry__.build()); "
                               "there is no fallback implementation")
        L = ctypes.CDLL(path)
        H = c_void_p
        L.rfb_solve_opts_default.argtypes = [POINTER(SolveOpts)]
        L.rfb_solve_opts_default.restype = None
        L.rfb_status_string.argtypes = [c_int]
        L.rfb_status_string.restype = c_char_p
        L.rfb_soc_last_error.argtypes = [H]
        L.rfb_soc_last_error.restype = c_char_p
        L.rfb_soc_create.argtypes = [POINTER(c_int32), c_double, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_double, POINTER(Kinetics), c_void_p, c_int,
                                     c_void_p, POINTER(H)]
        L.rfb_soc_destroy.argtypes = [H]
        L.rfb_soc_set_stream.argtypes = [H, c_void_p]
        L.rfb_soc_solve.argtypes = [H, c_double, c_double, c_double, POINTER(SolveOpts),
                                    POINTER(SolveResult)]
        L.rfb_soc_step.argtypes = [H, c_double, c_double, c_int64, POINTER(SolveOpts),
                                   POINTER(SolveResult)]
        L.rfb_soc_current.argtypes = [H, POINTER(SolveResult)]
        L.rfb_soc_current_noalloc.argtypes = [H, POINTER(SolveResult)]
        L.rfb_soc_umt.argtypes = [H, c_double, POINTER(SolveOpts), POINTER(c_double),
                                  POINTER(SolveResult)]
        L.rfb_soc_get_state.argtypes = [H, c_void_p, c_int]
        L.rfb_soc_set_state.argtypes = [H, c_void_p, c_int]
        L.rfb_soc_reset_state.argtypes = [H]
        L.rfb_soc_upsample.argtypes = [H, H]
        L.rfb_soc_set_area_mult.argtypes = [H, c_void_p, c_int]
        L.rfb_soc_batch_create.argtypes = [POINTER(c_void_p), c_int, POINTER(H)]
        L.rfb_soc_batch_solve.argtypes = [H, POINTER(c_double), POINTER(c_double),
                                          POINTER(c_double), POINTER(SolveOpts),
                                          POINTER(SolveResult), POINTER(BatchInfo)]
        L.rfb_soc_batch_destroy.argtypes = [H]
        L.rfb_soc_batch_set_stream.argtypes = [H, c_void_p]
        L.rfb_soc_batch_set_stream.restype = c_int
        L.rfb_soc_batch_last_error.argtypes = [H]
        L.rfb_soc_batch_last_error.restype = c_char_p
        L.rfb_soc_adjoint.argtypes = [H, c_int, c_double, POINTER(SolveOpts), c_void_p,
                                      POINTER(c_double), c_int, POINTER(SolveResult)]
        L.rfb_soc_info.argtypes = [H, POINTER(c_int64), POINTER(c_int64)]
        L.rfb_soc_kernel_launches.argtypes = [H]
        L.rfb_soc_kernel_launches.restype = c_int64
        L.rfb_soc_tuned_fp32_kernel.argtypes = [H, POINTER(c_int32), POINTER(c_double),
                                                POINTER(c_double)]
        L.rfb_selftest_bounded_wait.argtypes = [c_int64, POINTER(c_int32)]
        L.rfb_soc_solve_nernst.argtypes = [H, c_double, c_double, c_double, c_double,
                                           POINTER(SolveOpts), POINTER(SolveResult)]
        L.rfb_soc_get_overpotential.argtypes = [H, c_void_p, c_int]
        L.rfb_soc_solve_bv.argtypes = [H, c_double, c_double, c_double, POINTER(BVParams),
                                       POINTER(SolveOpts), POINTER(BVResult)]
        L.rfb_soc_get_bv_state.argtypes = [H, c_void_p, c_void_p, c_void_p, c_void_p, c_int]
        for name in ("rfb_soc_create", "rfb_soc_destroy", "rfb_soc_set_stream", "rfb_soc_solve",
                     "rfb_soc_step", "rfb_soc_current", "rfb_soc_umt", "rfb_soc_get_state",
                     "rfb_soc_set_state", "rfb_soc_info", "rfb_soc_reset_state",
                     "rfb_soc_current_noalloc", "rfb_soc_upsample", "rfb_soc_set_area_mult",
                     "rfb_soc_adjoint", "rfb_soc_batch_create", "rfb_soc_batch_solve",
                     "rfb_soc_batch_destroy", "rfb_soc_tuned_fp32_kernel",
                     "rfb_selftest_bounded_wait", "rfb_soc_solve_nernst",
                     "rfb_soc_get_overpotential", "rfb_soc_solve_bv", "rfb_soc_get_bv_state"):
            getattr(L, name).restype = c_int
        _LIB = L
    return _LIB


class RfbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (lib().rfb_status_string(status).decode(), msg))
        self.status = status


FP32_KERNEL = {"auto": 0, "plain": 1, "blocked": 2, "blocked_persistent": 3,
               "blocked_chunked": 4, "blocked4_persistent": 5, "blocked4_chunked": 6,
               "three_sweep_persistent": 7, "three_sweep_chunked": 8,
               "three_sweep5_persistent": 9, "three_sweep5_chunked": 10}


def make_opts(precision="fp64", inlet_bc="face", dt_mode="local", check_every=0, cfl=0.4,
              velocity_scale=1.0, max_sweeps=0, fp32_kernel="auto", timeout_ms=0) -> SolveOpts:
    o = SolveOpts()
    lib().rfb_solve_opts_default(byref(o))
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.inlet_bc = INLET[inlet_bc] if isinstance(inlet_bc, str) else int(inlet_bc)
    o.dt_mode = DT[dt_mode] if isinstance(dt_mode, str) else int(dt_mode)
    o.check_every = int(check_every)
    o.cfl = float(cfl)
    o.velocity_scale = float(velocity_scale)
    o.max_sweeps = int(max_sweeps)
    o.fp32_kernel = FP32_KERNEL[fp32_kernel] if isinstance(fp32_kernel, str) else int(fp32_kernel)
    o.timeout_ms = int(timeout_ms)
    return o


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _count(size, n, what):
    if n is not None and size != n:
        raise ValueError("%s holds %d values; the lattice needs %d" % (what, size, n))


def _ptr(x, dtype, n=None, what="array"):
    """(pointer, keepalive, kind) of a numpy array or CUDA torch tensor. With ``n`` the
    array must hold exactly n values (any shape): the C ABI reads that many from the
    pointer, so a smaller array would be read past its end."""
    if x is None:
        return None, None, None
    if _is_torch(x):
        if not x.is_cuda:
            x = x.numpy()
        else:
            import torch
            tdt = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
            if x.dtype != tdt or not x.is_contiguous():
                x = x.to(tdt).contiguous()
            _count(x.numel(), n, what)
            return c_void_p(x.data_ptr()), x, MEM_DEVICE
    a = np.ascontiguousarray(x, dtype=dtype)
    _count(a.size, n, what)
    return a.ctypes.data_as(c_void_p), a, MEM_HOST


class Solver:
    """One lattice + flow field on the GPU (a ``rfb_soc_handle``).

    ``state_generation`` counts the calls that may change what an adjoint differentiates
    (the forward or U_mt state, the operating point, the area multipliers); the
    autograd bridge compares it between its forward and backward."""

    def __init__(self, dims, dx, solid, U, V, W, D, k0, alpha=0.5, n_e=2, T=298.0, c0=20.0,
                 area_mult=None, stream=None, kinetics_mode=KIN_AFFINE):
        L = lib()
        self.dims = tuple(int(d) for d in dims)
        d = (c_int32 * 3)(*self.dims)
        kin = Kinetics(float(k0), float(alpha), int(n_e), int(kinetics_mode), float(T),
                       float(c0))
        nx, ny, nz = self.dims
        N = nx * ny * nz
        ptrs = [_ptr(solid, np.uint8, N, "solid"),
                _ptr(U, np.float64, (nx + 1) * ny * nz, "U"),
                _ptr(V, np.float64, nx * (ny + 1) * nz, "V"),
                _ptr(W, np.float64, nx * ny * (nz + 1), "W"),
                _ptr(area_mult, np.float64, N, "area_mult")]
        kinds = {p[2] for p in ptrs if p[2] is not None}
        if len(kinds) != 1:
            raise ValueError("all arrays must be host (numpy) or all CUDA tensors")
        kind = kinds.pop()
        self._keep = [p[1] for p in ptrs]
        h = c_void_p()
        st = L.rfb_soc_create(d, float(dx), ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0],
                              float(D), byref(kin), ptrs[4][0], kind, _stream_ptr(stream),
                              byref(h))
        self._keep = None
        if st != RFB_OK:
            raise RfbError(st, L.rfb_soc_last_error(None).decode())
        self.h = h
        self.state_generation = 0
        n, nf = c_int64(), c_int64()
        L.rfb_soc_info(h, byref(n), byref(nf))
        self.n_cells, self.n_fluid = n.value, nf.value

    @classmethod
    def from_case(cls, case, area_mult=None, stream=None, device_inputs=False,
                  kinetics_mode=0):
        arrays = [case.solid, case.U, case.V, case.W]
        if device_inputs:
            import torch
            arrays = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]
            if area_mult is not None:
                area_mult = torch.from_numpy(np.ascontiguousarray(area_mult)).cuda()
        return cls(case.dims, case.h, *arrays, case.D, case.k0, case.alpha, case.n_e, case.T,
                   case.c0, area_mult=area_mult, stream=stream, kinetics_mode=kinetics_mode)

    def _check(self, st, ok=(RFB_OK,)):
        if st not in ok:
            raise RfbError(st, lib().rfb_soc_last_error(self.h).decode())
        return st

    def _changing(self):
        """Called before every call that may change the handle's states or operating
        point (also when the call then fails: it may have changed them part way)."""
        self.state_generation = getattr(self, "state_generation", 0) + 1

    def solve(self, s_in, eta, tol, allow_not_converged=False, **opts) -> dict:
        r = SolveResult()
        o = make_opts(**opts)
        self._changing()
        st = lib().rfb_soc_solve(self.h, float(s_in), float(eta), float(tol), byref(o), byref(r))
        self._check(st, (RFB_OK, RFB_ERR_NOT_CONVERGED) if allow_not_converged else (RFB_OK,))
        out = r.as_dict()
        out["status"] = st
        return out

    def step(self, s_in, eta, n, **opts) -> dict:
        r = SolveResult()
        o = make_opts(**opts)
        self._changing()
        self._check(lib().rfb_soc_step(self.h, float(s_in), float(eta), int(n), byref(o), byref(r)))
        return r.as_dict()

    def solve_nernst(self, s_in, eta, tol, omega=1.0, allow_not_converged=False, **opts) -> dict:
        """rfb_soc_solve_nernst: the SBV steady state by the Nernst model (FP64)."""
        r = SolveResult()
        o = make_opts(**opts)
        self._changing()
        st = lib().rfb_soc_solve_nernst(self.h, float(s_in), float(eta), float(tol),
                                        float(omega), byref(o), byref(r))
        self._check(st, (RFB_OK, RFB_ERR_NOT_CONVERGED) if allow_not_converged else (RFB_OK,))
        out = r.as_dict()
        out["status"] = st
        return out

    def solve_bv(self, s_in, eta, tol, D_H=0.0, D_X=0.0, c_H_in=0.0, cg_rtol=0.0, cycle=0,
                 max_cg=0, start="auto", allow_not_converged=False, **opts) -> dict:
        """rfb_soc_solve_bv: the Butler-Volmer model with electromigration (FP64); zero
        parameters take the library's defaults."""
        q = BVParams(float(D_H), float(D_X), float(c_H_in), float(cg_rtol), int(cycle),
                     int(max_cg), BV_START[start] if isinstance(start, str) else int(start), 0)
        r = BVResult()
        o = make_opts(**opts)
        self._changing()
        st = lib().rfb_soc_solve_bv(self.h, float(s_in), float(eta), float(tol), byref(q),
                                    byref(o), byref(r))
        self._check(st, (RFB_OK, RFB_ERR_NOT_CONVERGED) if allow_not_converged else (RFB_OK,))
        out = r.as_dict()
        out["status"] = st
        return out

    def get_bv_state(self) -> dict:
        """The last Butler-Volmer state: C_O, C_R, C_H [mol/m^3] and phi [V] (host arrays)."""
        out = {k: np.empty(self.n_cells, dtype=np.float64) for k in ("O", "R", "H", "phi")}
        self._check(lib().rfb_soc_get_bv_state(
            self.h, out["O"].ctypes.data, out["R"].ctypes.data, out["H"].ctypes.data,
            out["phi"].ctypes.data, MEM_HOST))
        return out

    def get_overpotential(self, out=None):
        """eta~ of the last Nernst-model solve (N values, 0 off the electrode cells)."""
        if out is None:
            out = np.empty(self.n_cells, dtype=np.float64)
        p, keep, kind = _ptr(out, np.float64, self.n_cells, "out")
        if kind == MEM_HOST and keep is not out:
            raise ValueError("out must be a contiguous float64 array")
        self._check(lib().rfb_soc_get_overpotential(self.h, p, kind))
        return out

    def current(self) -> dict:
        r = SolveResult()
        self._check(lib().rfb_soc_current(self.h, byref(r)))
        return r.as_dict()

    def current_noalloc(self) -> dict:
        """rfb_soc_current_noalloc: the outputs without any device allocation (static
        scratch shared by every caller in the process; serialise overlapping calls)."""
        r = SolveResult()
        self._check(lib().rfb_soc_current_noalloc(self.h, byref(r)))
        return r.as_dict()

    def umt(self, tol, **opts):
        r = SolveResult()
        u = c_double()
        o = make_opts(**opts)
        self._changing()
        self._check(lib().rfb_soc_umt(self.h, float(tol), byref(o), byref(u), byref(r)))
        return u.value, r.as_dict()

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.n_cells, dtype=np.float64)
        p, keep, kind = _ptr(out, np.float64, self.n_cells, "out")
        if kind == MEM_HOST and keep is not out:
            raise ValueError("out must be a contiguous float64 array")
        self._check(lib().rfb_soc_get_state(self.h, p, kind))
        return out

    def set_state(self, s):
        p, keep, kind = _ptr(s, np.float64, self.n_cells, "state")
        self._changing()
        self._check(lib().rfb_soc_set_state(self.h, p, kind))

    def set_area_mult(self, m):
        """rfb_soc_set_area_mult (None = all ones)."""
        if m is None:
            self._changing()
            self._check(lib().rfb_soc_set_area_mult(self.h, None, MEM_HOST))
            return
        p, keep, kind = _ptr(m, np.float64, self.n_cells, "area_mult")
        self._changing()
        self._check(lib().rfb_soc_set_area_mult(self.h, p, kind))

    def adjoint(self, objective="I_tot", tol=1e-12, out=None, **opts):
        """rfb_soc_adjoint: returns (dJ/dm (N), dJ/dbeta, result dict)."""
        obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
        if out is None:
            out = np.empty(self.n_cells, dtype=np.float64)
        p, keep, kind = _ptr(out, np.float64, self.n_cells, "out")
        db = c_double()
        r = SolveResult()
        o = make_opts(**opts)
        self._check(lib().rfb_soc_adjoint(self.h, obj, float(tol), byref(o), p, byref(db), kind,
                                          byref(r)))
        return out, db.value, r.as_dict()

    def upsample_from(self, coarse: "Solver"):
        """rfb_soc_upsample: this (fine) handle's state := 2x prolongation of coarse's."""
        self._changing()
        self._check(lib().rfb_soc_upsample(coarse.h, self.h))

    def reset_state(self):
        self._changing()
        self._check(lib().rfb_soc_reset_state(self.h))

    def set_stream(self, stream):
        self._check(lib().rfb_soc_set_stream(self.h, _stream_ptr(stream)))

    @property
    def kernel_launches(self) -> int:
        return int(lib().rfb_soc_kernel_launches(self.h))

    def tuned_fp32_kernel(self):
        """(name, plain ms/sweep, blocked ms/sweep) chosen by the autotuner."""
        k, a, b = c_int32(), c_double(), c_double()
        self._check(lib().rfb_soc_tuned_fp32_kernel(self.h, byref(k), byref(a), byref(b)))
        names = {0: None, 1: "plain"}
        names.update({v: k for k, v in FP32_KERNEL.items() if v >= 3})
        return names[k.value], a.value, b.value

    def close(self):
        if getattr(self, "h", None):
            lib().rfb_soc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchInfo(ctypes.Structure):
    _fields_ = [("kchunk", c_int32), ("sweeps_per_cycle", c_int32), ("n_items", c_int32),
                ("grid_blocks", c_int32), ("sweep_ms", c_double), ("check_ms", c_double),
                ("cycles", c_int64), ("time_ms", c_double), ("launches", c_int64),
                ("graph_launches", c_int64), ("pass_stages", c_int32), ("pass_chunk", c_int32),
                ("pass_tile_cols", c_int32), ("df_cycles", c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Batch:
    """rfb_soc_batch_*: several Solvers advanced together (mixed precision)."""

    def __init__(self, solvers):
        L = lib()
        self.solvers = list(solvers)
        arr = (c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        b = c_void_p()
        st = L.rfb_soc_batch_create(arr, len(self.solvers), byref(b))
        if st != RFB_OK:
            raise RfbError(st, L.rfb_soc_batch_last_error(None).decode())
        self.b = b

    def set_stream(self, stream):
        st = lib().rfb_soc_batch_set_stream(self.b, _stream_ptr(stream))
        if st != RFB_OK:
            raise RfbError(st, lib().rfb_soc_batch_last_error(self.b).decode())

    def solve(self, s_in, eta, tol, allow_not_converged=False, **opts):
        n = len(self.solvers)
        s_in, eta, tol = (list(map(float, v)) for v in (s_in, eta, tol))
        if not len(s_in) == len(eta) == len(tol) == n:
            raise ValueError("s_in, eta and tol need one value per lattice (%d)" % n)
        opts.setdefault("precision", "mixed")
        D = c_double * n
        res = (SolveResult * n)()
        info = BatchInfo()
        o = make_opts(**opts)
        for sv in self.solvers:
            sv._changing()
        st = lib().rfb_soc_batch_solve(self.b, D(*s_in), D(*eta), D(*tol), byref(o), res,
                                       byref(info))
        ok = (RFB_OK, RFB_ERR_NOT_CONVERGED) if allow_not_converged else (RFB_OK,)
        if st not in ok:
            raise RfbError(st, lib().rfb_soc_batch_last_error(self.b).decode())
        return [r.as_dict() for r in res], info.as_dict()

    def close(self):
        if getattr(self, "b", None):
            lib().rfb_soc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(int(stream.cuda_stream))


def selftest_bounded_wait(spin_limit=1 << 12) -> bool:
    """rfb_selftest_bounded_wait: True if a wait on a barrier that never completes gave up
    after spin_limit polls, set the error word and let its kernel finish."""
    g = c_int32()
    st = lib().rfb_selftest_bounded_wait(int(spin_limit), byref(g))
    if st != RFB_OK:
        raise RfbError(st, lib().rfb_soc_last_error(None).decode())
    return bool(g.value)

