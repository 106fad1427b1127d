"""The C-ABI library builds, loads and exports every symbol its header declares (no GPU
work: only host-side entry points are called)."""
import ctypes
import os
import re

import pytest

from paper_2502_08034_gb300 import _build, rfb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rfb_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return rfb.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"rfb_soc_create", "rfb_soc_solve", "rfb_soc_umt", "rfb_soc_current"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_default_opts(lib):
    for st in range(8):
        assert lib.rfb_status_string(st)
    o = rfb.make_opts()
    assert o.cfl == 0.4 and o.velocity_scale == 1.0 and o.precision == 0
    assert o.dt_mode == rfb.DT["local"]


def test_create_rejects_bad_dims_before_touching_a_device(lib):
    import numpy as np
    dims = (ctypes.c_int32 * 3)(4, 4, 1)       # nz must be >= 2
    kin = rfb.Kinetics(1e-7, 0.5, 2, 0, 298.0, 20.0)
    a = np.zeros(64)
    h = ctypes.c_void_p()
    p = a.ctypes.data_as(ctypes.c_void_p)
    st = lib.rfb_soc_create(dims, 1e-6, p, p, p, p, 4e-10, ctypes.byref(kin), None, 0, None,
                            ctypes.byref(h))
    assert st == rfb.RFB_ERR_INVALID_ARG
    assert b"dims" in lib.rfb_soc_last_error(None)
    dims = (ctypes.c_int32 * 3)(4, 4, 4)
    kin = rfb.Kinetics(1e-7, 1.5, 2, 0, 298.0, 20.0)   # alpha out of range
    st = lib.rfb_soc_create(dims, 1e-6, p, p, p, p, 4e-10, ctypes.byref(kin), None, 0, None,
                            ctypes.byref(h))
    assert st == rfb.RFB_ERR_INVALID_ARG
    # largest lattice: N + nx*ny must stay below 2^31 (32-bit cell indices in the kernels)
    kin = rfb.Kinetics(1e-7, 0.5, 2, 0, 298.0, 20.0)
    dims = (ctypes.c_int32 * 3)(1024, 1024, 2048)
    st = lib.rfb_soc_create(dims, 1e-6, p, p, p, p, 4e-10, ctypes.byref(kin), None, 0, None,
                            ctypes.byref(h))
    assert st == rfb.RFB_ERR_INVALID_ARG and b"too large" in lib.rfb_soc_last_error(None)
    kin = rfb.Kinetics(1e-7, 0.5, 2, 7, 298.0, 20.0)     # unknown kinetics mode
    dims = (ctypes.c_int32 * 3)(4, 4, 4)
    st = lib.rfb_soc_create(dims, 1e-6, p, p, p, p, 4e-10, ctypes.byref(kin), None, 0, None,
                            ctypes.byref(h))
    assert st == rfb.RFB_ERR_INVALID_ARG
    assert lib.rfb_soc_destroy(None) == 0


def _create(lib, dims=(4, 4, 4), dx=1e-6, D=4e-10, kin=None, kind=0, null=(), out=True):
    import numpy as np
    a = np.zeros(256)
    p = a.ctypes.data_as(ctypes.c_void_p)
    ptrs = [None if i in null else p for i in range(4)]          # mask, U, V, W
    d = None if "dims" in null else (ctypes.c_int32 * 3)(*dims)
    k = None if "kin" in null else ctypes.byref(kin or rfb.Kinetics(1e-7, 0.5, 2, 0, 298.0, 20.0))
    h = ctypes.c_void_p()
    st = lib.rfb_soc_create(d, dx, *ptrs, D, k, None, kind, None,
                            ctypes.byref(h) if out else None)
    return st, lib.rfb_soc_last_error(None)


NAN = float("nan")


@pytest.mark.parametrize("case,kw,msg", [
    ("out NULL", dict(out=False), b"out is NULL"),
    ("dims NULL", dict(null=("dims",)), b"NULL input"),
    ("mask NULL", dict(null=(0,)), b"NULL input"),
    ("W NULL", dict(null=(3,)), b"NULL input"),
    ("kinetics NULL", dict(null=("kin",)), b"NULL input"),
    ("memory kind", dict(kind=5), b"kind"),
    ("nx = 0", dict(dims=(0, 4, 4)), b"dims"),
    ("nz = 1", dict(dims=(4, 4, 1)), b"dims"),
    ("N + nx ny >= 2^31", dict(dims=(2048, 1024, 1024)), b"too large"),
    ("dx = 0", dict(dx=0.0), b"dx and D"),
    ("dx NaN", dict(dx=NAN), b"dx and D"),
    ("D < 0", dict(D=-1.0), b"dx and D"),
    ("D inf", dict(D=float("inf")), b"dx and D"),
    ("k0 < 0", dict(kin=rfb.Kinetics(-1e-7, 0.5, 2, 0, 298.0, 20.0)), b"kinetics out of range"),
    ("k0 NaN", dict(kin=rfb.Kinetics(NAN, 0.5, 2, 0, 298.0, 20.0)), b"kinetics out of range"),
    ("alpha = 0", dict(kin=rfb.Kinetics(1e-7, 0.0, 2, 0, 298.0, 20.0)), b"kinetics out of range"),
    ("alpha = 1", dict(kin=rfb.Kinetics(1e-7, 1.0, 2, 0, 298.0, 20.0)), b"kinetics out of range"),
    ("n_e = 0", dict(kin=rfb.Kinetics(1e-7, 0.5, 0, 0, 298.0, 20.0)), b"kinetics out of range"),
    ("T = 0", dict(kin=rfb.Kinetics(1e-7, 0.5, 2, 0, 0.0, 20.0)), b"kinetics out of range"),
    ("c0 < 0", dict(kin=rfb.Kinetics(1e-7, 0.5, 2, 0, 298.0, -20.0)), b"kinetics out of range"),
    ("mode 2", dict(kin=rfb.Kinetics(1e-7, 0.5, 2, 2, 298.0, 20.0)), b"kinetics mode"),
    ("mode -1", dict(kin=rfb.Kinetics(1e-7, 0.5, 2, -1, 298.0, 20.0)), b"kinetics mode"),
])
def test_create_validates_arguments_on_the_host(lib, case, kw, msg):
    """Every argument check of rfb_soc_create that precedes device work, one at a time:
    RFB_ERR_INVALID_ARG and a message naming the argument."""
    st, err = _create(lib, **kw)
    assert st == rfb.RFB_ERR_INVALID_ARG, case
    assert msg in err, (case, err)


NO_STATUS = {"rfb_soc_last_error", "rfb_soc_batch_last_error", "rfb_soc_kernel_launches",
             "rfb_status_string", "rfb_solve_opts_default"}


def _neutral(t):
    if t is ctypes.c_double:
        return 0.5
    if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_long):
        return 1
    return None                      # handles, pointers, structs by pointer


def test_every_handle_call_refuses_a_null_handle(lib):
    """Each declared call whose first argument is a solver or batch handle returns
    RFB_ERR_INVALID_ARG for a NULL handle (destroy calls return RFB_OK), before any
    device work; the error getters return a string and the launch counter 0."""
    seen = 0
    for name in sorted(_declared()):
        f = getattr(lib, name)
        if name in NO_STATUS or not f.argtypes or f.argtypes[0] is not ctypes.c_void_p:
            continue
        args = [None] + [_neutral(t) for t in f.argtypes[1:]]
        want = rfb.RFB_OK if name.endswith("_destroy") else rfb.RFB_ERR_INVALID_ARG
        assert f(*args) == want, name
        seen += 1
    assert seen >= 20, seen
    assert isinstance(lib.rfb_soc_last_error(None), bytes)
    assert isinstance(lib.rfb_soc_batch_last_error(None), bytes)
    assert lib.rfb_soc_kernel_launches(None) == 0


def test_batch_create_and_bounded_wait_check_their_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.rfb_soc_batch_create(None, 0, ctypes.byref(out)) == rfb.RFB_ERR_INVALID_ARG
    assert b"at least one handle" in lib.rfb_soc_batch_last_error(None)
    handles = (ctypes.c_void_p * 2)(None, None)
    assert lib.rfb_soc_batch_create(handles, 2, ctypes.byref(out)) == rfb.RFB_ERR_INVALID_ARG
    assert b"NULL handle" in lib.rfb_soc_batch_last_error(None)
    assert lib.rfb_soc_batch_create(handles, 2, None) == rfb.RFB_ERR_INVALID_ARG
    gave_up = ctypes.c_int32()
    for limit, ptr in ((0, ctypes.byref(gave_up)), ((1 << 26) + 1, ctypes.byref(gave_up)),
                       (100, None)):
        assert lib.rfb_selftest_bounded_wait(limit, ptr) == rfb.RFB_ERR_INVALID_ARG
    assert b"spin_limit" in lib.rfb_soc_last_error(None)


@pytest.mark.parametrize("bad", ["solid", "U", "V", "W", "area_mult"])
def test_binding_checks_array_sizes_before_the_c_call(lib, bad):
    """The C ABI reads as many values as the lattice needs from each pointer; the binding
    refuses an array of another size (here one value short) before calling it."""
    import numpy as np
    nx, ny, nz = 4, 5, 6
    N = nx * ny * nz
    sizes = {"solid": N, "U": (nx + 1) * ny * nz, "V": nx * (ny + 1) * nz,
             "W": nx * ny * (nz + 1), "area_mult": N}
    arrays = {k: np.zeros(v - (1 if k == bad else 0)) for k, v in sizes.items()}
    with pytest.raises(ValueError, match=bad):
        rfb.Solver((nx, ny, nz), 1e-6, arrays["solid"].astype(np.uint8), arrays["U"],
                   arrays["V"], arrays["W"], 4e-10, 1e-7, area_mult=arrays["area_mult"])


def test_binding_checks_batch_argument_lengths(lib):
    b = rfb.Batch.__new__(rfb.Batch)          # no device: only the argument check runs
    b.solvers, b.b = [None, None], None
    with pytest.raises(ValueError, match="one value per lattice"):
        b.solve([0.5], [-0.1, -0.1], [1e-8, 1e-8])
    with pytest.raises(ValueError, match="one value per lattice"):
        b.solve([0.5, 0.5], [-0.1, -0.1], [1e-8, 1e-8, 1e-8])


def test_binding_passes_arrays_of_the_right_size_to_the_c_call(lib):
    """Arrays in the face layouts of the synthetic inputs pass the size checks and reach
    rfb_soc_create (which, without a GPU, then reports the CUDA error)."""
    import numpy as np
    from paper_2502_08034_gb300 import synth
    for dims in ((6, 5, 4), (3, 7, 2)):
        nx, ny, nz = dims
        solid = np.zeros((nz, ny, nx), dtype=np.uint8)
        U, V, W = np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))
        try:
            rfb.Solver(dims, 1e-6, solid, U, V, W, 4e-10, 1e-7, area_mult=np.ones(solid.shape)).close()
        except rfb.RfbError as e:
            assert e.status == rfb.RFB_ERR_CUDA, str(e)
    assert synth.logpile_dims(10e-6) == (16, 64, 128)


# ------------------------------------------------------- the binding matches the header

def _header_text():
    txt = open(os.path.join(ROOT, "include", "rfb_soc.h")).read()
    return re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)


def _header_enums():
    out = {}
    for body in re.findall(r"typedef enum \w+ \{(.*?)\}", _header_text(), flags=re.S):
        for name, val in re.findall(r"(\w+)\s*=\s*(\d+)", body):
            out[name] = int(val)
    return out


def _header_structs():
    out = {}
    for name, body in re.findall(r"typedef struct (\w+) \{(.*?)\}", _header_text(), flags=re.S):
        fields = []
        for ctype, fname, arr in re.findall(r"(int32_t|int64_t|double)\s+(\w+)\s*(?:\[(\d+)\])?;",
                                            body):
            fields.append((fname, ctype, int(arr) if arr else None))
        out[name] = fields
    return out


def test_binding_enums_match_the_header():
    e = _header_enums()
    assert (e["RFB_OK"], e["RFB_ERR_INVALID_ARG"], e["RFB_ERR_CUDA"], e["RFB_ERR_OOM"],
            e["RFB_ERR_NOT_CONVERGED"], e["RFB_ERR_NONFINITE"], e["RFB_ERR_STATE"],
            e["RFB_ERR_UNSUPPORTED"]) == (rfb.RFB_OK, rfb.RFB_ERR_INVALID_ARG, rfb.RFB_ERR_CUDA,
                                          rfb.RFB_ERR_OOM, rfb.RFB_ERR_NOT_CONVERGED,
                                          rfb.RFB_ERR_NONFINITE, rfb.RFB_ERR_STATE,
                                          rfb.RFB_ERR_UNSUPPORTED)
    assert (e["RFB_MEM_HOST"], e["RFB_MEM_DEVICE"]) == (rfb.MEM_HOST, rfb.MEM_DEVICE)
    assert rfb.PREC == {"fp64": e["RFB_PREC_FP64"], "mixed": e["RFB_PREC_MIXED"]}
    assert rfb.INLET == {"face": e["RFB_INLET_FACE"], "ghost": e["RFB_INLET_GHOST"]}
    assert rfb.DT == {"global": e["RFB_DT_GLOBAL"], "local": e["RFB_DT_LOCAL"]}
    assert (rfb.KIN_AFFINE, rfb.KIN_UNIFORM_ETA) == (e["RFB_KIN_AFFINE"], e["RFB_KIN_UNIFORM_ETA"])
    assert rfb.OBJECTIVES == {"I_tot": e["RFB_OBJ_I_TOT"], "U": e["RFB_OBJ_U"],
                              "U_mt": e["RFB_OBJ_U_MT"]}


def test_binding_structs_match_the_header():
    """Field names, order, types and array lengths of every struct the binding mirrors."""
    cmap = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    s = _header_structs()
    for cname, py in (("rfb_kinetics", rfb.Kinetics), ("rfb_solve_opts", rfb.SolveOpts),
                      ("rfb_solve_result", rfb.SolveResult), ("rfb_batch_info", rfb.BatchInfo),
                      ("rfb_bv_params", rfb.BVParams), ("rfb_bv_result", rfb.BVResult)):
        want = s[cname]
        got = py._fields_
        assert [f[0] for f in got] == [f[0] for f in want], cname
        for (fname, ftype), (_, ctype, arr) in zip(got, want):
            if arr is None:
                assert ftype is cmap[ctype], (cname, fname)
            else:
                assert ftype._type_ is cmap[ctype] and ftype._length_ == arr, (cname, fname)


def test_binding_argument_types_match_the_header(lib):
    """Each declared function's parameters against the ctypes argtypes: pointers to
    pointer types, doubles to c_double, 64-bit integers to c_int64, 32-bit integers and
    enums to c_int32."""
    txt = _header_text()
    protos = re.findall(r"\b(?:rfb_status|void|const char\*|int64_t)\s+(rfb_\w+)\s*\((.*?)\);",
                        txt, flags=re.S)
    assert len(protos) >= 25
    for name, params in protos:
        f = getattr(lib, name)
        plist = [p.strip() for p in params.split(",")] if params.strip() else []
        assert len(plist) == len(f.argtypes), name
        for p, t in zip(plist, f.argtypes):
            if "*" in p or "[" in p:
                assert t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and \
                    t.__name__.startswith("LP_"), (name, p, t)
            elif p.startswith("double"):
                assert t is ctypes.c_double, (name, p, t)
            elif p.startswith("int64_t"):
                assert t is ctypes.c_int64, (name, p, t)
            else:
                assert t is ctypes.c_int32, (name, p, t)


def test_no_fallback_when_the_library_is_missing(monkeypatch, tmp_path):
    """Without the built CUDA library every entry point raises: there is no CPU path."""
    import numpy as np
    monkeypatch.setattr(rfb, "_LIB", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "librfbsoc.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        rfb.lib()
    z = np.zeros(2 * 2 * 3)
    with pytest.raises(RuntimeError, match="no fallback"):
        rfb.Solver((2, 2, 3), 1e-6, z.astype(np.uint8), np.zeros(3 * 2 * 3),
                   np.zeros(2 * 3 * 3), np.zeros(2 * 2 * 4), 4e-10, 1e-7)
