"""Python binding of the C ABI in ``include/nuasm.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but check argument shapes/dtypes, pass pointers and translate status
codes into exceptions: all computation runs in ``libnuasm.so``.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; host arrays are staged by the
library itself.  Importing this module does not need a GPU; loading the
library does need the shared object, and a missing library is an error (there
is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# NUASM_LIBRARY selects another build of the same C ABI (the bounds-checking
# debug library, libnuasm_debug.so); it must exist like the default one.
LIB_PATH = os.environ.get("NUASM_LIBRARY") or os.path.join(_PKG, "libnuasm.so")

KIND_ASM, KIND_FRESNEL = 0, 1
PREC_F32_F64PHASE, PREC_F64 = 0, 1

STATUS = {0: "NUASM_OK", 1: "NUASM_EINVAL", 2: "NUASM_ERANGE", 3: "NUASM_ENOMEM",
          4: "NUASM_ECUDA", 5: "NUASM_ETIMEOUT", 6: "NUASM_EUNSUPPORTED"}
STAGES = ["h2d", "spread", "col_fwd_fold", "row_t1", "col_inv", "col_fwd", "row_t2",
          "col_inv_fold", "interp", "d2h", "row_t3"]


class NuasmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_strerror(code)})")


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_pad", ctypes.c_int32), ("pitch", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("z", ctypes.c_double), ("ox", ctypes.c_double),
                ("oy", ctypes.c_double), ("band_auto", ctypes.c_int32), ("c_m", ctypes.c_double),
                ("c_n", ctypes.c_double), ("w_m", ctypes.c_double), ("w_n", ctypes.c_double),
                ("kind", ctypes.c_int32), ("prec", ctypes.c_int32), ("tol", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("tile", ctypes.c_int32), ("interp_chunk", ctypes.c_int32),
                ("spread_chunk", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_pad", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("window", ctypes.c_int32), ("window_origin", ctypes.c_int32),
                ("kernel_width", ctypes.c_int32), ("kernel_beta", ctypes.c_double),
                ("tile", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("band_lo_x", ctypes.c_int32), ("band_hi_x", ctypes.c_int32),
                ("band_lo_y", ctypes.c_int32), ("band_hi_y", ctypes.c_int32),
                ("points", ctypes.c_int64), ("records", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("phase_table_bytes", ctypes.c_int64),
                ("bank_skew", ctypes.c_int32), ("spread_split_ctas", ctypes.c_int32),
                ("double_float", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("type", ctypes.c_int32),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("device", ctypes.c_int32), ("hbm_budget", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("p", Params), ("type", ctypes.c_int32), ("points_id", ctypes.c_uint64), ("m", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reused_points", ctypes.c_int32), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "failed", "points")] + \
               [("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("wall_s", ctypes.c_double)] + \
               [(f, ctypes.c_int64) for f in ("resident_sets", "resident_bytes", "bins_built", "bins_reused",
                                              "evictions", "peak_bytes")]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "nuasm_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params), ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nuasm_plan_lattice": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_void_p]),
    "nuasm1_execute": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "nuasm2_execute": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "nufresnel_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "nuasm3_execute": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "nufresnel3_execute": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "nuasm_rs_direct": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nuasm_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "nuasm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "nuasm_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "nuasm_band": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int32)]),
    "nuasm_kernel_shape": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "nuasm_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "nuasm_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "nuasm_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "nuasm2_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nuasm_autotune_tile": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double)]),
    "nuasm_autotune": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Params),
                                      ctypes.POINTER(ctypes.c_double)]),
    "nuasm_debug_bounded_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p]),
    "nuasm_debug_plan_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "nuasm_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int64]),
    "nuasm_debug_live_resources": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "nuasm_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.c_int32]),
    "nuasm_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(BatchItem),
                                          ctypes.c_int32, ctypes.c_int32]),
    "nuasm_batch_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "nuasm_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "nuasm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "nuasm_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ServerConfig)]),
    "nuasm_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
    "nuasm_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                         ctypes.POINTER(RequestResult)]),
    "nuasm_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats), ctypes.c_int32]),
    "nuasm_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def lib() -> ctypes.CDLL:
    """Load libnuasm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _strerror(code: int) -> str:
    try:
        return lib().nuasm_strerror(int(code)).decode()
    except Exception:  # pragma: no cover
        return "?"


def _check(code: int, where: str):
    if code != 0:
        raise NuasmError(code, where)


# ---------------------------------------------------------------- marshalling
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _numel(a) -> int:
    return int(a.numel()) if _is_torch(a) else int(a.size)


def _dtype_name(a) -> str:
    return str(a.dtype).replace("torch.", "")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


KERNEL_ES, KERNEL_GAUSSIAN = 0, 1


def make_params(n, pitch, lam, z, ox=0.0, oy=0.0, kind="asm", prec="f32", tol=0.0, n_pad=0,
                band=None, kernel="es", tile=0, interp_chunk=0, spread_chunk=0) -> Params:
    """nuasm_params_t from keyword values; band = (c_m, c_n, w_m, w_n) or None
    (auto rule); kernel = "es" (exponential of semicircle) or "gaussian";
    tile = gridding tile side (0: the library's rule); interp_chunk /
    spread_chunk = records per CTA of split tiles (0: the library's rule)."""
    p = Params()
    p.n, p.n_pad, p.pitch, p.lambda_, p.z, p.ox, p.oy = int(n), int(n_pad), pitch, lam, z, ox, oy
    if band is None:
        p.band_auto = 1
    else:
        p.band_auto = 0
        p.c_m, p.c_n, p.w_m, p.w_n = (float(v) for v in band)
    p.kind = KIND_ASM if kind in ("asm", KIND_ASM) else KIND_FRESNEL
    p.prec = PREC_F64 if prec in ("f64", PREC_F64) else PREC_F32_F64PHASE
    p.tol = float(tol)
    p.kernel = KERNEL_GAUSSIAN if kernel in ("gaussian", KERNEL_GAUSSIAN) else KERNEL_ES
    p.tile = int(tile)
    p.interp_chunk = int(interp_chunk)
    p.spread_chunk = int(spread_chunk)
    return p


class Plan:
    """Owner of a nuasm_plan_t handle."""

    def __init__(self, handle: ctypes.c_void_p, params: Params, m: int):
        self.handle = handle
        self.params = params
        self.m = m
        self.n = params.n
        self.complex_dtype = "complex128" if params.prec == PREC_F64 else "complex64"

    @property
    def _h(self):
        if not self.handle:
            raise RuntimeError("plan has been destroyed")
        return self.handle

    def info(self) -> dict:
        return nuasm_plan_info(self)

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(lib().nuasm_destroy(h), "nuasm_destroy")

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.destroy()
        except Exception:
            pass


def _expect(a, count: int, dtype: str, what: str):
    if a is None:
        if count == 0:
            return
        raise ValueError(f"{what} is required")
    if _numel(a) != count:
        raise ValueError(f"{what} must have {count} elements, got {_numel(a)}")
    if _dtype_name(a) != dtype:
        raise TypeError(f"{what} must be {dtype}, got {_dtype_name(a)}")


def nuasm_plan(params: Params, x, y, w=None, stream=None) -> Plan:
    """Build a plan (see nuasm_plan in include/nuasm.h).  x, y, w: float64 arrays of M entries."""
    m = 0 if x is None else _numel(x)
    for a, name in ((x, "x"), (y, "y"), (w, "w")):
        if a is not None:
            _expect(a, m, "float64", name)
    h = ctypes.c_void_p()
    _check(lib().nuasm_plan(ctypes.byref(h), ctypes.byref(params), m, _ptr(x), _ptr(y), _ptr(w),
                            _stream(stream)), "nuasm_plan")
    return Plan(h, params, m)


def nuasm_plan_lattice(params: Params, nx: int, ny: int, pitch2: float, x0: float, y0: float,
                       stream=None) -> Plan:
    """Plan over the lattice x0 + i pitch2, y0 + j pitch2 (point index j nx + i)."""
    h = ctypes.c_void_p()
    _check(lib().nuasm_plan_lattice(ctypes.byref(h), ctypes.byref(params), int(nx), int(ny), float(pitch2),
                                    float(x0), float(y0), _stream(stream)), "nuasm_plan_lattice")
    return Plan(h, params, int(nx) * int(ny))


def nuasm1_execute(plan: Plan, c, u2, stream=None):
    """NU-ASM_1: c (M complex) -> u2 (N*N complex)."""
    _expect(c, plan.m, plan.complex_dtype, "c")
    _expect(u2, plan.n * plan.n, plan.complex_dtype, "u2")
    _check(lib().nuasm1_execute(plan._h, _ptr(c), _ptr(u2), _stream(stream)), "nuasm1_execute")
    return u2


def nuasm2_execute(plan: Plan, u1, v, stream=None):
    """NU-ASM_2: u1 (N*N complex) -> v (M complex)."""
    _expect(u1, plan.n * plan.n, plan.complex_dtype, "u1")
    _expect(v, plan.m, plan.complex_dtype, "v")
    _check(lib().nuasm2_execute(plan._h, _ptr(u1), _ptr(v), _stream(stream)), "nuasm2_execute")
    return v


def nufresnel_execute(plan: Plan, type_: int, inp, out, stream=None):
    """NU-FRE_1 (type 1: M -> N*N) or NU-FRE_2 (type 2: N*N -> M)."""
    if type_ == 1:
        _expect(inp, plan.m, plan.complex_dtype, "in")
        _expect(out, plan.n * plan.n, plan.complex_dtype, "out")
    elif type_ == 2:
        _expect(inp, plan.n * plan.n, plan.complex_dtype, "in")
        _expect(out, plan.m, plan.complex_dtype, "out")
    _check(lib().nufresnel_execute(plan._h, int(type_), _ptr(inp), _ptr(out), _stream(stream)),
           "nufresnel_execute")
    return out


def nuasm3_execute(src: Plan, dst: Plan, c, v, stream=None):
    """NU-ASM_3: c (src.m complex, at src's points) -> v (dst.m complex, at dst's points)."""
    _expect(c, src.m, src.complex_dtype, "c")
    _expect(v, dst.m, dst.complex_dtype, "v")
    _check(lib().nuasm3_execute(src._h, dst._h, _ptr(c), _ptr(v), _stream(stream)), "nuasm3_execute")
    return v


def nufresnel3_execute(src: Plan, dst: Plan, c, v, stream=None):
    """NU-FRE_3: as nuasm3_execute with the Fresnel transfer function."""
    _expect(c, src.m, src.complex_dtype, "c")
    _expect(v, dst.m, dst.complex_dtype, "v")
    _check(lib().nufresnel3_execute(src._h, dst._h, _ptr(c), _ptr(v), _stream(stream)), "nufresnel3_execute")
    return v


def nuasm_rs_direct(params: Params, x1, y1, c, area, x2, y2, out, stream=None):
    """Rayleigh-Sommerfeld direct sum (Eq. 10): device arrays x1, y1, area
    (float64, m1), c (complex, m1), x2, y2 (float64, m2) -> out (complex, m2)."""
    m1 = 0 if x1 is None else _numel(x1)
    m2 = _numel(x2)
    cdt = "complex128" if params.prec == PREC_F64 else "complex64"
    for a, nm in ((x1, "x1"), (y1, "y1"), (area, "area")):
        if a is not None:
            _expect(a, m1, "float64", nm)
    _expect(c, m1, cdt, "c")
    _expect(y2, m2, "float64", "y2")
    _expect(out, m2, cdt, "out")
    _check(lib().nuasm_rs_direct(ctypes.byref(params), m1, _ptr(x1), _ptr(y1), _ptr(c), _ptr(area), m2, _ptr(x2),
                                 _ptr(y2), _ptr(out), _stream(stream)), "nuasm_rs_direct")
    return out


def nuasm_destroy(plan: Plan):
    plan.destroy()


def nuasm_strerror(code: int) -> str:
    return _strerror(code)


def nuasm_plan_info(plan: Plan) -> dict:
    info = PlanInfo()
    _check(lib().nuasm_plan_info(plan._h, ctypes.byref(info)), "nuasm_plan_info")
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def nuasm_band(params: Params) -> tuple:
    out = (ctypes.c_int32 * 4)()
    _check(lib().nuasm_band(ctypes.byref(params), out), "nuasm_band")
    return tuple(int(v) for v in out)


def nuasm_kernel_shape(tol: float, prec: int, kernel: int = KERNEL_ES) -> tuple:
    w = ctypes.c_int32()
    b = ctypes.c_double()
    _check(lib().nuasm_kernel_shape(float(tol), int(prec), int(kernel), ctypes.byref(w), ctypes.byref(b)),
           "nuasm_kernel_shape")
    return int(w.value), float(b.value)


def nuasm_profile_enable(plan: Plan, enable: bool = True):
    _check(lib().nuasm_profile_enable(plan._h, 1 if enable else 0), "nuasm_profile_enable")


def nuasm_profile_read(plan: Plan) -> dict:
    """{stage name: (total ms, launches)} since the last read."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(lib().nuasm_profile_read(plan._h, ms, cnt), "nuasm_profile_read")
    return {lib().nuasm_stage_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}


def nuasm2_solve_noalloc(params: Params, x, y, u1, v, stream=None):
    """One-shot NU-ASM_2 that allocates nothing (see include/nuasm.h): float64
    device coordinates x, y (M), complex64 device u1 (N*N) -> complex64 v (M)."""
    m = 0 if x is None else _numel(x)
    for a, name in ((x, "x"), (y, "y")):
        if a is not None:
            _expect(a, m, "float64", name)
    _expect(u1, params.n * params.n, "complex64", "u1")
    _expect(v, m, "complex64", "v")
    _check(lib().nuasm2_solve_noalloc(ctypes.byref(params), m, _ptr(x), _ptr(y), _ptr(u1), _ptr(v),
                                      _stream(stream)), "nuasm2_solve_noalloc")
    return v


def nuasm_autotune_tile(params: Params, x, y, type_: int, stream=None) -> tuple:
    """(fastest tile side, its solve time in ms) for these device points."""
    m = _numel(x)
    _expect(x, m, "float64", "x")
    _expect(y, m, "float64", "y")
    t, ms = ctypes.c_int32(), ctypes.c_double()
    _check(lib().nuasm_autotune_tile(ctypes.byref(params), m, _ptr(x), _ptr(y), int(type_), _stream(stream),
                                     ctypes.byref(t), ctypes.byref(ms)), "nuasm_autotune_tile")
    return int(t.value), float(ms.value)


def nuasm_autotune(params: Params, x, y, type_: int, stream=None) -> tuple:
    """(the fastest Params over tile sides and split chunks, its solve time in
    ms) for these device points."""
    m = _numel(x)
    _expect(x, m, "float64", "x")
    _expect(y, m, "float64", "y")
    best, ms = Params(), ctypes.c_double()
    _check(lib().nuasm_autotune(ctypes.byref(params), m, _ptr(x), _ptr(y), int(type_), _stream(stream),
                                ctypes.byref(best), ctypes.byref(ms)), "nuasm_autotune")
    return best, float(ms.value)


def nuasm_debug_bounded_wait(spins: int, stream=None) -> int:
    """Status of a device wait that is made to run out after `spins` tries
    (NUASM_ETIMEOUT = 5 is the expected answer)."""
    code = lib().nuasm_debug_bounded_wait(int(spins), _stream(stream))
    if code not in (0, 5):
        _check(code, "nuasm_debug_bounded_wait")
    return int(code)


def nuasm_debug_plan_wait(plan: Plan, spins: int, stream=None):
    """Leave `plan`'s error word as a column pass whose copy never arrived
    would: its next execute call returns NUASM_ETIMEOUT."""
    _check(lib().nuasm_debug_plan_wait(plan._h, int(spins), _stream(stream)), "nuasm_debug_plan_wait")


def nuasm_debug_fail_alloc(k: int):
    """Make the k-th resource acquisition of the library from now fail
    (k = 0 disarms)."""
    _check(lib().nuasm_debug_fail_alloc(int(k)), "nuasm_debug_fail_alloc")


def nuasm_debug_live_resources() -> int:
    """The library's resource acquisitions not yet released."""
    n = ctypes.c_int64()
    _check(lib().nuasm_debug_live_resources(ctypes.byref(n)), "nuasm_debug_live_resources")
    return int(n.value)


def nuasm_debug_bounds(reset: bool = True):
    """(skipped out-of-range accesses, first site, its index, its extent) of
    the bounds-checking debug library; None from the normal library."""
    hits, site, index, limit = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    code = lib().nuasm_debug_bounds(ctypes.byref(hits), ctypes.byref(site), ctypes.byref(index), ctypes.byref(limit),
                                    int(bool(reset)))
    if code == 6:   # NUASM_EUNSUPPORTED: built without the checks
        return None
    _check(code, "nuasm_debug_bounds")
    return int(hits.value), int(site.value), int(index.value), int(limit.value)


# ---------------------------------------------------------------- batches
class Batch:
    """Owner of a nuasm_batch_t handle; keeps the plans and arrays it records alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def execute(self, stream=None):
        return nuasm_batch_execute(self, stream)

    def info(self) -> tuple:
        return nuasm_batch_info(self)

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(lib().nuasm_batch_destroy(h), "nuasm_batch_destroy")

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.destroy()
        except Exception:
            pass


def nuasm_batch_create(items, lanes: int = 0) -> Batch:
    """items: sequence of (plan, type, in, out) or (plan, type, in, out, dst) with device arrays."""
    arr = (BatchItem * len(items))()
    keep = []
    for i, it in enumerate(items):
        plan, type_, inp, out = it[:4]
        dst = it[4] if len(it) > 4 else None
        n_in = plan.m if type_ in (1, 3) else plan.n * plan.n
        n_out = plan.n * plan.n if type_ == 1 else (plan.m if type_ == 2 else (dst.m if dst else 0))
        _expect(inp, n_in, plan.complex_dtype, f"items[{i}].in")
        _expect(out, n_out, plan.complex_dtype, f"items[{i}].out")
        arr[i] = BatchItem(plan._h, dst._h if dst is not None else None, int(type_), _ptr(inp), _ptr(out))
        keep += [plan, dst, inp, out]
    h = ctypes.c_void_p()
    _check(lib().nuasm_batch_create(ctypes.byref(h), arr, len(items), int(lanes)), "nuasm_batch_create")
    return Batch(h, keep)


def nuasm_batch_execute(batch: Batch, stream=None):
    _check(lib().nuasm_batch_execute(batch.handle, _stream(stream)), "nuasm_batch_execute")


def nuasm_batch_info(batch: Batch) -> tuple:
    """(lanes used, kernel launches per execute)."""
    lanes, kernels = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().nuasm_batch_info(batch.handle, ctypes.byref(lanes), ctypes.byref(kernels)), "nuasm_batch_info")
    return int(lanes.value), int(kernels.value)


def nuasm_batch_destroy(batch: Batch):
    batch.destroy()


# ---------------------------------------------------------------- serving
class Server:
    """Owner of a nuasm_server_t handle.  Submitted arrays are referenced until
    their wait returns."""

    def __init__(self, handle):
        self.handle = handle
        self._pending = {}

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(lib().nuasm_server_destroy(h), "nuasm_server_destroy")
            self._pending.clear()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.destroy()
        except Exception:
            pass


def nuasm_server_create(slots: int = 0, device: int = 0, hbm_budget: int = 0) -> Server:
    cfg = ServerConfig(int(slots), int(device), int(hbm_budget))
    h = ctypes.c_void_p()
    _check(lib().nuasm_server_create(ctypes.byref(h), ctypes.byref(cfg)), "nuasm_server_create")
    return Server(h)


def nuasm_server_submit(server: Server, params: Params, type_: int, x, y, inp, out, points_id: int = 0) -> int:
    """Queue one solve; x, y: float64 (M), inp/out: host or device arrays.  Returns the ticket."""
    m = _numel(x)
    _expect(y, m, "float64", "y")
    _expect(x, m, "float64", "x")
    cdt = "complex128" if params.prec == PREC_F64 else "complex64"
    nn = params.n * params.n
    _expect(inp, m if type_ == 1 else nn, cdt, "in")
    _expect(out, nn if type_ == 1 else m, cdt, "out")
    req = Request(params, int(type_), int(points_id), m, _ptr(x), _ptr(y), _ptr(inp), _ptr(out))
    t = ctypes.c_int64()
    _check(lib().nuasm_server_submit(server.handle, ctypes.byref(req), ctypes.byref(t)), "nuasm_server_submit")
    server._pending[int(t.value)] = (x, y, inp, out)
    return int(t.value)


def nuasm_server_wait(server: Server, ticket: int, timeout_s: float = -1.0) -> dict:
    """Block until the request completes; returns its status and timings
    (raises NuasmError with NUASM_ETIMEOUT when the limit passes first)."""
    r = RequestResult()
    _check(lib().nuasm_server_wait(server.handle, int(ticket), float(timeout_s), ctypes.byref(r)),
           "nuasm_server_wait")
    server._pending.pop(int(ticket), None)
    return {"status": int(r.status), "reused_points": bool(r.reused_points), "latency_ms": float(r.latency_ms),
            "queue_ms": float(r.queue_ms)}


def nuasm_server_stats(server: Server, reset: bool = False) -> dict:
    st = ServerStats()
    _check(lib().nuasm_server_stats(server.handle, ctypes.byref(st), 1 if reset else 0), "nuasm_server_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def nuasm_server_destroy(server: Server):
    server.destroy()
