"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every symbol include/nuasm.h declares, validates parameters
before touching the device, and its host-only band and kernel queries agree
with the oracle and the documented rules."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_6644_gb300 as pkg
    return pkg


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "nuasm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:nuasm|nufresnel)\w*)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("nuasm_plan", "nuasm1_execute", "nuasm2_execute", "nufresnel_execute",
                     "nuasm_destroy", "nuasm_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(P):
    from paper_1308_6644_gb300 import nuasm as B
    assert set(_declared_functions()) <= set(B._SIGS)


def test_strerror_names_every_status(P):
    for code in range(7):
        assert P.nuasm_strerror(code) not in ("unknown status", "")
    assert P.nuasm_strerror(99) == "unknown status"


@pytest.mark.parametrize("kw,code", [
    (dict(n=64, pitch=10e-6, lam=-1.0, z=0.1), 1),            # lambda <= 0
    (dict(n=64, pitch=0.0, lam=633e-9, z=0.1), 1),            # pitch <= 0
    (dict(n=63, pitch=10e-6, lam=633e-9, z=0.1), 1),          # odd N
    (dict(n=64, pitch=10e-6, lam=633e-9, z=0.0, kind="fresnel"), 1),   # Fresnel z = 0
    (dict(n=64, pitch=10e-6, lam=633e-9, z=0.1, n_pad=129), 1),  # N' odd
    (dict(n=64, pitch=10e-6, lam=633e-9, z=0.1, n_pad=192), 6),  # N' even, not a power of two
    (dict(n=64, pitch=10e-6, lam=633e-9, z=0.1, n_pad=64), 1),  # N' < 2N
    (dict(n=64, pitch=10e-6, lam=633e-9, z=0.1, tol=0.5), 1),   # tolerance out of range
    (dict(n=48, pitch=10e-6, lam=633e-9, z=0.1), 6),          # N even, not a power of two
    (dict(n=384, pitch=10e-6, lam=633e-9, z=0.1), 6),
    (dict(n=1000, pitch=10e-6, lam=633e-9, z=0.1), 6),
    (dict(n=8192, pitch=10e-6, lam=633e-9, z=0.1), 6),        # N' beyond 8192
    (dict(n=4096, pitch=10e-6, lam=633e-9, z=0.1, prec="f64"), 6),
])
def test_plan_rejects_bad_parameters_before_device_work(P, kw, code):
    x = np.zeros(4)
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(P.make_params(**kw), x, x)
    assert ei.value.code == code


def test_plan_rejects_null_arguments(P):
    from paper_1308_6644_gb300 import nuasm as B
    lib = P.lib()
    h = ctypes.c_void_p()
    params = P.make_params(64, 10e-6, 633e-9, 0.1)
    assert lib.nuasm_plan(None, ctypes.byref(params), 0, None, None, None, None) == 1
    assert lib.nuasm_plan(ctypes.byref(h), None, 0, None, None, None, None) == 1
    assert lib.nuasm_plan(ctypes.byref(h), ctypes.byref(params), 5, None, None, None, None) == 1
    assert lib.nuasm_plan(ctypes.byref(h), ctypes.byref(params), -1, None, None, None, None) == 1
    assert lib.nuasm1_execute(None, None, None, None) == 1
    assert lib.nuasm_destroy(None) == 0
    info = B.PlanInfo()
    assert lib.nuasm_plan_info(None, ctypes.byref(info)) == 1


@pytest.mark.parametrize("o", [0.0, 300e-6, -1.5e-3])
@pytest.mark.parametrize("z", [0.05, -0.2, 0.0])
def test_band_matches_oracle(P, o, z):
    n, pitch, lam = 64, 10e-6, 633e-9
    lo_x, hi_x, lo_y, hi_y = P.nuasm_band(P.make_params(n, pitch, lam, z, ox=o, oy=-o / 2))
    k = O.modes(2 * n)
    for lo, hi, oo in ((lo_x, hi_x, o), (lo_y, hi_y, -o / 2)):
        mask = O.band_mask_1d(n, 2 * n, pitch, lam, z, oo)
        if mask.any():
            assert (lo, hi) == (k[mask].min(), k[mask].max())
            assert mask[(k >= lo) & (k <= hi)].all()     # the kept set is an interval
        else:
            assert lo > hi


def test_explicit_band_matches_oracle(P):
    lo_x, hi_x, lo_y, hi_y = P.nuasm_band(P.make_params(32, 10e-6, 633e-9, 0.01, band=(2.0, -3.5, 10.0, 7.0)))
    k = O.modes(64)
    mx = O.band_mask_1d(32, 64, 10e-6, 633e-9, 0.01, 0.0, 2.0, 10.0)
    my = O.band_mask_1d(32, 64, 10e-6, 633e-9, 0.01, 0.0, -3.5, 7.0)
    assert (lo_x, hi_x) == (k[mx].min(), k[mx].max())
    assert (lo_y, hi_y) == (k[my].min(), k[my].max())


def test_fresnel_band_is_full(P):
    assert P.nuasm_band(P.make_params(32, 10e-6, 633e-9, 1.0, kind="fresnel")) == (-32, 31, -32, 31)


@pytest.mark.parametrize("tol,prec,w", [(0, 0, 7), (0, 1, 13), (1e-6, 0, 7), (1e-3, 0, 4), (1e-11, 1, 12),
                                        (1e-9, 1, 10), (1e-15, 1, 16)])
def test_kernel_width_rule(P, tol, prec, w):
    width, beta = P.nuasm_kernel_shape(tol, prec)
    assert width == w and abs(beta - 2.30 * w) < 1e-12


def test_kernel_shape_rejects_bad_input(P):
    with pytest.raises(P.NuasmError):
        P.nuasm_kernel_shape(0.5, 0)
    with pytest.raises(P.NuasmError):
        P.nuasm_kernel_shape(1e-6, 7)


def test_binding_checks_shapes_and_dtypes(P):
    plan = P.Plan(ctypes.c_void_p(1), P.make_params(16, 10e-6, 633e-9, 0.01), 10)
    plan.handle = None          # never reaches the library
    from paper_1308_6644_gb300 import nuasm as B
    with pytest.raises(ValueError):
        B._expect(np.zeros(9, np.complex64), 10, "complex64", "c")
    with pytest.raises(TypeError):
        B._expect(np.zeros(10, np.complex128), 10, "complex64", "c")
    with pytest.raises(RuntimeError):
        plan.info()


@pytest.mark.parametrize("tol,w", [(1e-3, 7), (1e-5, 11), (1e-6, 13), (1e-7, 15), (1e-10, 21), (1e-12, 25)])
def test_gaussian_kernel_width_rule(P, tol, w):
    width, beta = P.nuasm_kernel_shape(tol, 0, P.KERNEL_GAUSSIAN)
    assert width == w and abs(beta - np.sqrt(2) * np.pi / w) < 1e-12


def test_gaussian_kernel_limits(P):
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_kernel_shape(1e-13, 1, P.KERNEL_GAUSSIAN)
    assert ei.value.code == 6        # 27 taps: beyond the 26 this build runs
    assert P.nuasm_kernel_shape(0.0, 1, P.KERNEL_GAUSSIAN)[0] == 25   # the F64 default tolerance 1e-12
    x = np.zeros(2)
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01, prec="f64", kernel="gaussian", tol=1e-13), x, x)
    assert ei.value.code == 6
    with pytest.raises(P.NuasmError) as ei:   # a 16-cell tile is too small for 21 taps
        P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01, prec="f64", kernel="gaussian", tol=1e-10, tile=16),
                     x, x)
    assert ei.value.code == 6
    bad = P.make_params(32, 10e-6, 633e-9, 0.01)
    bad.kernel = 7
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(bad, x, x)
    assert ei.value.code == 1


def test_batch_and_server_reject_bad_arguments_before_device_work(P):
    lib = P.lib()
    h = ctypes.c_void_p()
    assert lib.nuasm_batch_create(ctypes.byref(h), None, 1, 0) == 1
    items = (P.nuasm.BatchItem * 1)()
    assert lib.nuasm_batch_create(ctypes.byref(h), items, 0, 0) == 1        # empty batch
    assert lib.nuasm_batch_create(ctypes.byref(h), items, 1, 65) == 1       # too many lanes
    assert lib.nuasm_batch_create(ctypes.byref(h), items, 1, 0) == 1        # NULL plan
    assert lib.nuasm_batch_execute(None, None) == 1
    assert lib.nuasm_batch_destroy(None) == 0
    cfg = P.nuasm.ServerConfig(33, 0, 0)
    assert lib.nuasm_server_create(ctypes.byref(h), ctypes.byref(cfg)) == 1  # too many slots
    cfg = P.nuasm.ServerConfig(2, -1, 0)
    assert lib.nuasm_server_create(ctypes.byref(h), ctypes.byref(cfg)) == 1  # bad device
    t = ctypes.c_int64()
    req = P.nuasm.Request()
    assert lib.nuasm_server_submit(None, ctypes.byref(req), ctypes.byref(t)) == 1
    assert lib.nuasm_server_wait(None, 1, 0.0, ctypes.byref(P.nuasm.RequestResult())) == 1
    assert lib.nuasm_server_destroy(None) == 0


@pytest.mark.parametrize("tile", [8, 48, 128, -16])
def test_plan_rejects_unsupported_tiles(P, tile):
    x = np.zeros(2)
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01, tile=tile), x, x)
    assert ei.value.code == 1


@pytest.mark.parametrize("field,value", [("interp_chunk", 32), ("interp_chunk", -1), ("spread_chunk", -2),
                                         ("spread_chunk", 16)])
def test_chunk_knobs_are_validated(P, field, value):
    """interp_chunk is 0 or >= 64 records, spread_chunk -1, 0 or >= 32."""
    x = np.zeros(2)
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01, **{field: value}), x, x)
    assert ei.value.code == 1


def test_bounded_wait_diagnostic_rejects_bad_counts(P):
    lib = P.lib()
    assert lib.nuasm_debug_bounded_wait(0, None) == 1
    assert lib.nuasm_debug_bounded_wait((1 << 24) + 1, None) == 1
    assert lib.nuasm_debug_plan_wait(None, 10, None) == 1


def test_allocation_failure_hook_is_host_only_and_arms_and_disarms(P):
    lib = P.lib()
    n = ctypes.c_int64(-1)
    assert lib.nuasm_debug_live_resources(None) == 1
    assert lib.nuasm_debug_live_resources(ctypes.byref(n)) == 0 and n.value >= 0
    assert lib.nuasm_debug_fail_alloc(-1) == 1
    assert lib.nuasm_debug_fail_alloc(3) == 0
    assert lib.nuasm_debug_fail_alloc(0) == 0
    # validation failures acquire nothing
    before = n.value
    with pytest.raises(P.NuasmError):
        P.nuasm_plan(P.make_params(63, 10e-6, 633e-9, 0.1), np.zeros(2), np.zeros(2))
    assert lib.nuasm_debug_live_resources(ctypes.byref(n)) == 0 and n.value == before


def test_normal_library_has_no_bounds_checks(P):
    """The bounds records exist only in the debug library; the normal one
    answers NUASM_EUNSUPPORTED without touching the device."""
    lib = P.lib()
    hits = ctypes.c_int64(7)
    assert lib.nuasm_debug_bounds(None, None, None, None, 0) == 1
    assert lib.nuasm_debug_bounds(ctypes.byref(hits), None, None, None, 0) == 6 and hits.value == -1
    assert P.nuasm_debug_bounds() is None


def test_debug_library_is_selected_by_environment(tmp_path):
    """NUASM_LIBRARY names the library the binding loads, and a missing one is
    an error at load time (no fallback)."""
    import subprocess
    import sys
    code = ("import paper_1308_6644_gb300 as P\n"
            "print(P.LIB_PATH)\n"
            "try:\n    P.lib()\nexcept RuntimeError as e:\n    print('missing')\n")
    env = dict(os.environ, NUASM_LIBRARY=str(tmp_path / "libnuasm_debug.so"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == [str(tmp_path / "libnuasm_debug.so"), "missing"]


_CTYPE_OF = {"int32_t": "c_int32", "int64_t": "c_int64", "uint64_t": "c_uint64", "double": "c_double",
             "float": "c_float"}


def _header_structs():
    """name -> [(field, C type)] for every typedef'd struct of include/nuasm.h."""
    src = open(os.path.join(ROOT, "include", "nuasm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(const\s+)?([\w]+)(\s*\*)?\s+(.*)", decl)
            ctype, ptr, names = m.group(2), m.group(3), m.group(4)
            for nm in names.split(","):
                nm = nm.strip()
                fields.append((nm.lstrip("*"), "ptr" if (ptr or nm.startswith("*") or ctype.endswith("_t")
                                                            and ctype.startswith("nuasm_plan")) else ctype))
        out[name] = fields
    return out


@pytest.mark.parametrize("c_name,py_name", [
    ("nuasm_params_t", "Params"), ("nuasm_plan_info_t", "PlanInfo"), ("nuasm_batch_item_t", "BatchItem"),
    ("nuasm_server_config_t", "ServerConfig"), ("nuasm_request_t", "Request"),
    ("nuasm_request_result_t", "RequestResult"), ("nuasm_server_stats_t", "ServerStats"),
])
def test_binding_structs_mirror_the_header(c_name, py_name):
    """The ctypes mirrors list the header's fields in the same order with the
    same scalar types (pointers and handles as pointers), so the ABI cannot
    drift silently."""
    from paper_1308_6644_gb300 import nuasm as B
    fields = _header_structs()[c_name]
    py = getattr(B, py_name)._fields_
    # a Python keyword gets a trailing underscore (lambda -> lambda_)
    assert [f for f, _ in fields] == [f.rstrip("_") for f, _ in py], (c_name, fields, py)
    for (fname, ctype), (pname, ptype) in zip(fields, py):
        if ctype == "ptr":
            assert ptype in (ctypes.c_void_p,) or issubclass(ptype, ctypes._Pointer) or ptype is ctypes.c_char_p, \
                (c_name, fname, ptype)
        elif ctype in _CTYPE_OF:
            assert ptype is getattr(ctypes, _CTYPE_OF[ctype]), (c_name, fname, ctype, ptype)
