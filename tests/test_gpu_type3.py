"""NU-ASM_3 / NU-FRE_3 (both planes non-uniform) on the GPU against the oracle
and, at full size, against the Gaussian-beam closed form."""
import numpy as np
import pytest

import oracle as O
from paper_1308_6644_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
TOL = {"f32": 1e-5, "f64": 1e-10}
CDT = {"f32": np.complex64, "f64": np.complex128}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_6644_gb300 as pkg
    return pkg


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run3(P, kind, prec, params, x1, y1, c, x2, y2, w=None):
    import torch
    src = P.nuasm_plan(params, _dev(x1), _dev(y1), None if w is None else _dev(w))
    dst = P.nuasm_plan(params, _dev(x2), _dev(y2))
    try:
        tdt = torch.complex64 if prec == "f32" else torch.complex128
        v = torch.zeros(len(x2), dtype=tdt, device="cuda")
        cc = _dev(np.asarray(c).astype(CDT[prec]))
        (P.nuasm3_execute if kind == "asm" else P.nufresnel3_execute)(src, dst, cc, v)
        torch.cuda.synchronize()
        return v.cpu().numpy()
    finally:
        src.destroy()
        dst.destroy()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["asm", "fresnel"])
@pytest.mark.parametrize("n", [16, 64, 256])
def test_type3_random_points(P, prec, kind, n):
    """Type 3 against the oracle; at N = 256 (N' = 512) the FP64 passes,
    the type-3 row pass included, run in double-float arithmetic."""
    rng = np.random.default_rng(300 + n)
    pitch = 10e-6
    half = 0.5 * n * pitch
    m1, m2 = (600, 500) if n == 64 else (120, 90)
    x1 = WL.clamp_window(rng.uniform(-half, half, m1), n, pitch)
    y1 = WL.clamp_window(rng.uniform(-half, half, m1), n, pitch)
    x2 = WL.clamp_window(rng.uniform(-half, half, m2), n, pitch)
    y2 = WL.clamp_window(rng.uniform(-half, half, m2), n, pitch)
    c = rng.normal(size=m1) + 1j * rng.normal(size=m1)
    kw = dict(lam=633e-9, z=0.03, ox=20e-6, oy=-10e-6)
    params = P.make_params(n, pitch, kw["lam"], kw["z"], ox=kw["ox"], oy=kw["oy"], kind=kind, prec=prec)
    got = run3(P, kind, prec, params, x1, y1, c, x2, y2)
    p = dict(n=n, pitch=pitch, kind=kind, **kw)
    ref = O.diffraction_type3(x1, y1, c.astype(CDT[prec]), x2, y2, p)
    assert O.rel_l2(got, ref) < TOL[prec]


def test_type3_weights_and_graded_destination(P):
    n, pitch = 64, 8e-6
    rng = np.random.default_rng(7)
    wl = WL.nuasm2_graded(seed=31, n=n, pitch=pitch)
    x1, y1 = WL.dense_centre_lattice(rng, n, pitch, 0.4, 16)
    x1, y1 = WL.clamp_window(x1, n, pitch), WL.clamp_window(y1, n, pitch)
    c = WL.random_phasor(rng, len(x1))
    w = rng.uniform(0.5, 1.5, len(x1))
    params = P.make_params(n, pitch, 532e-9, 0.05, ox=100e-6, prec="f64")
    got = run3(P, "asm", "f64", params, x1, y1, c, wl.x, wl.y, w=w)
    ref = O.nuasm3(x1, y1, c, wl.x, wl.y, dict(n=n, pitch=pitch, lam=532e-9, z=0.05, ox=100e-6), weights=w)
    assert O.rel_l2(got, ref) < TOL["f64"]


def test_type3_rejects_mismatched_plans(P):
    import torch
    x = _dev(np.zeros(4))
    a = P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01), x, x)
    b = P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.02), x, x)
    try:
        with pytest.raises(P.NuasmError) as ei:
            P.nuasm3_execute(a, b, torch.zeros(4, dtype=torch.complex64, device="cuda"),
                             torch.zeros(4, dtype=torch.complex64, device="cuda"))
        assert ei.value.code == 1
        with pytest.raises(P.NuasmError):
            P.nufresnel3_execute(a, a, torch.zeros(4, dtype=torch.complex64, device="cuda"),
                                 torch.zeros(4, dtype=torch.complex64, device="cuda"))
    finally:
        a.destroy()
        b.destroy()


def _gaussian_fresnel(x, y, lam, z, w0):
    a, b, zr = 1 / w0 ** 2, np.pi / (lam * z), np.pi * w0 ** 2 / lam
    ph = np.longdouble(z) / np.longdouble(lam)
    ph = float(ph - np.rint(ph))
    return np.exp(2j * np.pi * ph) / (1 + 1j * z / zr) * np.exp(1j * a * b * (x * x + y * y) / (a - 1j * b))


@pytest.mark.parametrize("kind", ["fresnel", "asm"])
def test_type3_full_size_closed_form(P, kind):
    """N = 2048: 4,194,304 warped-lattice sources (Jacobian weights, Gaussian
    beam) to the 4,194,304 clustered destination points.  The beam is wide
    (w0 = 0.5 mm), so the ASM agrees with the paraxial closed form far below
    the tolerance."""
    n, pitch, lam, z, w0 = 2048, 4e-6, 633e-9, 1.0, 0.5e-3
    L = n * pitch
    t = O.lattice(n) * pitch
    phi = t + 0.3 * L / (2 * np.pi) * np.sin(2 * np.pi * t / L)
    dphi = 1 + 0.3 * np.cos(2 * np.pi * t / L)
    ty, tx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x1, y1 = phi[tx].ravel(), phi[ty].ravel()
    wts = (dphi[tx] * dphi[ty]).ravel()
    c = np.exp(-(x1 * x1 + y1 * y1) / w0 ** 2)
    dst = WL.fresnel_clustered(type_=2, n=n)
    params = P.make_params(n, pitch, lam, z, kind=kind)
    got = run3(P, kind, "f32", params, x1, y1, c, dst.x, dst.y, w=wts)
    assert O.rel_l2(got, _gaussian_fresnel(dst.x, dst.y, lam, z, w0)) < TOL["f32"]


# ---------------------------------------------------------------- scaled diffraction (lattice plans)
@pytest.mark.parametrize("kind", ["asm", "fresnel"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_scaled_type2_destination_lattice(P, kind, prec):
    """Uniform 64^2 source at 10 um -> 48^2 destination lattice at 12 um."""
    import torch
    n, pitch, p2, nd = 64, 10e-6, 12e-6, 48
    rng = np.random.default_rng(41)
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    x0 = y0 = -(nd // 2) * p2
    params = P.make_params(n, pitch, 633e-9, 0.02, ox=30e-6, kind=kind, prec=prec)
    plan = P.nuasm_plan_lattice(params, nd, nd, p2, x0, y0)
    try:
        v = torch.zeros(nd * nd, dtype=torch.complex64 if prec == "f32" else torch.complex128, device="cuda")
        src = _dev(u1.astype(CDT[prec]).ravel())
        if kind == "asm":
            P.nuasm2_execute(plan, src, v)
        else:
            P.nufresnel_execute(plan, 2, src, v)
        torch.cuda.synchronize()
        got = v.cpu().numpy()
    finally:
        plan.destroy()
    g = x0 + np.arange(nd) * p2
    gy, gx = np.meshgrid(g, g, indexing="ij")
    p = dict(n=n, pitch=pitch, lam=633e-9, z=0.02, ox=30e-6, kind=kind)
    ref = O.diffraction_type2(u1.astype(CDT[prec]), gx.ravel(), gy.ravel(), p)
    assert O.rel_l2(got, ref) < TOL[prec]


def test_scaled_type1_source_lattice(P):
    """80^2 source lattice at 7 um -> uniform 64^2 plane at 10 um."""
    import torch
    n, pitch, p1, ns = 64, 10e-6, 7e-6, 80
    rng = np.random.default_rng(42)
    c = rng.normal(size=ns * ns) + 1j * rng.normal(size=ns * ns)
    x0 = y0 = -(ns // 2) * p1
    params = P.make_params(n, pitch, 532e-9, 0.03, prec="f64")
    plan = P.nuasm_plan_lattice(params, ns, ns, p1, x0, y0)
    try:
        u2 = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
        P.nuasm1_execute(plan, _dev(c), u2)
        torch.cuda.synchronize()
        got = u2.cpu().numpy().reshape(n, n)
    finally:
        plan.destroy()
    g = x0 + np.arange(ns) * p1
    gy, gx = np.meshgrid(g, g, indexing="ij")
    ref = O.nuasm1(gx.ravel(), gy.ravel(), c, dict(n=n, pitch=pitch, lam=532e-9, z=0.03))
    assert O.rel_l2(got, ref) < TOL["f64"]


@pytest.mark.parametrize("prec,tile,nx,ny,p2", [("f32", 0, 300, 260, 8e-6), ("f64", 16, 70, 90, 7e-6),
                                                 ("f32", 32, 1000, 1000, 2.5e-6)])
def test_lattice_plan_bins_like_the_sorted_path(P, prec, tile, nx, ny, p2):
    """The lattice plan's no-sort binning gives the records the counting sort
    of the same points gives: equal record counts, type 2 equal (each output
    depends on its own record only; bit for bit in FP32, to the last bits of
    the fractions in FP64, whose lattice coordinates x0 + i p2 are formed on
    the device with one rounding) and type 1 to rounding (the shared-memory
    sums run in another order)."""
    import torch
    n, pitch = 256, 10e-6
    x0, y0 = -0.5 * nx * p2 + 0.3e-6, -0.5 * ny * p2 - 1.1e-6
    params = P.make_params(n, pitch, 633e-9, 0.05, prec=prec, tile=tile)
    gx = x0 + np.arange(nx) * p2
    gy = y0 + np.arange(ny) * p2
    yy, xx = np.meshgrid(gy, gx, indexing="ij")
    lat = P.nuasm_plan_lattice(params, nx, ny, p2, x0, y0)
    pts = P.nuasm_plan(params, _dev(xx.ravel()), _dev(yy.ravel()))
    try:
        assert P.nuasm_plan_info(lat)["records"] == P.nuasm_plan_info(pts)["records"]
        rng = np.random.default_rng(44)
        ct = CDT[prec]
        tdt = torch.complex64 if prec == "f32" else torch.complex128
        u1 = _dev((rng.normal(size=n * n) + 1j * rng.normal(size=n * n)).astype(ct))
        va, vb = (torch.zeros(nx * ny, dtype=tdt, device="cuda") for _ in range(2))
        P.nuasm2_execute(lat, u1, va)
        P.nuasm2_execute(pts, u1, vb)
        c = _dev((rng.normal(size=nx * ny) + 1j * rng.normal(size=nx * ny)).astype(ct))
        ua, ub = (torch.zeros(n * n, dtype=tdt, device="cuda") for _ in range(2))
        P.nuasm1_execute(lat, c, ua)
        P.nuasm1_execute(pts, c, ub)
        torch.cuda.synchronize()
        if prec == "f32":
            assert torch.equal(va, vb)
        else:
            assert O.rel_l2(va.cpu().numpy(), vb.cpu().numpy()) < 1e-13
        assert O.rel_l2(ua.cpu().numpy(), ub.cpu().numpy()) < (1e-6 if prec == "f32" else 1e-13)
    finally:
        lat.destroy()
        pts.destroy()


def test_lattice_outside_window_is_rejected(P):
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan_lattice(P.make_params(32, 10e-6, 633e-9, 0.01), 40, 40, 10e-6, -200e-6, -200e-6)
    assert ei.value.code == 2
