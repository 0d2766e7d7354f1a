"""Full-size parity: the benchmark workload and the large NU-FRE workloads in
the launch configuration bench.py uses, checked on outputs the oracle can
compute one by one (sampled points), on sparse inputs, through the adjoint
identity between the type-1 and type-2 paths, and against closed forms that
hold at any size.  Tolerances: rel-L2 1e-5 (FP32 with FP64-derived phase),
1e-10 (FP64), and beside every rel-L2 an element-wise bound
max |got - ref| <= 10 tol ||ref||_2 / sqrt(n), so that one bad tile edge or
halo row cannot hide in the norm of millions of outputs."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1308_6644_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-5
TOL64 = 1e-10


def assert_close(got, ref, tol):
    """rel-L2 <= tol and every element within 10 tol of the RMS of ref."""
    got, ref = np.asarray(got).ravel(), np.asarray(ref).ravel()
    err = O.rel_l2(got, ref)
    assert err < tol, err
    bound = 10.0 * tol * np.linalg.norm(ref) / np.sqrt(ref.size)
    worst = np.max(np.abs(got - ref))
    assert worst <= bound, (worst, bound, int(np.argmax(np.abs(got - ref))))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1308_6644_gb300 as pkg
    return pkg


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solve(P, w, type_, values, weights=None, kind=None, prec="f32", z=None, tol=0.0):
    import torch
    kind = kind or w.kind
    cdt, tdt = (np.complex128, torch.complex128) if prec == "f64" else (np.complex64, torch.complex64)
    params = P.make_params(w.n, w.pitch, w.lam, w.z if z is None else z, ox=w.ox, oy=w.oy, kind=kind, prec=prec,
                           tol=tol)
    plan = P.nuasm_plan(params, _dev(w.x), _dev(w.y), None if weights is None else _dev(weights))
    try:
        src = _dev(np.asarray(values).astype(cdt).reshape(-1))
        out = torch.zeros(w.n * w.n if type_ == 1 else w.m, dtype=tdt, device="cuda")
        if kind == "asm":
            (P.nuasm1_execute if type_ == 1 else P.nuasm2_execute)(plan, src, out)
        else:
            P.nufresnel_execute(plan, type_, src, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        plan.destroy()


def _transfer(w, kind):
    n, n_pad = w.n, 2 * w.n
    if kind == "asm":
        return O.asm_transfer(n, n_pad, w.pitch, w.lam, w.z, w.ox, w.oy)
    return O.fresnel_transfer(n_pad, w.pitch, w.lam, w.z, w.ox, w.oy)


@functools.lru_cache(maxsize=2)
def _fresnel_clustered(type_):
    return WL.fresnel_clustered(type_=type_, n=2048)


@functools.lru_cache(maxsize=2)
def _clustered_transfer():
    return _transfer(_fresnel_clustered(1), "fresnel")


@functools.lru_cache(maxsize=2)
def _clustered_spectrum(rounded_to_f32):
    """G(k) H(k) / N'^2 of the C3 type-2 source (rounded to complex64 first
    when the GPU input is complex64)."""
    w = _fresnel_clustered(2)
    u1 = np.asarray(w.values).astype(np.complex64 if rounded_to_f32 else np.complex128).astype(np.complex128)
    return O.uniform_dft(u1, 2 * w.n) * _clustered_transfer() / float(2 * w.n) ** 2


def _oracle_type2_sampled(w, idx, kind):
    n_pad = 2 * w.n
    u1 = w.values.astype(np.complex64).astype(np.complex128)
    g = O.uniform_dft(u1, n_pad)
    h = _transfer(w, kind)
    return O.nudft_type2(g * h / float(n_pad) ** 2, w.x[idx] / w.pitch, w.y[idx] / w.pitch, n_pad)


def gaussian_fresnel(x, y, lam, z, w0):
    """Fresnel propagation of exp(-|x|^2/w0^2) (completing the square)."""
    a, b, zr = 1 / w0 ** 2, np.pi / (lam * z), np.pi * w0 ** 2 / lam
    ph = np.longdouble(z) / np.longdouble(lam)
    ph = float(ph - np.rint(ph))
    return np.exp(2j * np.pi * ph) / (1 + 1j * z / zr) * np.exp(1j * a * b * (x * x + y * y) / (a - 1j * b))


def test_nuasm2_benchmark_workload_sampled(P):
    """NU-ASM_2, N = 1024, M = 1,048,576 graded points (the bench workload):
    4096 sampled points against the direct NUDFT oracle."""
    w = WL.nuasm2_graded(seed=1002, n=1024, pitch=8e-6)
    got = _solve(P, w, 2, w.values)
    idx = np.sort(np.random.default_rng(11).choice(w.m, 4096, replace=False))
    ref = _oracle_type2_sampled(w, idx, "asm")
    assert_close(got[idx], ref, TOL)


def test_nufresnel2_clustered_full_size(P):
    """NU-FRE_2, N = 2048, M = 4,194,304 clustered points, Gaussian-beam
    source: sampled points against the oracle, every point against the
    closed form."""
    w = _fresnel_clustered(2)
    got = _solve(P, w, 2, w.values)
    want = gaussian_fresnel(w.x + w.ox, w.y + w.oy, w.lam, w.z, w.extra["w0"])
    assert_close(got, want, TOL)
    idx = np.sort(np.random.default_rng(12).choice(w.m, 2048, replace=False))
    ref = O.nudft_type2(_clustered_spectrum(True), w.x[idx] / w.pitch, w.y[idx] / w.pitch, 2 * w.n)
    assert_close(got[idx], ref, TOL)


@pytest.mark.parametrize("plan_tol", [0.0, TOL64])
def test_nufresnel2_clustered_full_size_fp64(P, plan_tol):
    """NU-FRE_2 in FP64 mode (complex128 data, double-float gridding; ES kernel at the FP64
    default 1e-12, 13 taps, and at a plan tolerance of 1e-10, 11 taps) on the
    same 4,194,304 clustered points: 2048 sampled points against the oracle
    at rel-L2 1e-10, and every point against the Gaussian-beam closed form at
    the accuracy of the sampled Fresnel transform itself."""
    w = _fresnel_clustered(2)
    got = _solve(P, w, 2, w.values, prec="f64", tol=plan_tol)
    idx = np.sort(np.random.default_rng(14).choice(w.m, 2048, replace=False))
    ref = O.nudft_type2(_clustered_spectrum(False), w.x[idx] / w.pitch, w.y[idx] / w.pitch, 2 * w.n)
    assert_close(got[idx], ref, TOL64)
    want = gaussian_fresnel(w.x + w.ox, w.y + w.oy, w.lam, w.z, w.extra["w0"])
    assert_close(got, want, TOL)


def test_nufresnel1_full_size_warped_lattice_closed_form(P):
    """NU-FRE_1 at N = 2048 with all 4,194,304 source points non-zero: a
    smoothly warped lattice with Jacobian weights is a spectrally accurate
    quadrature, so the output is the Gaussian-beam closed form."""
    n, pitch, lam, z, w0 = 2048, 4e-6, 633e-9, 1.0, 0.5e-3
    L = n * pitch
    t = O.lattice(n) * pitch
    phi = t + 0.3 * L / (2 * np.pi) * np.sin(2 * np.pi * t / L)
    dphi = 1 + 0.3 * np.cos(2 * np.pi * t / L)
    ty, tx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x, y = phi[tx].ravel(), phi[ty].ravel()
    wts = (dphi[tx] * dphi[ty]).ravel()
    c = np.exp(-(x * x + y * y) / w0 ** 2)
    wl = WL.Workload("warped", "fresnel", 1, n, pitch, lam, z, x=x, y=y, values=c)
    got = _solve(P, wl, 1, c, weights=wts).reshape(n, n)
    g = O.lattice(n) * pitch
    gy, gx = np.meshgrid(g, g, indexing="ij")
    assert_close(got, gaussian_fresnel(gx, gy, lam, z, w0), TOL)


@pytest.mark.parametrize("prec,tol,plan_tol", [("f32", TOL, 0.0), ("f64", TOL64, 0.0), ("f64", TOL64, TOL64)])
def test_nufresnel1_clustered_full_size_sparse_sources(P, prec, tol, plan_tol):
    """NU-FRE_1 on the 4,194,304 clustered points with 4096 non-zero sources
    (drawn from the point set, so ~3/4 in the clusters): every output pixel
    against the oracle (the full launch configuration with an oracle cost of
    4096 points), in FP32 and in FP64 mode (at the default plan tolerance and
    at 1e-10)."""
    w = _fresnel_clustered(1)
    rng = np.random.default_rng(13)
    c = np.zeros(w.m, np.complex128)
    nz = np.sort(rng.choice(w.m, 4096, replace=False))
    c[nz] = rng.normal(size=nz.size) + 1j * rng.normal(size=nz.size)
    got = _solve(P, w, 1, c, prec=prec, tol=plan_tol).reshape(w.n, w.n)
    p = dict(n=w.n, pitch=w.pitch, lam=w.lam, z=w.z, kind="fresnel")
    cin = c[nz].astype(np.complex64) if prec == "f32" else c[nz]
    ref = O.diffraction_type1(w.x[nz], w.y[nz], cin, p, h=_clustered_transfer())
    assert_close(got, ref, tol)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-6), ("f64", 1e-11)])
def test_nufresnel1_clustered_full_size_all_sources_adjoint(P, prec, tol):
    """NU-FRE_1 with all 4,194,304 clustered sources non-zero (random
    phasors: the integer-batch spreading at full cluster density) against the
    independent type-2 path through the adjoint identity
    <NU-FRE_1^(z) c, v> = <c, NU-FRE_2^(-z) v>: with o = 0 the Fresnel
    transfer function of -z is the complex conjugate of that of z (the
    sampled impulse response depends on |m pitch|^2 only), so the identity is
    exact up to rounding.  FP32 and FP64 mode; the bound is tol ||u2|| ||v||."""
    import torch
    w = _fresnel_clustered(1)
    assert w.ox == 0 and w.oy == 0
    cdt = np.complex128 if prec == "f64" else np.complex64
    rng = np.random.default_rng(78)
    c = np.exp(2j * np.pi * rng.uniform(size=w.m)).astype(cdt)
    v = (rng.normal(size=w.n * w.n) + 1j * rng.normal(size=w.n * w.n)).astype(cdt)
    u2 = _solve(P, w, 1, c, prec=prec)
    vb = _solve(P, w, 2, v, prec=prec, z=-w.z)
    lhs = np.vdot(u2.astype(np.complex128), v.astype(np.complex128))
    rhs = np.vdot(c.astype(np.complex128), vb.astype(np.complex128))
    scale = np.linalg.norm(u2) * np.linalg.norm(v)
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("plane", [0, 1, 2, 3])
def test_mixed_planes(P, plane):
    """Planes of the mixed batch (N up to 2048, 0.25-4 N^2 points): type 2 on
    sampled points, type 1 with 128 non-zero sources, against the oracle."""
    w = WL.mixed_plane(1004, plane)
    rng = np.random.default_rng(100 + plane)
    if w.type == 2:
        got = _solve(P, w, 2, w.values)
        idx = np.sort(rng.choice(w.m, min(w.m, 1024), replace=False))
        assert_close(got[idx], _oracle_type2_sampled(w, idx, "asm"), TOL)
    else:
        c = np.zeros(w.m, np.complex128)
        nz = rng.choice(w.m, min(w.m, 128), replace=False)
        c[nz] = w.values[nz]
        got = _solve(P, w, 1, c).reshape(w.n, w.n)
        p = dict(n=w.n, pitch=w.pitch, lam=w.lam, z=w.z)
        assert_close(got, O.nuasm1(w.x[nz], w.y[nz], c[nz].astype(np.complex64), p), TOL)


def test_asm_n4096_exact_helmholtz_solution(P):
    """N = 4096 (N' = 8192: the row passes run their two transforms in turn
    and read the phase-factor table from L2): NU-ASM_2 of a complex-source-
    point beam, an exact solution of the Helmholtz equation, against that
    solution at 200,000 random points, 2 mm away (a non-separable phase of
    ~50 cycles at the band edge), through a plan (tabulated factor, FP64) and
    through the server (factor evaluated per mode in double-float FP32)."""
    n, pitch, lam, w0, z, m = 4096, 0.2e-6, 0.5e-6, 20e-6, 2e-3, 200_000
    k, b = 2 * np.pi / lam, np.pi * w0 ** 2 / lam

    def csp(x, y, zz):
        R = -1j * np.sqrt(b * b - (x * x + y * y) + 0j) if zz == 0 else np.sqrt(x * x + y * y + (zz - 1j * b) ** 2)
        return np.exp(1j * k * (R + 1j * b)) / R

    g = (np.arange(n) - n // 2) * pitch
    gx, gy = np.meshgrid(g, g)
    u1 = csp(gx, gy, 0.0)
    scale = np.abs(u1).max()
    u1 = (u1 / scale).astype(np.complex64)
    rng = np.random.default_rng(4096)
    half = 0.25 * n * pitch   # the beam (width ~25 um at z) sits well inside
    x = rng.uniform(-half, half, m)
    y = rng.uniform(-half, half, m)
    want = csp(x, y, z) / scale
    params = P.make_params(n, pitch, lam, z)
    import torch
    plan = P.nuasm_plan(params, _dev(x), _dev(y))
    try:
        assert plan.info()["phase_table_bytes"] > 0
        v = torch.zeros(m, dtype=torch.complex64, device="cuda")
        P.nuasm2_execute(plan, _dev(u1.reshape(-1)), v)
        torch.cuda.synchronize()
        got = v.cpu().numpy()
    finally:
        plan.destroy()
    assert_close(got, want, TOL)
    srv = P.nuasm_server_create(slots=1)
    try:
        served = np.zeros(m, np.complex64)
        t = P.nuasm_server_submit(srv, params, 2, x, y, u1.reshape(-1), served, points_id=0)
        assert P.nuasm_server_wait(srv, t, 120.0)["status"] == 0
    finally:
        srv.destroy()
    assert_close(served, want, TOL)


def test_adjoint_identity_at_the_benchmark_size(P):
    """<NU-ASM_1 c, v> = <c, NU-ASM_2^(-z,-o) v> on the benchmark geometry
    (N = 1024, 1,048,576 graded points, off-axis): the type-1 path (batched
    integer spreading, the row pass with T1x and E) against the type-2 path
    (interpolation, the Tx-folded table) at full size, where the oracle
    cannot run."""
    import torch
    w = WL.nuasm2_graded(seed=1002, n=1024, pitch=8e-6)
    rng = np.random.default_rng(77)
    c = (rng.normal(size=w.m) + 1j * rng.normal(size=w.m)).astype(np.complex64)
    v = (rng.normal(size=w.n * w.n) + 1j * rng.normal(size=w.n * w.n)).astype(np.complex64)
    fwd = P.make_params(w.n, w.pitch, w.lam, w.z, ox=w.ox, oy=w.oy)
    back = P.make_params(w.n, w.pitch, w.lam, -w.z, ox=-w.ox, oy=-w.oy)
    u2 = torch.zeros(w.n * w.n, dtype=torch.complex64, device="cuda")
    vb = torch.zeros(w.m, dtype=torch.complex64, device="cuda")
    pf = P.nuasm_plan(fwd, _dev(w.x), _dev(w.y))
    pb = P.nuasm_plan(back, _dev(w.x), _dev(w.y))
    try:
        P.nuasm1_execute(pf, _dev(c), u2)
        P.nuasm2_execute(pb, _dev(v), vb)
        torch.cuda.synchronize()
    finally:
        pf.destroy()
        pb.destroy()
    lhs = np.vdot(u2.cpu().numpy().astype(np.complex128), v.astype(np.complex128))
    rhs = np.vdot(c.astype(np.complex128), vb.cpu().numpy().astype(np.complex128))
    scale = np.linalg.norm(u2.cpu().numpy()) * np.linalg.norm(v)
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs, scale)   # |lhs| ~ 1e-3 scale (random phases)


def test_unaligned_user_arrays_at_n2048(P):
    """At N' = 4096 the column passes read the type-2 input and write the
    type-1 output through TMA tensor maps, which need 16-byte aligned
    arrays; a caller's array 8 bytes off that alignment (a view one complex64
    element into a buffer) takes the per-thread path of the same pass and
    gives the same result as an aligned one."""
    import torch
    rng = np.random.default_rng(45)
    n, pitch, m = 2048, 4e-6, 20000
    h = 0.5 * n * pitch * (1 - 1e-9)
    x, y = rng.uniform(-h, h, m), rng.uniform(-h, h, m)
    params = P.make_params(n, pitch, 633e-9, 0.5, kind="fresnel")
    plan = P.nuasm_plan(params, _dev(x), _dev(y))
    try:
        u1 = (rng.normal(size=n * n) + 1j * rng.normal(size=n * n)).astype(np.complex64)
        c = (rng.normal(size=m) + 1j * rng.normal(size=m)).astype(np.complex64)
        a_in = _dev(u1)
        b_buf = torch.zeros(n * n + 1, dtype=torch.complex64, device="cuda")
        b_in = b_buf[1:]
        b_in.copy_(a_in)
        assert b_in.data_ptr() % 16 == 8
        va, vb = (torch.zeros(m, dtype=torch.complex64, device="cuda") for _ in range(2))
        P.nufresnel_execute(plan, 2, a_in, va)
        P.nufresnel_execute(plan, 2, b_in, vb)
        ua = torch.zeros(n * n, dtype=torch.complex64, device="cuda")
        ub_buf = torch.zeros(n * n + 1, dtype=torch.complex64, device="cuda")
        ub = ub_buf[1:]
        P.nufresnel_execute(plan, 1, _dev(c), ua)
        P.nufresnel_execute(plan, 1, _dev(c), ub)
        torch.cuda.synchronize()
        assert O.rel_l2(vb.cpu().numpy(), va.cpu().numpy()) < 1e-6
        assert O.rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) < 1e-6
        assert float(ub_buf[0].abs()) == 0.0   # nothing written before the view
    finally:
        plan.destroy()
