"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances (relative L2 over all outputs or the stated sample):
* F32 plans (complex64 data, FP64-derived phase): 1e-5;
* F64 plans (complex128, default NUFFT tolerance 1e-12): 1e-10.
"""
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


def _t(a, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def run_gpu(P, kind, type_, prec, n, pitch, lam, z, x, y, values, ox=0.0, oy=0.0, w=None, n_pad=0,
            band=None, tol=0.0, host=False, kernel="es", tile=0, interp_chunk=0, spread_chunk=0):
    """One plan + one execute; returns the output as a numpy array."""
    import torch
    params = P.make_params(n, pitch, lam, z, ox=ox, oy=oy, kind=kind, prec=prec, tol=tol,
                           n_pad=n_pad, band=band, kernel=kernel, tile=tile, interp_chunk=interp_chunk,
                           spread_chunk=spread_chunk)
    cdt = CDT[prec]
    tdt = torch.complex64 if prec == "f32" else torch.complex128
    if host:
        xs, ys = np.ascontiguousarray(x, np.float64), np.ascontiguousarray(y, np.float64)
        ws = None if w is None else np.ascontiguousarray(w, np.float64)
    else:
        xs, ys = _t(np.asarray(x, np.float64)), _t(np.asarray(y, np.float64))
        ws = None if w is None else _t(np.asarray(w, np.float64))
    plan = P.nuasm_plan(params, xs, ys, ws)
    try:
        inp = np.ascontiguousarray(np.asarray(values).astype(cdt).reshape(-1))
        if type_ == 1:
            out = np.zeros(n * n, cdt) if host else torch.zeros(n * n, dtype=tdt, device="cuda")
        else:
            out = np.zeros(len(x), cdt) if host else torch.zeros(len(x), dtype=tdt, device="cuda")
        src = inp if host else _t(inp)
        if kind == "asm":
            (P.nuasm1_execute if type_ == 1 else P.nuasm2_execute)(plan, src, out)
        else:
            P.nufresnel_execute(plan, type_, src, out)
        torch.cuda.synchronize()
        res = out if host else out.cpu().numpy()
    finally:
        plan.destroy()
    return res.reshape(n, n) if type_ == 1 else res


def run_oracle(kind, type_, n, pitch, lam, z, x, y, values, ox=0.0, oy=0.0, w=None, n_pad=0, band=None,
               prec="f32"):
    p = dict(n=n, n_pad=n_pad or 2 * n, pitch=pitch, lam=lam, z=z, ox=ox, oy=oy, kind=kind, band=band)
    vals = np.asarray(values).astype(CDT[prec]).astype(np.complex128)   # the inputs the GPU saw
    if type_ == 1:
        return O.diffraction_type1(x, y, vals.reshape(-1), p, weights=w)
    return O.diffraction_type2(vals.reshape(n, n), x, y, p)


def random_case(seed, n, m, pitch=10e-6, type_=1):
    rng = np.random.default_rng(seed)
    half = 0.5 * n * pitch
    x = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    y = WL.clamp_window(rng.uniform(-half, half, m), n, pitch)
    if type_ == 1:
        vals = rng.normal(size=m) + 1j * rng.normal(size=m)
    else:
        vals = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return x, y, vals


# ---------------------------------------------------------------- small end-to-end parity
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["asm", "fresnel"])
@pytest.mark.parametrize("type_", [1, 2])
@pytest.mark.parametrize("n", [16, 64])
def test_random_points_parity(P, prec, kind, type_, n):
    m = 700 if n == 64 else 150
    x, y, vals = random_case(11 + n + type_, n, m, type_=type_)
    kw = dict(pitch=10e-6, lam=633e-9, z=0.03, ox=25e-6, oy=-12e-6)
    got = run_gpu(P, kind, type_, prec, n, x=x, y=y, values=vals, **kw)
    ref = run_oracle(kind, type_, n, x=x, y=y, values=vals, prec=prec, **kw)
    assert O.rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nuasm1_dense_core_config(P, prec):
    """NU-ASM_1, 64 x 64 jittered source with a 2x denser core (M = 4864),
    10 um pitch, 633 nm, z = 5 cm, N' = 128, auto band."""
    w = WL.nuasm1_small()
    got = run_gpu(P, "asm", 1, prec, w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values)
    ref = run_oracle("asm", 1, w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values, prec=prec)
    assert O.rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nuasm2_graded_small(P, prec):
    """NU-ASM_2 with the graded destination (4 -> 16 um) and off-axis offset at N = 128."""
    w = WL.nuasm2_graded(n=128)
    got = run_gpu(P, "asm", 2, prec, w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values, ox=w.ox, oy=w.oy)
    ref = run_oracle("asm", 2, w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values, ox=w.ox, oy=w.oy, prec=prec)
    assert O.rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("type_", [1, 2])
def test_fresnel_clustered_small(P, type_):
    """NU-FRE with clustered points and a Gaussian-beam input at N = 128."""
    w = WL.fresnel_clustered(type_=type_, n=128, m=6000)
    got = run_gpu(P, "fresnel", type_, "f32", w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values)
    ref = run_oracle("fresnel", type_, w.n, w.pitch, w.lam, w.z, w.x, w.y, w.values)
    assert O.rel_l2(got, ref) < TOL["f32"]


# ---------------------------------------------------------------- options and edge cases
def test_weights_type1(P):
    x, y, vals = random_case(21, 32, 400)
    wts = np.random.default_rng(3).uniform(0.5, 2.0, len(x))
    kw = dict(pitch=10e-6, lam=633e-9, z=0.02)
    got = run_gpu(P, "asm", 1, "f64", 32, x=x, y=y, values=vals, w=wts, **kw)
    ref = run_oracle("asm", 1, 32, x=x, y=y, values=vals, w=wts, prec="f64", **kw)
    assert O.rel_l2(got, ref) < TOL["f64"]


@pytest.mark.parametrize("type_", [1, 2])
def test_explicit_band_and_larger_padding(P, type_):
    x, y, vals = random_case(22 + type_, 32, 300, type_=type_)
    kw = dict(pitch=10e-6, lam=633e-9, z=0.04, ox=30e-6, n_pad=128, band=(3.0, -2.0, 40.0, 30.0))
    got = run_gpu(P, "asm", type_, "f64", 32, x=x, y=y, values=vals, **kw)
    ref = run_oracle("asm", type_, 32, x=x, y=y, values=vals, prec="f64", **kw)
    assert O.rel_l2(got, ref) < TOL["f64"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("type_", [1, 2])
def test_tabulated_phase_factor_large_phase(P, prec, type_):
    """Eq. 4 with the full mode set kept (explicit band) and a non-separable
    phase rc Q(s)^2 of about 1.6 cycles at the corner modes: the plan's FP64
    table of that factor against the oracle, and (F32, type 2) against the
    no-allocation path, which evaluates the factor per mode in double-float
    FP32."""
    import torch
    n, m = 64, 900
    x, y, vals = random_case(41 + type_, n, m, pitch=4e-6, type_=type_)
    kw = dict(pitch=4e-6, lam=633e-9, z=0.05, ox=20e-6, oy=-8e-6, band=(0.0, 0.0, 128.0, 128.0))
    got = run_gpu(P, "asm", type_, prec, n, x=x, y=y, values=vals, **kw)
    ref = run_oracle("asm", type_, n, x=x, y=y, values=vals, prec=prec, **kw)
    assert O.rel_l2(got, ref) < TOL[prec]
    params = P.make_params(n, kw["pitch"], kw["lam"], kw["z"], ox=kw["ox"], oy=kw["oy"], band=kw["band"], prec=prec)
    plan = P.nuasm_plan(params, _t(x), _t(y))
    try:
        half = 64   # E over |k| in [0, 64]; FP32 plans add type 2's Tx-folded rows of N' = 128 entries
        want = (half + 1) * (half + 2) * 16 if prec == "f64" else ((half + 1) * (half + 2) + (half + 1) * 128) * 8
        assert plan.info()["phase_table_bytes"] == want
    finally:
        plan.destroy()
    if prec == "f32" and type_ == 2:
        v = torch.zeros(m, dtype=torch.complex64, device="cuda")
        P.nuasm2_solve_noalloc(params, _t(x), _t(y), _t(np.asarray(vals, np.complex64).reshape(-1)), v)
        torch.cuda.synchronize()
        per_mode = v.cpu().numpy()
        assert O.rel_l2(per_mode, ref) < TOL["f32"]
        assert O.rel_l2(per_mode, got) < TOL["f32"]


def test_phase_table_only_where_the_phase_is_not_separable(P):
    x, y, _ = random_case(5, 32, 100)
    for kind, z, expect in (("asm", 0.03, True), ("asm", 0.0, False), ("fresnel", 0.03, False)):
        params = P.make_params(32, 10e-6, 633e-9, z, kind=kind)
        plan = P.nuasm_plan(params, _t(x), _t(y))
        try:
            info = plan.info()
            assert (info["phase_table_bytes"] > 0) == expect
            assert info["device_bytes"] > info["phase_table_bytes"]
        finally:
            plan.destroy()


def test_bank_skew_follows_the_point_distribution(P):
    """A graded lattice (points every few fine-grid columns, as at the edge of
    the NU-ASM_2 benchmark plane) gets a skewed tile layout, uniformly random
    points the plain one (or, with a skew per tile, any candidate); type 2
    gives the same bits whatever the layout (each point's taps are summed in a
    fixed order) and agrees with the oracle."""
    wl = WL.nuasm2_graded(seed=7, n=256, pitch=8e-6)
    xr, yr, _ = random_case(8, 256, wl.m, pitch=8e-6)
    params = P.make_params(256, 8e-6, 532e-9, 0.05, tile=64)
    skews = []
    for x, y in ((wl.x, wl.y), (xr, yr)):
        plan = P.nuasm_plan(params, _t(x), _t(y))
        try:
            skews.append(plan.info()["bank_skew"])
        finally:
            plan.destroy()
    assert skews[0] != 0 and skews[1] in (0, 2, 4, 6, 8)
    u1 = np.random.default_rng(9).normal(size=(256, 256)) + 0j
    kw = dict(pitch=8e-6, lam=532e-9, z=0.05)
    got = run_gpu(P, "asm", 2, "f32", 256, x=wl.x, y=wl.y, values=u1, tile=64, **kw)
    idx = np.random.default_rng(10).choice(wl.m, 4000, replace=False)
    ref = run_oracle("asm", 2, 256, x=wl.x[idx], y=wl.y[idx], values=u1, **kw)
    assert O.rel_l2(got[idx], ref) < TOL["f32"]


def test_window_edges_and_single_tile(P):
    """Points exactly on the lower window edge, just inside the upper edge and
    all crowded into one tile."""
    n, pitch = 64, 10e-6
    half = 0.5 * n * pitch
    edge = np.array([-half, half * (1 - 1e-12), -half, 0.0, half * (1 - 1e-12)])
    rng = np.random.default_rng(5)
    cx = rng.uniform(-3e-6, 3e-6, 200)
    x = np.concatenate([edge, cx])
    y = np.concatenate([np.roll(edge, 2), rng.uniform(-3e-6, 3e-6, 200)])
    vals = rng.normal(size=len(x)) + 1j * rng.normal(size=len(x))
    kw = dict(pitch=pitch, lam=633e-9, z=0.01)
    for t in (1, 2):
        v = vals if t == 1 else rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        got = run_gpu(P, "asm", t, "f64", n, x=x, y=y, values=v, **kw)
        ref = run_oracle("asm", t, n, x=x, y=y, values=v, prec="f64", **kw)
        assert O.rel_l2(got, ref) < TOL["f64"]


def test_zero_points(P):
    import torch
    params = P.make_params(32, 10e-6, 633e-9, 0.02)
    plan = P.nuasm_plan(params, None, None)
    try:
        u2 = torch.full((32 * 32,), 1 + 1j, dtype=torch.complex64, device="cuda")
        P.nuasm1_execute(plan, None, u2)
        u1 = torch.ones(32 * 32, dtype=torch.complex64, device="cuda")
        P.nuasm2_execute(plan, u1, None)
        torch.cuda.synchronize()
        assert torch.count_nonzero(u2).item() == 0
    finally:
        plan.destroy()


def test_out_of_window_point_is_rejected(P):
    n, pitch = 32, 10e-6
    x = np.array([0.0, 0.5 * n * pitch])      # x / pitch == N/2 is outside [-N/2, N/2)
    y = np.zeros(2)
    with pytest.raises(P.NuasmError) as ei:
        P.nuasm_plan(P.make_params(n, pitch, 633e-9, 0.01), _t(x), _t(y))
    assert ei.value.code == 2


def test_kind_mismatch_is_rejected(P):
    import torch
    x, y, _ = random_case(1, 32, 10)
    plan = P.nuasm_plan(P.make_params(32, 10e-6, 633e-9, 0.01, kind="fresnel"), _t(x), _t(y))
    try:
        with pytest.raises(P.NuasmError):
            P.nuasm1_execute(plan, torch.zeros(10, dtype=torch.complex64, device="cuda"),
                             torch.zeros(1024, dtype=torch.complex64, device="cuda"))
    finally:
        plan.destroy()


@pytest.mark.parametrize("type_", [1, 2])
def test_host_buffers_match_device_buffers(P, type_):
    x, y, vals = random_case(31, 64, 500, type_=type_)
    kw = dict(pitch=10e-6, lam=633e-9, z=0.02)
    a = run_gpu(P, "asm", type_, "f32", 64, x=x, y=y, values=vals, host=True, **kw)
    b = run_gpu(P, "asm", type_, "f32", 64, x=x, y=y, values=vals, host=False, **kw)
    assert O.rel_l2(a, b) < 1e-6


def test_type2_is_deterministic(P):
    x, y, vals = random_case(41, 64, 2000, type_=2)
    kw = dict(pitch=10e-6, lam=633e-9, z=0.02)
    a = run_gpu(P, "asm", 2, "f32", 64, x=x, y=y, values=vals, **kw)
    b = run_gpu(P, "asm", 2, "f32", 64, x=x, y=y, values=vals, **kw)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_fp32_type1_dense_random_phase_cluster(P, tile):
    """20000 random-phase points within a few fine-grid cells (hundreds per
    cell): every shared-memory accumulation (warp-private copies for 16 and
    32, batched integer sums for 64) must keep the FP32 tolerance where the
    cell sums cancel far below the sum of magnitudes, and two runs agree to
    rounding (atomics add in varying order)."""
    rng = np.random.default_rng(43)
    n, pitch, m = 64, 10e-6, 20000
    x = WL.clamp_window(rng.normal(0, 20e-6, m), n, pitch)
    y = WL.clamp_window(rng.normal(0, 20e-6, m), n, pitch)
    c = rng.normal(size=m) + 1j * rng.normal(size=m)
    kw = dict(pitch=pitch, lam=633e-9, z=0.02, tile=tile)
    a = run_gpu(P, "asm", 1, "f32", n, x=x, y=y, values=c, **kw)
    b = run_gpu(P, "asm", 1, "f32", n, x=x, y=y, values=c, **kw)
    del kw["tile"]
    ref = run_oracle("asm", 1, n, x=x, y=y, values=c, **kw)
    assert O.rel_l2(a, ref) < TOL["f32"] and O.rel_l2(b, ref) < TOL["f32"]
    assert O.rel_l2(a, b) < 1e-6


def test_fp32_type1_large_tiles_dynamic_range_and_non_finite(P):
    """Batched integer spreading (tile 64): values spanning eight decades in
    one batch and weights keep the FP32 tolerance; an all-zero input gives
    zeros; a NaN or an infinity among the values reaches the output as in
    float arithmetic."""
    rng = np.random.default_rng(47)
    n, pitch, m = 128, 10e-6, 6000
    x, y, c = random_case(47, n, m, pitch=pitch)
    c[:7] *= 1e4
    c[7:20] *= 1e-4
    wts = rng.uniform(0.2, 2.0, m)
    kw = dict(pitch=pitch, lam=633e-9, z=0.03, ox=10e-6)
    got = run_gpu(P, "asm", 1, "f32", n, x=x, y=y, values=c, w=wts, tile=64, **kw)
    ref = run_oracle("asm", 1, n, x=x, y=y, values=c, w=wts, **kw)
    assert O.rel_l2(got, ref) < TOL["f32"]
    zero = run_gpu(P, "asm", 1, "f32", n, x=x, y=y, values=np.zeros(m), tile=64, **kw)
    assert not np.any(zero)
    for bad in (np.nan, np.inf):
        cb = c.copy()
        cb[100] = bad
        out = run_gpu(P, "asm", 1, "f32", n, x=x, y=y, values=cb, tile=64, **kw)
        assert not np.all(np.isfinite(out))


# ---------------------------------------------------------------- Gaussian (Greengard-Lee) kernel option
@pytest.mark.parametrize("kind", ["asm", "fresnel"])
@pytest.mark.parametrize("type_", [1, 2])
@pytest.mark.parametrize("prec,tol,bound", [("f32", 0.0, 1e-5), ("f64", 1e-7, 1e-6), ("f64", 1e-10, 1e-10),
                                            ("f64", 0.0, 1e-10)])
def test_gaussian_kernel_parity(P, kind, type_, prec, tol, bound):
    """The paper's Gaussian gridding kernel on every path: FP32 at its default
    tolerance, FP64 at 1e-7 (15 taps), 1e-10 (21 taps) and the FP64 default
    1e-12 (25 taps, tiles of at least 32 cells), against the oracle."""
    x, y, vals = random_case(51 + type_, 64, 600, type_=type_)
    kw = dict(pitch=10e-6, lam=633e-9, z=0.03, ox=25e-6, oy=-12e-6)
    got = run_gpu(P, kind, type_, prec, 64, x=x, y=y, values=vals, tol=tol, kernel="gaussian", **kw)
    ref = run_oracle(kind, type_, 64, x=x, y=y, values=vals, prec=prec, **kw)
    assert O.rel_l2(got, ref) < bound


# ---------------------------------------------------------------- gridding tile sides
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tile_sides_agree(P, prec):
    """Type 2 is the same gather whatever the tile side (bit for bit); type 1
    differs only by the accumulation order / fixed-point quantum."""
    kw = dict(pitch=10e-6, lam=633e-9, z=0.03, ox=25e-6)
    x, y, u1 = random_case(61, 128, 5000, type_=2)
    outs2 = [run_gpu(P, "asm", 2, prec, 128, x=x, y=y, values=u1, tile=t, **kw) for t in (16, 32, 64)]
    assert np.array_equal(outs2[0], outs2[1]) and np.array_equal(outs2[0], outs2[2])
    x, y, c = random_case(62, 128, 5000, type_=1)
    outs1 = [run_gpu(P, "asm", 1, prec, 128, x=x, y=y, values=c, tile=t, **kw) for t in (16, 32, 64)]
    ref = run_oracle("asm", 1, 128, x=x, y=y, values=c, prec=prec, **kw)
    for o in outs1:
        assert O.rel_l2(o, ref) < TOL[prec]


def test_autotune_tile_picks_a_supported_side(P):
    w = WL.nuasm2_graded(n=256)
    params = P.make_params(w.n, w.pitch, w.lam, w.z, ox=w.ox)
    tile, ms = P.nuasm_autotune_tile(params, _t(w.x), _t(w.y), 2)
    assert tile in (16, 32, 64) and ms > 0


def test_split_work_knobs_keep_results(P):
    """interp_chunk splits dense tiles' interpolation over CTAs (type 2 equal
    bit for bit); spread_chunk splits or keeps dense tiles in spreading
    (type 1 equal to rounding: the chunks add into the window in any order;
    in FP64 whole tiles spread in double-float arithmetic with exact integer
    sums at a quantum of 2^-52 of a 512-record batch's magnitude, split tiles
    with FP64 atomics, so the two agree to about 1e-13, below the FP64
    default tolerance 1e-12)."""
    rng = np.random.default_rng(46)
    n, pitch, m = 64, 10e-6, 30000
    x = WL.clamp_window(rng.normal(0, 40e-6, m), n, pitch)
    y = WL.clamp_window(rng.normal(0, 40e-6, m), n, pitch)
    c = rng.normal(size=m) + 1j * rng.normal(size=m)
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    kw = dict(pitch=pitch, lam=633e-9, z=0.02, x=x, y=y)
    v0 = run_gpu(P, "asm", 2, "f32", n, values=u1, **kw)
    v1 = run_gpu(P, "asm", 2, "f32", n, values=u1, **kw, interp_chunk=64)
    assert np.array_equal(v0, v1)
    for prec in ("f32", "f64"):
        tile = 16 if prec == "f64" else 32   # the split-capable spreading kernels
        a = run_gpu(P, "asm", 1, prec, n, values=c, tile=tile, spread_chunk=-1, **kw)
        b = run_gpu(P, "asm", 1, prec, n, values=c, tile=tile, spread_chunk=32, **kw)
        d = run_gpu(P, "asm", 1, prec, n, values=c, tile=tile, **kw)
        lim = 1e-6 if prec == "f32" else 1e-12
        assert O.rel_l2(b, a) < lim and O.rel_l2(d, a) < lim


@pytest.mark.parametrize("kind", ["asm", "fresnel"])
@pytest.mark.parametrize("tile,tol,chunk", [(16, 0.0, -1), (64, 0.0, -1), (32, 1e-10, -1), (64, 1e-10, -1),
                                            (16, 0.0, 64), (64, 1e-10, 700)])
def test_fp64_double_float_spreading(P, kind, tile, tol, chunk):
    """FP64-mode spreading on the double-float path (ES kernel at w = 13, the
    FP64 default, and w = 11, tolerance 1e-10), by whole tiles and with dense
    tiles split into chunks (one batch or several per chunk): a cluster and a
    uniform background give tiles of one record batch and of several, the
    values span twelve decades and carry point weights.  rel-L2 1e-10 against
    the oracle, and every pixel within 10 x 1e-10 of the RMS."""
    rng = np.random.default_rng(61)
    n, pitch, m = 64, 10e-6, 6000
    half = 0.5 * n * pitch

    def coord():
        return WL.clamp_window(np.concatenate([rng.normal(0, 30e-6, m // 2),
                                               rng.uniform(-half, half, m - m // 2)]), n, pitch)
    x, y = coord(), coord()
    c = rng.normal(size=m) + 1j * rng.normal(size=m)
    c[:10] *= 1e6
    c[10:40] *= 1e-6
    wts = rng.uniform(0.5, 1.5, m)
    kw = dict(pitch=pitch, lam=633e-9, z=0.03, ox=10e-6)
    got = run_gpu(P, kind, 1, "f64", n, x=x, y=y, values=c, w=wts, tile=tile, tol=tol, spread_chunk=chunk, **kw)
    ref = run_oracle(kind, 1, n, x=x, y=y, values=c, w=wts, prec="f64", **kw)
    assert O.rel_l2(got, ref) < TOL["f64"]
    assert np.max(np.abs(got - ref)) <= 10 * TOL["f64"] * np.linalg.norm(ref) / np.sqrt(ref.size)


@pytest.mark.parametrize("n,m", [(64, 3000), (256, 1000)])
@pytest.mark.parametrize("type_", [1, 2])
@pytest.mark.parametrize("scale", [1e-300, 1e-200, 1e200])
def test_fp64_double_float_gridding_extreme_magnitudes(P, n, m, type_, scale):
    """The double-float FP64 gridding scales each batch (spreading) and each
    staged tile (interpolation), and the double-float row passes (N' >= 512)
    each CTA's rows, by a power of two before splitting values into float
    pairs, so inputs far outside the float range keep FP64-mode accuracy: the
    scaled input's output is the scaled output (rel-L2 1e-10 against the
    oracle on the scaled input, whose results reach 1e-300)."""
    pitch = 10e-6
    x, y, vals = random_case(63 + type_, n, m, pitch=pitch, type_=type_)
    kw = dict(pitch=pitch, lam=633e-9, z=0.03, ox=10e-6)
    got = run_gpu(P, "fresnel", type_, "f64", n, x=x, y=y, values=vals * scale, tile=64, spread_chunk=-1, **kw)
    ref = run_oracle("fresnel", type_, n, x=x, y=y, values=vals * scale, prec="f64", **kw)
    got, ref = got / scale, ref / scale   # norms of values near 1e-300 would underflow
    assert np.all(np.isfinite(got)) and np.linalg.norm(ref) > 0
    assert O.rel_l2(got, ref) < TOL["f64"]


@pytest.mark.parametrize("n", [512, 1024])
@pytest.mark.parametrize("type_", [1, 2])
def test_fp64_double_float_passes_mid_sizes(P, n, type_):
    """FP64 mode at N' = 1024 and 2048, where the row passes run one row per
    CTA and the column passes four columns per CTA in double-float: 600
    points (type 1: sources; type 2: destinations of a random N x N plane)
    against the oracle at rel-L2 1e-10."""
    x, y, vals = random_case(70 + n + type_, n, 600, pitch=8e-6, type_=type_)
    kw = dict(pitch=8e-6, lam=532e-9, z=0.04, ox=20e-6, oy=-8e-6)
    got = run_gpu(P, "asm", type_, "f64", n, x=x, y=y, values=vals, **kw)
    ref = run_oracle("asm", type_, n, x=x, y=y, values=vals, prec="f64", **kw)
    assert O.rel_l2(got, ref) < TOL["f64"]


def test_fp64_double_float_spreading_zero_and_non_finite(P):
    """The double-float FP64 spreading: an all-zero input gives zeros, and an
    infinity or a NaN among the values reaches the output."""
    n, pitch, m = 64, 10e-6, 4000
    x, y, c = random_case(62, n, m, pitch=pitch)
    kw = dict(pitch=pitch, lam=633e-9, z=0.03, tile=64, spread_chunk=-1)
    zero = run_gpu(P, "asm", 1, "f64", n, x=x, y=y, values=np.zeros(m), **kw)
    assert not np.any(zero)
    for bad in (np.nan, np.inf):
        cb = c.copy()
        cb[100] = bad
        out = run_gpu(P, "asm", 1, "f64", n, x=x, y=y, values=cb, **kw)
        assert not np.all(np.isfinite(out))


def test_autotuner_returns_working_parameters(P):
    """nuasm_autotune returns the plane's own parameters with a tile side and
    split chunks from its search space, and a plan made with them gives the
    default plan's result (to rounding; both are parity-tested elsewhere)."""
    rng = np.random.default_rng(47)
    n, pitch, m = 128, 8e-6, 50000
    h = 0.5 * n * pitch * (1 - 1e-9)
    x, y = rng.uniform(-h, h, m), rng.uniform(-h, h, m)
    params = P.make_params(n, pitch, 532e-9, 0.05)
    for type_ in (1, 2):
        best, ms = P.nuasm_autotune(params, _t(x), _t(y), type_)
        assert best.tile in (16, 32, 64) and ms > 0
        assert best.interp_chunk in (0, 1024, 2048) and best.spread_chunk in (0, -1, 256)
        assert (best.n, best.pitch, best.z) == (params.n, params.pitch, params.z)
        kw = dict(pitch=pitch, lam=532e-9, z=0.05, x=x, y=y, tile=best.tile, interp_chunk=best.interp_chunk,
                  spread_chunk=best.spread_chunk)
        vals = rng.normal(size=m) + 1j * rng.normal(size=m) if type_ == 1 else \
            rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        got = run_gpu(P, "asm", type_, "f32", n, values=vals, **kw)
        ref2 = run_gpu(P, "asm", type_, "f32", n, values=vals, pitch=pitch, lam=532e-9, z=0.05, x=x, y=y)
        assert O.rel_l2(got, ref2) < 1e-6
