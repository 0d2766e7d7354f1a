"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a result the mathematics fixes: brute
force on tiny grids, numpy's FFT on lattice points, closed forms (Dirichlet
kernel at z = 0, Fresnel Gaussian beam, the exact complex-source-point
solution of the Helmholtz equation for the ASM), Parseval, the adjoint
identity, linearity and integer shifts, and the classic band-limited ASM
limit.  A plausible slip in the oracle (a dropped 1/N'^2, a flipped exponent
sign, a transposed operand, the wrong mode range, a missing pitch^2, a wrong
band edge) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _points(rng, n, pitch, m):
    half = 0.5 * n * pitch
    return rng.uniform(-half, half, m), rng.uniform(-half, half, m)


def _asm_params(n, pitch=10e-6, lam=633e-9, z=0.03, ox=0.0, oy=0.0, **kw):
    return dict(n=n, n_pad=2 * n, pitch=pitch, lam=lam, z=z, ox=ox, oy=oy, **kw)


def _h_tilde(h, n_pad, rx, ry):
    """(1/N'^2) sum_k H(k) exp(2 pi i k . r / N') by plain loops."""
    k = range(-n_pad // 2, n_pad // 2)
    acc = 0j
    for iy, ky in enumerate(k):
        for ix, kx in enumerate(k):
            acc += h[iy, ix] * np.exp(2j * np.pi * (kx * rx + ky * ry) / n_pad)
    return acc / n_pad ** 2


# ----------------------------------------------------------------------------
# P1: brute-force pairwise sums on tiny grids
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["asm", "fresnel"])
def test_type1_matches_pairwise_sum(kind):
    rng = _rng(1)
    n, pitch = 4, 10e-6
    p = _asm_params(n, pitch, z=0.004, ox=3e-6, oy=-7e-6, kind=kind)
    x, y = _points(rng, n, pitch, 6)
    c = rng.normal(size=6) + 1j * rng.normal(size=6)
    h = O.diffraction._transfer(p)
    got = O.diffraction_type1(x, y, c, p)
    for iy, my in enumerate(range(-n // 2, n // 2)):
        for ix, mx in enumerate(range(-n // 2, n // 2)):
            want = sum(c[j] * _h_tilde(h, 2 * n, mx - x[j] / pitch, my - y[j] / pitch)
                       for j in range(len(c)))
            assert abs(got[iy, ix] - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("kind", ["asm", "fresnel"])
def test_type2_matches_pairwise_sum(kind):
    rng = _rng(2)
    n, pitch = 4, 10e-6
    p = _asm_params(n, pitch, z=0.004, ox=-5e-6, oy=2e-6, kind=kind)
    x, y = _points(rng, n, pitch, 5)
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    h = O.diffraction._transfer(p)
    got = O.diffraction_type2(u1, x, y, p)
    for j in range(len(x)):
        want = 0j
        for iy, my in enumerate(range(-n // 2, n // 2)):
            for ix, mx in enumerate(range(-n // 2, n // 2)):
                want += u1[iy, ix] * _h_tilde(h, 2 * n, x[j] / pitch - mx, y[j] / pitch - my)
        assert abs(got[j] - want) <= 1e-13 * max(1.0, abs(want))


# ----------------------------------------------------------------------------
# P2: lattice points reproduce the FFT-based ASM of Eq. 3 (numpy.fft)
# ----------------------------------------------------------------------------

def _fft_asm(u1, h):
    n = u1.shape[0]
    n_pad = h.shape[0]
    idx = O.lattice(n) % n_pad
    pad = np.zeros((n_pad, n_pad), complex)
    pad[np.ix_(idx, idx)] = u1
    out = np.fft.ifft2(np.fft.fft2(pad) * np.fft.ifftshift(h))
    return out[np.ix_(idx, idx)]


@pytest.mark.parametrize("kind", ["asm", "fresnel"])
def test_lattice_points_equal_fft_asm(kind):
    rng = _rng(3)
    n, pitch = 16, 8e-6
    p = _asm_params(n, pitch, lam=532e-9, z=0.02, ox=40e-6, oy=-24e-6, kind=kind)
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    m = O.lattice(n) * pitch
    gy, gx = np.meshgrid(m, m, indexing="ij")
    h = O.diffraction._transfer(p)
    ref = _fft_asm(u1, h)
    u2 = O.diffraction_type1(gx.ravel(), gy.ravel(), u1.ravel(), p)
    assert O.rel_l2(u2, ref) < 1e-13
    v = O.diffraction_type2(u1, gx.ravel(), gy.ravel(), p)
    assert O.rel_l2(v, ref.ravel()) < 1e-13


# ----------------------------------------------------------------------------
# P3: z = 0, o = 0, full band: Dirichlet-kernel closed form
# ----------------------------------------------------------------------------

def _dirichlet(t, n_pad):
    t = np.asarray(t, float)
    out = np.ones_like(t, dtype=complex)
    nz = np.abs(t) > 1e-300
    tt = t[nz]
    out[nz] = np.exp(-1j * np.pi * tt / n_pad) * np.sin(np.pi * tt) / (n_pad * np.sin(np.pi * tt / n_pad))
    return out


def test_z0_dirichlet_closed_form():
    rng = _rng(4)
    n, pitch = 8, 10e-6
    p = _asm_params(n, pitch, z=0.0)
    x, y = _points(rng, n, pitch, 20)
    c = rng.normal(size=20) + 1j * rng.normal(size=20)
    u2 = O.nuasm1(x, y, c, p)
    m = O.lattice(n)
    want = np.zeros((n, n), complex)
    for j in range(len(c)):
        want += c[j] * np.outer(_dirichlet(m - y[j] / pitch, 2 * n), _dirichlet(m - x[j] / pitch, 2 * n))
    assert O.rel_l2(u2, want) < 1e-13
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    v = O.nuasm2(u1, x, y, p)
    wv = np.array([np.sum(u1 * np.outer(_dirichlet(y[j] / pitch - m, 2 * n),
                                        _dirichlet(x[j] / pitch - m, 2 * n))) for j in range(len(x))])
    assert O.rel_l2(v, wv) < 1e-13


def test_z0_identity_on_lattice():
    rng = _rng(5)
    n, pitch = 16, 10e-6
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    m = O.lattice(n) * pitch
    gy, gx = np.meshgrid(m, m, indexing="ij")
    u2 = O.nuasm1(gx.ravel(), gy.ravel(), u1.ravel(), _asm_params(n, pitch, z=0.0))
    assert O.rel_l2(u2, u1) < 1e-14


# ----------------------------------------------------------------------------
# P4: energy in band (Parseval, |H| = 1 inside the Rect band, 0 outside)
# ----------------------------------------------------------------------------

def test_energy_in_band():
    rng = _rng(6)
    n, pitch = 16, 10e-6
    p = _asm_params(n, pitch, z=0.05, ox=30e-6)
    n_pad = 2 * n
    x, y = _points(rng, n, pitch, 40)
    c = rng.normal(size=40) + 1j * rng.normal(size=40)
    f = O.nudft_type1(x / pitch, y / pitch, c, n_pad)
    h = O.asm_transfer(n, n_pad, pitch, p["lam"], p["z"], p["ox"], 0.0)
    full = O.uniform_idft_crop(f * h, n_pad) / n_pad ** 2
    band = np.abs(h) > 0.5
    assert np.allclose(np.abs(h[band]), 1.0, atol=1e-15)
    assert 0 < band.sum() < n_pad * n_pad
    lhs = np.sum(np.abs(full) ** 2)
    rhs = np.sum(np.abs(f[band]) ** 2) / n_pad ** 2
    assert abs(lhs - rhs) <= 1e-12 * rhs


# ----------------------------------------------------------------------------
# P5: adjoint identity <NUASM_1(c), v> = <c, NUASM_2^{(-z,-o)}(v)>
# ----------------------------------------------------------------------------

def test_adjoint_identity():
    rng = _rng(7)
    n, pitch = 16, 8e-6
    p = _asm_params(n, pitch, lam=532e-9, z=0.07, ox=60e-6, oy=-20e-6)
    q = dict(p, z=-p["z"], ox=-p["ox"], oy=-p["oy"])
    x, y = _points(rng, n, pitch, 50)
    c = rng.normal(size=50) + 1j * rng.normal(size=50)
    v = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    lhs = np.vdot(O.nuasm1(x, y, c, p), v)
    rhs = np.vdot(c, O.nuasm2(v, x, y, q))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the band rule is symmetric under (z, o) -> (-z, -o)
    assert np.array_equal(O.band_mask_1d(n, 2 * n, pitch, p["lam"], p["z"], p["ox"]),
                          O.band_mask_1d(n, 2 * n, pitch, p["lam"], -p["z"], -p["ox"]))


# ----------------------------------------------------------------------------
# P6: closed forms
# ----------------------------------------------------------------------------

def gaussian_fresnel_closed_form(x, y, lam, z, w0):
    """Fresnel integral of exp(-|x|^2/w0^2), by completing the square:
    exp(ikz)/(1 + i z/z_R) * exp(i a b r^2 / (a - i b)), a = 1/w0^2,
    b = pi/(lambda z), z_R = pi w0^2 / lambda."""
    a = 1.0 / w0 ** 2
    b = np.pi / (lam * z)
    zr = np.pi * w0 ** 2 / lam
    ph = np.longdouble(z) / np.longdouble(lam)
    ph = float(ph - np.rint(ph))
    r2 = x * x + y * y
    return np.exp(2j * np.pi * ph) / (1 + 1j * z / zr) * np.exp(1j * a * b * r2 / (a - 1j * b))


FRE = dict(n=128, pitch=10e-6, lam=633e-9, z=0.05, w0=0.1e-3)


def _grid(n, pitch):
    m = O.lattice(n) * pitch
    gy, gx = np.meshgrid(m, m, indexing="ij")
    return gx, gy


def test_fresnel_gaussian_type2_closed_form():
    n, pitch, lam, z, w0 = FRE["n"], FRE["pitch"], FRE["lam"], FRE["z"], FRE["w0"]
    ox, oy = 50e-6, -30e-6
    gx, gy = _grid(n, pitch)
    u1 = np.exp(-(gx ** 2 + gy ** 2) / w0 ** 2)
    rng = _rng(8)
    x, y = _points(rng, n, pitch * 0.8, 300)      # keep away from the window edge
    p = dict(n=n, pitch=pitch, lam=lam, z=z, ox=ox, oy=oy)
    v = O.nufresnel(2, u1, x, y, p)
    want = gaussian_fresnel_closed_form(x + ox, y + oy, lam, z, w0)
    assert O.rel_l2(v, want) < 1e-10


def test_fresnel_gaussian_type1_jacobian_weights():
    """Warped lattice x = phi(t) with quadrature weights phi'(t_x) phi'(t_y):
    the weighted NUFFT_1 is a spectrally accurate quadrature of the Fourier
    integral, so NU-FRE_1 reproduces the Gaussian-beam closed form."""
    n, pitch, lam, z, w0 = FRE["n"], FRE["pitch"], FRE["lam"], FRE["z"], FRE["w0"]
    L = n * pitch
    alpha = 0.3
    t = O.lattice(n) * pitch
    phi = t + alpha * L / (2 * np.pi) * np.sin(2 * np.pi * t / L)
    dphi = 1 + alpha * np.cos(2 * np.pi * t / L)
    ty, tx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x, y = phi[tx].ravel(), phi[ty].ravel()
    wts = (dphi[tx] * dphi[ty]).ravel()
    c = np.exp(-(x ** 2 + y ** 2) / w0 ** 2)
    p = dict(n=n, pitch=pitch, lam=lam, z=z, ox=0.0, oy=0.0)
    u2 = O.nufresnel(1, c, x, y, p, weights=wts)
    gx, gy = _grid(n, pitch)
    want = gaussian_fresnel_closed_form(gx, gy, lam, z, w0)
    assert O.rel_l2(u2, want) < 1e-9


def csp_field(x, y, z, lam, b):
    """Complex-source-point beam exp(ik(R + ib)) / R with
    R = sqrt(|x|^2 + (z - ib)^2): an exact solution of the Helmholtz equation
    for z > 0 (a Gaussian-like beam of waist sqrt(2b/k)); z = 0 is the limit
    from above, R = -i sqrt(b^2 - |x|^2)."""
    k = 2 * np.pi / lam
    r2 = x * x + y * y
    if z == 0:
        R = -1j * np.sqrt(b * b - r2 + 0j)
    else:
        R = np.sqrt(r2 + (z - 1j * b) ** 2 + 0j)
    return np.exp(1j * k * (R + 1j * b)) / R


CSP = dict(n=128, pitch=0.2e-6, lam=0.5e-6, w0=2e-6)


@pytest.mark.parametrize("z", [5e-6, 20e-6])
def test_asm_exact_helmholtz_solution(z):
    """Non-paraxial pin of Eq. 4: the ASM propagates the complex-source-point
    beam exactly (its spectrum is negligible outside the band and beyond
    1/lambda for these parameters)."""
    n, pitch, lam, w0 = CSP["n"], CSP["pitch"], CSP["lam"], CSP["w0"]
    b = np.pi * w0 ** 2 / lam
    ox, oy = 1.0e-6, -0.6e-6
    gx, gy = _grid(n, pitch)
    u1 = csp_field(gx, gy, 0.0, lam, b)
    p = dict(n=n, pitch=pitch, lam=lam, z=z, ox=ox, oy=oy)
    rng = _rng(9)
    x, y = _points(rng, n, pitch * 0.6, 200)
    v = O.nuasm2(u1, x, y, p)
    want = csp_field(x + ox, y + oy, z, lam, b)
    assert O.rel_l2(v, want) < 1e-10
    # sensitivity: the paraxial transfer function (square root expanded to
    # second order) misses the exact solution by far more than the tolerance
    n_pad = 2 * n
    f = O.modes(n_pad) / (n_pad * pitch)
    fx, fy = f[None, :], f[:, None]
    hp = np.exp(2j * np.pi * (ox * fx + oy * fy + z / lam - z * lam * (fx ** 2 + fy ** 2) / 2))
    hp *= np.abs(O.asm_transfer(n, n_pad, pitch, lam, z, ox, oy)) > 0
    vp = O.diffraction_type2(u1, x, y, p, h=hp)
    assert O.rel_l2(vp, want) > 1e-5


def test_asm_exact_solution_type1_lattice():
    n, pitch, lam, w0 = CSP["n"], CSP["pitch"], CSP["lam"], CSP["w0"]
    b = np.pi * w0 ** 2 / lam
    z = 10e-6
    gx, gy = _grid(n, pitch)
    c = csp_field(gx, gy, 0.0, lam, b).ravel()
    u2 = O.nuasm1(gx.ravel(), gy.ravel(), c, dict(n=n, pitch=pitch, lam=lam, z=z))
    assert O.rel_l2(u2, csp_field(gx, gy, z, lam, b)) < 1e-10


# ----------------------------------------------------------------------------
# P7: linearity and integer shifts
# ----------------------------------------------------------------------------

def test_linearity_and_integer_shift():
    rng = _rng(10)
    n, pitch = 16, 10e-6
    p = _asm_params(n, pitch, z=0.02, ox=20e-6)
    x, y = _points(rng, n, pitch * 0.5, 30)
    c1 = rng.normal(size=30) + 1j * rng.normal(size=30)
    c2 = rng.normal(size=30) + 1j * rng.normal(size=30)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = O.nuasm1(x, y, a * c1 + b * c2, p)
    rhs = a * O.nuasm1(x, y, c1, p) + b * O.nuasm1(x, y, c2, p)
    assert O.rel_l2(lhs, rhs) < 1e-14
    sx, sy = 3, -2
    u = O.nuasm1(x, y, c1, p)
    us = O.nuasm1(x + sx * pitch, y + sy * pitch, c1, p)
    # u_shift[m] = u[m - s] where both are inside the window
    assert O.rel_l2(us[max(sy, 0):n + min(sy, 0), max(sx, 0):n + min(sx, 0)],
                    u[max(-sy, 0):n + min(-sy, 0), max(-sx, 0):n + min(-sx, 0)]) < 1e-13


# ----------------------------------------------------------------------------
# Band rule (Eq. 4's Rect)
# ----------------------------------------------------------------------------

def test_band_rule_classic_limit_on_axis():
    """o = 0 reduces to the classic band-limited ASM: |f| <= 1/(lambda sqrt((2 df z)^2 + 1))
    with df = 1/(N' pitch)."""
    n, pitch, lam, z = 64, 10e-6, 633e-9, 0.05
    df = 1 / (2 * n * pitch)
    flim = 1 / (lam * np.sqrt((2 * df * z) ** 2 + 1))
    lo, hi = O.band_limits(n, pitch, lam, z, 0.0)
    assert abs(hi - flim) < 1e-9 * flim and abs(lo + flim) < 1e-9 * flim
    lo2, hi2 = O.band_limits(n, pitch, lam, -z, 0.0)
    assert (lo2, hi2) == (lo, hi)


@pytest.mark.parametrize("o", [0.0, 300e-6, -1.2e-3])
def test_band_edges_put_impulse_response_on_window_edge(o):
    n, pitch, lam, z = 64, 10e-6, 633e-9, 0.05
    s = n * pitch
    lo, hi = O.band_limits(n, pitch, lam, z, o)
    pos = lambda f: z * f / np.sqrt(1 / lam ** 2 - f ** 2) - o  # noqa: E731
    assert abs(abs(pos(lo)) - s) < 1e-12 and abs(abs(pos(hi)) - s) < 1e-12
    f = np.linspace(lo, hi, 101)[1:-1]
    assert np.all(np.abs(pos(f)) < s)


def test_explicit_band_overrides_rule():
    h = O.asm_transfer(8, 16, 10e-6, 633e-9, 0.01, band=(2.0, -1.0, 4.0, 2.0))
    k = O.modes(16)
    keep_x = np.abs(k - 2.0) <= 2.0
    keep_y = np.abs(k + 1.0) <= 1.0
    assert np.array_equal(np.abs(h) > 0, np.outer(keep_y, keep_x))


def test_evanescent_modes_are_zero():
    # pitch below lambda/2: the grid reaches beyond 1/lambda
    n, pitch, lam = 16, 0.2e-6, 0.5e-6
    h = O.asm_transfer(n, 2 * n, pitch, lam, 1e-6)
    f = O.modes(2 * n) / (2 * n * pitch)
    ev = f[None, :] ** 2 + f[:, None] ** 2 >= 1 / lam ** 2
    assert ev.any() and np.all(h[ev] == 0)


# ----------------------------------------------------------------------------
# The paper's experiment geometry (golden parameters, cited in the fixture)
# ----------------------------------------------------------------------------

def test_paper_quadrant_geometry_fits_window():
    with open(os.path.join(GOLDEN, "paper_experiment.json")) as fh:
        g = json.load(fh)
    from paper_1308_6644_gb300 import workloads as W
    n, pitch = g["n"], g["pitch_m"]
    x, y = W.quadrant_lattice(n, pitch, tuple(g["quadrant_pitch_scale"]))
    assert len(x) == n * n
    assert np.all(np.abs(x) < n * pitch / 2) and np.all(np.abs(y) < n * pitch / 2)
    # each quadrant carries its own pitch (first quadrant 0.9, ..., fourth 1.0)
    for (sx, sy), s in zip([(1, 1), (-1, 1), (-1, -1), (1, -1)], g["quadrant_pitch_scale"]):
        sel = (np.sign(x) == sx) & (np.sign(y) == sy)
        xs = np.unique(np.round(np.abs(x[sel]) / pitch, 9))
        assert np.allclose(np.diff(xs), s)


# ----------------------------------------------------------------------------
# Type 3 (NU-ASM_3 / NU-FRE_3): both planes non-uniform
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["asm", "fresnel"])
def test_type3_matches_pairwise_sum(kind):
    rng = _rng(20)
    n, pitch = 4, 10e-6
    p = _asm_params(n, pitch, z=0.004, ox=4e-6, oy=-3e-6, kind=kind)
    x1, y1 = _points(rng, n, pitch, 5)
    x2, y2 = _points(rng, n, pitch, 4)
    c = rng.normal(size=5) + 1j * rng.normal(size=5)
    h = O.diffraction._transfer(p)
    got = O.diffraction_type3(x1, y1, c, x2, y2, p)
    for j in range(len(x2)):
        want = sum(c[i] * _h_tilde(h, 2 * n, (x2[j] - x1[i]) / pitch, (y2[j] - y1[i]) / pitch)
                   for i in range(len(c)))
        assert abs(got[j] - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("kind", ["asm", "fresnel"])
def test_type3_reduces_to_types_1_and_2_on_lattices(kind):
    rng = _rng(21)
    n, pitch = 16, 8e-6
    p = _asm_params(n, pitch, lam=532e-9, z=0.03, ox=16e-6, oy=-8e-6, kind=kind)
    m = O.lattice(n) * pitch
    gy, gx = np.meshgrid(m, m, indexing="ij")
    xs, ys = _points(rng, n, pitch, 40)
    c = rng.normal(size=40) + 1j * rng.normal(size=40)
    u1 = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    # lattice destination: type 3 == type 1
    assert O.rel_l2(O.diffraction_type3(xs, ys, c, gx.ravel(), gy.ravel(), p),
                    O.diffraction_type1(xs, ys, c, p).ravel()) < 1e-13
    # lattice source: type 3 == type 2
    assert O.rel_l2(O.diffraction_type3(gx.ravel(), gy.ravel(), u1.ravel(), xs, ys, p),
                    O.diffraction_type2(u1, xs, ys, p)) < 1e-13


def test_type3_z0_dirichlet_closed_form():
    rng = _rng(22)
    n, pitch = 8, 10e-6
    p = _asm_params(n, pitch, z=0.0)
    x1, y1 = _points(rng, n, pitch, 12)
    x2, y2 = _points(rng, n, pitch, 9)
    c = rng.normal(size=12) + 1j * rng.normal(size=12)
    got = O.nuasm3(x1, y1, c, x2, y2, p)
    want = np.array([np.sum(c * _dirichlet((x2[j] - x1) / pitch, 2 * n) * _dirichlet((y2[j] - y1) / pitch, 2 * n))
                     for j in range(len(x2))])
    assert O.rel_l2(got, want) < 1e-13


# ----------------------------------------------------------------------------
# Rayleigh-Sommerfeld direct sum (Eq. 10)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("z", [5e-6, 20e-6])
def test_rs_direct_propagates_the_exact_solution(z):
    """Rayleigh-Sommerfeld of the first kind is exact for fields without
    sources in z > 0; its Riemann sum over well-sampled data reproduces the
    complex-source-point beam."""
    n, pitch, lam, w0 = 96, 0.2e-6, 0.5e-6, 2e-6
    b = np.pi * w0 ** 2 / lam
    gx, gy = _grid(n, pitch)
    u1 = csp_field(gx, gy, 0.0, lam, b)
    rng = _rng(30)
    x2, y2 = _points(rng, n, pitch * 0.5, 150)
    ox, oy = 0.8e-6, -0.4e-6
    got = O.rs_direct(gx.ravel(), gy.ravel(), u1.ravel(), np.full(n * n, pitch * pitch), x2, y2, lam, z, ox, oy)
    assert O.rel_l2(got, csp_field(x2 + ox, y2 + oy, z, lam, b)) < 1e-9


def test_rs_direct_agrees_with_asm_for_a_smooth_field():
    n, pitch, lam, w0, z = 64, 0.25e-6, 0.5e-6, 1.5e-6, 8e-6
    gx, gy = _grid(n, pitch)
    u1 = np.exp(-(gx ** 2 + gy ** 2) / w0 ** 2)
    rng = _rng(31)
    x2, y2 = _points(rng, n, pitch * 0.5, 100)
    rs = O.rs_direct(gx.ravel(), gy.ravel(), u1.ravel(), np.full(n * n, pitch * pitch), x2, y2, lam, z)
    asm = O.nuasm2(u1, x2, y2, dict(n=n, pitch=pitch, lam=lam, z=z))
    assert O.rel_l2(rs, asm) < 1e-8
