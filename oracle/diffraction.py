"""Plain FP64 CPU oracle for non-uniform sampled ASM and Fresnel diffraction.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` use it.  It shares no code with the CUDA library.

Every function evaluates the definition the paper gives, written out directly:

* the NUFFTs of Eq. 7 (type 1) and Eq. 8 (type 2) are evaluated as direct
  non-uniform DFTs (no gridding, no kernel, no FFT), as matrix products of
  explicit exponential matrices;
* the uniform FFT / inverse FFT of Eq. 3, 6 and 9 are evaluated as explicit
  DFT matrix products on the zero-padded N' x N' period (N' = 2N);
* the transfer functions are Eq. 4 (band-limited, off-axis shifted ASM) and
  Eq. 5 (Fresnel, DFT of the sampled impulse response).

Readings of the paper that this module fixes (the paper is silent, garbled or
defers to an unavailable reference at these points):

* Eq. 7/8 exponent: the physical form exp(-/+ 2 pi i f_k . x) with
  f_k = k / (N' * pitch), k in [-N'/2, N'/2)^2.  The paper's normalised
  coordinate x' = 2 pi (o' + x) / N maps the window onto the padded period;
  the points occupy its central half.
* The offset term of Eq. 4 is o . f_k with o in metres.
* The Rect band of Eq. 4 ("see Ref. shift_asm") is re-derived from Nyquist
  sampling of the transfer-function phase: along each axis keep f where the
  local impulse-response position |o - z f / sqrt(1/lambda^2 - f^2)| <= S with
  S = N * pitch (band_limits()).  Explicit (c, w) in mode units override it:
  R = 1 iff |k - c| <= w / 2.
* Evanescent modes (|f| >= 1/lambda) get H = 0.
* Eq. 5 phase is read as exp(i pi |m pitch + o|^2 / (lambda z)) (the standard
  Fresnel kernel; the printed formula drops the pi) and the sum carries the
  pitch^2 area element so that amplitudes match the Fresnel integral.
* Both inverse transforms carry 1/N'^2 (FFTW's backward transform is
  unnormalised; with the factor, z = 0 ASM is the identity on lattice points).
* Points must lie in [-N pitch / 2, N pitch / 2) (the half-open range the
  paper states for x1 and x2).

The transfer-function phase z sqrt(1/lambda^2 - |f|^2) reaches 1e5-1e6 cycles
for the paper's geometries, where FP64 resolves only ~1e-10 cycles, so this
oracle evaluates that phase (and z/lambda in the Fresnel constant) in the
platform's extended precision (numpy.longdouble: 80-bit on x86-64, binary128
on aarch64) and reduces it mod 1 before the FP64 exponential.
"""
from __future__ import annotations

import numpy as np

_LD = np.longdouble
if np.finfo(_LD).eps > 1e-18:  # pragma: no cover - platform guard
    raise RuntimeError("oracle needs an extended-precision numpy.longdouble")

TWO_PI = 2.0 * np.pi


def modes(n_pad: int) -> np.ndarray:
    """Integer mode indices k in [-N'/2, N'/2) (the FFT-natural range, Eq. 3)."""
    return np.arange(-n_pad // 2, n_pad // 2, dtype=np.int64)


def lattice(n: int) -> np.ndarray:
    """Centred uniform-plane indices m in [-N/2, N/2) (Eq. 3, plane layout)."""
    return np.arange(-n // 2, n // 2, dtype=np.int64)


def _cis_cycles(c: np.ndarray) -> np.ndarray:
    """exp(2 pi i c) for c in cycles, reduced mod 1 first (exact in FP64)."""
    c = np.asarray(c)
    frac = (c - np.rint(c)).astype(np.float64)
    return np.exp(1j * TWO_PI * frac)


def _dft_matrix(k: np.ndarray, m: np.ndarray, n_pad: int, sign: int) -> np.ndarray:
    """E[a, b] = exp(sign * 2 pi i k_a m_b / N') built from exact integer products."""
    prod = np.mod(np.outer(k, m), n_pad)            # exact integer reduction
    roots = np.exp(sign * 1j * TWO_PI * np.arange(n_pad) / n_pad)
    return roots[prod]


# ----------------------------------------------------------------------------
# Transfer functions (Eq. 4 and Eq. 5)
# ----------------------------------------------------------------------------

def band_limits(n: int, pitch: float, lam: float, z: float, o: float):
    """Frequency interval [f_lo, f_hi] of the Rect band along one axis.

    Reading of Eq. 4's band (the paper defers it to another reference): the
    transfer-function phase 2 pi (o f + z sqrt(1/lambda^2 - f^2)) has local
    spatial position o - z f / sqrt(1/lambda^2 - f^2); sampling it at
    1/(N' pitch) without aliasing needs that position inside [-S, S] with
    S = N pitch.  Inverting t = z f / sqrt(1/lambda^2 - f^2) gives
    f = sign(z) t / (lambda sqrt(z^2 + t^2)).  For z = 0 the band is the full
    axis when |o| <= S and empty otherwise.
    """
    s = n * pitch
    if z == 0.0:
        return (-np.inf, np.inf) if abs(o) <= s else (np.inf, -np.inf)

    def ginv(t):
        return np.sign(z) * t / (lam * np.sqrt(z * z + t * t))

    a, b = ginv(o - s), ginv(o + s)
    return (min(a, b), max(a, b))


def band_mask_1d(n: int, n_pad: int, pitch: float, lam: float, z: float, o: float,
                 centre=None, width=None) -> np.ndarray:
    """Rect factor along one axis over k in [-N'/2, N'/2).

    With explicit ``centre``/``width`` (mode units, Eq. 4's c and w) the mode
    is kept iff |k - c| <= w/2; otherwise the band of band_limits() is used,
    edges inclusive.
    """
    k = modes(n_pad)
    if centre is not None:
        return np.abs(k - centre) <= width / 2.0
    f = k / (n_pad * pitch)
    lo, hi = band_limits(n, pitch, lam, z, o)
    return (f >= lo) & (f <= hi)


def asm_transfer(n: int, n_pad: int, pitch: float, lam: float, z: float,
                 ox: float = 0.0, oy: float = 0.0, band=None,
                 rows: np.ndarray | None = None) -> np.ndarray:
    """Band-limited, off-axis shifted ASM transfer function H[ky, kx] (Eq. 4).

    H(k) = Rect(k) * exp(2 pi i (o . f_k + z sqrt(1/lambda^2 - |f_k|^2))),
    f_k = k / (N' pitch); zero for evanescent modes.  ``band`` is None for the
    derived rule or (c_m, c_n, w_m, w_n) in mode units.  ``rows`` restricts
    the output to a subset of ky indices (array positions) to bound memory.
    """
    k = modes(n_pad)
    ky_idx = np.arange(n_pad) if rows is None else np.asarray(rows)
    if band is None:
        rx = band_mask_1d(n, n_pad, pitch, lam, z, ox)
        ry = band_mask_1d(n, n_pad, pitch, lam, z, oy)
    else:
        c_m, c_n, w_m, w_n = band
        rx = band_mask_1d(n, n_pad, pitch, lam, z, ox, c_m, w_m)
        ry = band_mask_1d(n, n_pad, pitch, lam, z, oy, c_n, w_n)
    denom = _LD(n_pad) * _LD(pitch)
    fx = (k.astype(_LD) / denom)[None, :]
    fy = (k[ky_idx].astype(_LD) / denom)[:, None]
    arg = _LD(1.0) / (_LD(lam) * _LD(lam)) - fx * fx - fy * fy
    prop = arg > 0
    phase = _LD(ox) * fx + _LD(oy) * fy + _LD(z) * np.sqrt(np.where(prop, arg, _LD(0)))
    h = _cis_cycles(phase)
    h[~prop] = 0.0
    h *= (ry[ky_idx][:, None] & rx[None, :])
    return h


def fresnel_transfer(n_pad: int, pitch: float, lam: float, z: float,
                     ox: float = 0.0, oy: float = 0.0) -> np.ndarray:
    """Fresnel transfer function H[ky, kx] (Eq. 5): the N' x N' DFT of the
    sampled impulse response

        h(x) = exp(i k z) / (i lambda z) * exp(i pi |x|^2 / (lambda z)),
        H(k) = pitch^2 * sum_{m in [-N'/2, N'/2)^2} h(m pitch + o) exp(-2 pi i k.m / N').

    The full 2-D sampled array is built and transformed by the 2-D DFT
    definition (written as E h E^T); separability is not assumed.
    """
    if z == 0.0:
        raise ValueError("Fresnel transfer function needs z != 0")
    m = lattice(n_pad)
    xs = (m * pitch + ox).astype(np.float64)
    ys = (m * pitch + oy).astype(np.float64)
    r2 = ys[:, None] ** 2 + xs[None, :] ** 2
    h = _cis_cycles(r2 / (2.0 * lam * z))
    const = pitch * pitch * _cis_cycles(_LD(z) / _LD(lam)) / (1j * lam * z)
    e = _dft_matrix(modes(n_pad), m, n_pad, -1)
    return const * (e @ h @ e.T)


# ----------------------------------------------------------------------------
# Direct transforms (Eq. 3, 6, 7, 8, 9)
# ----------------------------------------------------------------------------

def _chunk_len(n_pad: int) -> int:
    return max(64, min(4096, (1 << 24) // max(n_pad, 1)))


def nudft_type1(xi_x: np.ndarray, xi_y: np.ndarray, c: np.ndarray, n_pad: int) -> np.ndarray:
    """Direct NUFFT type 1 (Eq. 7): F[ky, kx] = sum_j c_j exp(-2 pi i k . xi_j / N').

    xi = x / pitch are point positions in pixel units of the uniform plane.
    """
    k = modes(n_pad)
    out = np.zeros((n_pad, n_pad), dtype=np.complex128)
    step = _chunk_len(n_pad)
    c = np.asarray(c, dtype=np.complex128)
    for s in range(0, len(c), step):
        sl = slice(s, s + step)
        ax = _cis_cycles(-np.outer(xi_x[sl], k) / n_pad)          # [J, kx]
        ay = _cis_cycles(-np.outer(xi_y[sl], k) / n_pad)          # [J, ky]
        out += (ay * c[sl, None]).T @ ax
    return out


def nudft_type2(a: np.ndarray, xi_x: np.ndarray, xi_y: np.ndarray, n_pad: int) -> np.ndarray:
    """Direct NUFFT type 2 (Eq. 8): v_j = sum_k a[ky, kx] exp(+2 pi i k . xi_j / N')."""
    k = modes(n_pad)
    v = np.empty(len(xi_x), dtype=np.complex128)
    step = _chunk_len(n_pad)
    for s in range(0, len(xi_x), step):
        sl = slice(s, s + step)
        bx = _cis_cycles(np.outer(xi_x[sl], k) / n_pad)            # [J, kx]
        by = _cis_cycles(np.outer(xi_y[sl], k) / n_pad)            # [J, ky]
        t = a @ bx.T                                               # [ky, J]
        v[sl] = np.einsum("jk,kj->j", by, t)
    return v


def uniform_dft(u1: np.ndarray, n_pad: int) -> np.ndarray:
    """G[ky, kx] = sum_m u1[m] exp(-2 pi i k . m / N'), m in [-N/2, N/2)^2:
    the forward FFT of the zero-padded uniform plane (Eq. 3, 9)."""
    n = u1.shape[0]
    e = _dft_matrix(modes(n_pad), lattice(n), n_pad, -1)           # [N', N]
    return e @ np.asarray(u1, dtype=np.complex128) @ e.T


def uniform_idft_crop(f: np.ndarray, n: int) -> np.ndarray:
    """u[my, mx] = sum_k f[ky, kx] exp(+2 pi i k . m / N'), m in [-N/2, N/2)^2:
    the unnormalised inverse FFT of Eq. 3/6 cropped to the N x N plane."""
    n_pad = f.shape[0]
    d = _dft_matrix(modes(n_pad), lattice(n), n_pad, +1)           # [N', N]
    return d.T @ f @ d


def _check_window(xi, n):
    if len(xi) and (np.min(xi) < -n / 2 or np.max(xi) >= n / 2):
        raise ValueError("point outside [-N pitch/2, N pitch/2)")


def _transfer(p: dict) -> np.ndarray:
    n, n_pad = p["n"], p.get("n_pad") or 2 * p["n"]
    if p.get("kind", "asm") == "asm":
        return asm_transfer(n, n_pad, p["pitch"], p["lam"], p["z"],
                            p.get("ox", 0.0), p.get("oy", 0.0), p.get("band"))
    return fresnel_transfer(n_pad, p["pitch"], p["lam"], p["z"],
                            p.get("ox", 0.0), p.get("oy", 0.0))


def diffraction_type1(x, y, c, p: dict, weights=None, h=None) -> np.ndarray:
    """NU-ASM_1 (Eq. 6) or NU-FRE_1: non-uniform source -> uniform N x N plane.

    u2(m) = (1/N'^2) sum_k F(k) H(k) exp(2 pi i k . m / N'),
    F = NUFFT_1[w c] evaluated directly (Eq. 7).  ``p`` holds n, n_pad
    (0 => 2N), pitch (the destination pitch Delta_2), lam, z, ox, oy, band,
    kind ('asm' | 'fresnel').  ``h`` overrides the transfer function.
    """
    n = p["n"]
    n_pad = p.get("n_pad") or 2 * n
    xi_x = np.asarray(x, np.float64) / p["pitch"]
    xi_y = np.asarray(y, np.float64) / p["pitch"]
    _check_window(xi_x, n)
    _check_window(xi_y, n)
    c = np.asarray(c, np.complex128)
    if weights is not None:
        c = c * np.asarray(weights, np.float64)
    f = nudft_type1(xi_x, xi_y, c, n_pad)
    hh = _transfer(p) if h is None else h
    return uniform_idft_crop(f * hh, n) / float(n_pad) ** 2


def diffraction_type2(u1, x, y, p: dict, h=None) -> np.ndarray:
    """NU-ASM_2 (Eq. 9) or NU-FRE_2: uniform N x N source -> non-uniform points.

    u2(x_j) = (1/N'^2) sum_k G(k) H(k) exp(2 pi i f_k . x_j),
    G = FFT of the zero-padded source (Eq. 9), the outer sum being NUFFT_2
    (Eq. 8) evaluated directly.  ``p`` as in diffraction_type1 (pitch is the
    source pitch Delta_1).
    """
    n = p["n"]
    n_pad = p.get("n_pad") or 2 * n
    xi_x = np.asarray(x, np.float64) / p["pitch"]
    xi_y = np.asarray(y, np.float64) / p["pitch"]
    _check_window(xi_x, n)
    _check_window(xi_y, n)
    g = uniform_dft(u1, n_pad)
    hh = _transfer(p) if h is None else h
    return nudft_type2(g * hh / float(n_pad) ** 2, xi_x, xi_y, n_pad)


def diffraction_type3(x1, y1, c, x2, y2, p: dict, weights=None, h=None) -> np.ndarray:
    """NU-ASM_3 / NU-FRE_3: non-uniform source points -> non-uniform
    destination points, the combination of Eq. 6 and Eq. 9 through the
    spectrum:  v_j = (1/N'^2) sum_k F(k) H(k) exp(2 pi i f_k . x2_j),
    F = NUFFT_1[w c] at the source points (Eq. 7), the outer sum NUFFT_2 at
    the destination points (Eq. 8), both evaluated directly.
    """
    n = p["n"]
    n_pad = p.get("n_pad") or 2 * n
    xi1x = np.asarray(x1, np.float64) / p["pitch"]
    xi1y = np.asarray(y1, np.float64) / p["pitch"]
    xi2x = np.asarray(x2, np.float64) / p["pitch"]
    xi2y = np.asarray(y2, np.float64) / p["pitch"]
    for xi in (xi1x, xi1y, xi2x, xi2y):
        _check_window(xi, n)
    c = np.asarray(c, np.complex128)
    if weights is not None:
        c = c * np.asarray(weights, np.float64)
    f = nudft_type1(xi1x, xi1y, c, n_pad)
    hh = _transfer(p) if h is None else h
    return nudft_type2(f * hh / float(n_pad) ** 2, xi2x, xi2y, n_pad)


def rs_direct(x1, y1, c, area, x2, y2, lam: float, z: float, ox: float = 0.0, oy: float = 0.0) -> np.ndarray:
    """Rayleigh-Sommerfeld diffraction (Eq. 10) as a direct sum over source
    samples with area elements:
        u2(x2) = (1/2 pi) sum_j area_j c_j (z/r)(1 - i k r) exp(i k r) / r^2,
        r = sqrt(|x2 + o - x1_j|^2 + z^2),  k = 2 pi / lambda,
    destination points given relative to the destination window centre o.
    The phase k r is evaluated as 2 pi (z/lambda + (r - z)/lambda) with
    r - z = rho^2 / (r + z) and z/lambda reduced mod 1 in extended precision.
    """
    x1 = np.asarray(x1, np.float64)
    y1 = np.asarray(y1, np.float64)
    ca = np.asarray(c, np.complex128) * np.asarray(area, np.float64)
    X2 = np.asarray(x2, np.float64) + ox
    Y2 = np.asarray(y2, np.float64) + oy
    zl = _LD(z) / _LD(lam)
    zfrac = float(zl - np.rint(zl))
    k = TWO_PI / lam
    out = np.empty(len(X2), np.complex128)
    step = max(1, (1 << 22) // max(len(x1), 1))
    for s in range(0, len(X2), step):
        dx = X2[s:s + step, None] - x1[None, :]
        dy = Y2[s:s + step, None] - y1[None, :]
        rho2 = dx * dx + dy * dy
        r = np.sqrt(rho2 + z * z)
        ph = zfrac + (rho2 / (r + z)) / lam
        kern = (z / r) * (1.0 - 1j * k * r) * _cis_cycles(ph) / (r * r) / TWO_PI
        out[s:s + step] = kern @ ca
    return out


def nuasm1(x, y, c, p, weights=None):
    """NU-ASM_1 (Eq. 6)."""
    return diffraction_type1(x, y, c, dict(p, kind="asm"), weights)


def nuasm2(u1, x, y, p):
    """NU-ASM_2 (Eq. 9)."""
    return diffraction_type2(u1, x, y, dict(p, kind="asm"))


def nuasm3(x1, y1, c, x2, y2, p, weights=None):
    """NU-ASM_3: non-uniform source -> non-uniform destination (ASM, Eq. 4)."""
    return diffraction_type3(x1, y1, c, x2, y2, dict(p, kind="asm"), weights)


def nufresnel3(x1, y1, c, x2, y2, p, weights=None):
    """NU-FRE_3: non-uniform source -> non-uniform destination (Fresnel, Eq. 5)."""
    return diffraction_type3(x1, y1, c, x2, y2, dict(p, kind="fresnel"), weights)


def nufresnel(type_: int, inp, x, y, p, weights=None):
    """NU-FRE_1 / NU-FRE_2: Eq. 6 / Eq. 9 with the Fresnel transfer function of Eq. 5."""
    q = dict(p, kind="fresnel")
    if type_ == 1:
        return diffraction_type1(x, y, inp, q, weights)
    if type_ == 2:
        return diffraction_type2(inp, x, y, q)
    raise ValueError("type must be 1 or 2")


def rel_l2(y: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error ||y - ref|| / ||ref|| over complex values."""
    ref = np.asarray(ref).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(y).ravel() - ref) / (den if den else 1.0))
