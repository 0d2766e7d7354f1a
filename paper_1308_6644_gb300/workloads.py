"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws coordinates and field values; it holds none of the
diffraction arithmetic, so the CUDA path and the CPU oracle can both be fed
from it.  Every generator uses numpy's PCG64 (``numpy.random.default_rng``)
with an explicit seed.

The paper's test images (an amplitude picture and a phase picture, both
256 x 256) are not available, so random fields with the same shapes stand in
for them; the non-uniform coordinate sets reproduce the geometries described
in the paper (jittered lattices, graded pitch, quadrant pitches) and the
clustered distributions used for stress cases.

All coordinates are metres relative to the centre of the uniform plane, and
every point lies in the half-open window [-N pitch / 2, N pitch / 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Points are clamped to at most this fraction of the half-window so that
# x / pitch stays strictly below N/2 after rounding.
_EDGE = 1.0 - 1e-12


@dataclass
class Workload:
    """One synthetic problem: geometry, points and input field."""
    name: str
    kind: str              # "asm" | "fresnel"
    type: int              # 1: non-uniform source -> uniform plane; 2: uniform -> non-uniform
    n: int
    pitch: float
    lam: float
    z: float
    ox: float = 0.0
    oy: float = 0.0
    x: np.ndarray = field(default_factory=lambda: np.zeros(0))
    y: np.ndarray = field(default_factory=lambda: np.zeros(0))
    values: np.ndarray = field(default_factory=lambda: np.zeros(0, np.complex128))
    weights: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(len(self.x))

    def params(self) -> dict:
        return dict(n=self.n, n_pad=2 * self.n, pitch=self.pitch, lam=self.lam, z=self.z,
                    ox=self.ox, oy=self.oy, kind=self.kind)


def clamp_window(v: np.ndarray, n: int, pitch: float) -> np.ndarray:
    half = 0.5 * n * pitch
    return np.clip(v, -half, half * _EDGE)


def random_phasor(rng, shape, amp="uniform") -> np.ndarray:
    """Field values: amplitude U[0,1) (or Bernoulli(1/2) with amp='binary')
    times a uniform random phase."""
    if amp == "binary":
        a = (rng.random(shape) < 0.5).astype(np.float64)
    else:
        a = rng.random(shape)
    return a * np.exp(1j * 2.0 * np.pi * rng.random(shape))


def gaussian_beam(x: np.ndarray, y: np.ndarray, w0: float) -> np.ndarray:
    """Input field exp(-|x|^2 / w0^2) sampled at (x, y)."""
    return np.exp(-(x * x + y * y) / (w0 * w0)).astype(np.complex128)


def jittered_lattice(rng, n: int, pitch: float, jitter: float) -> tuple[np.ndarray, np.ndarray]:
    """Lattice (i - n/2) * pitch, i in [0, n), jittered by U(+-jitter*pitch) per axis."""
    m = (np.arange(n) - n // 2) * pitch
    yy, xx = np.meshgrid(m, m, indexing="ij")
    xx = xx + rng.uniform(-jitter, jitter, xx.shape) * pitch
    yy = yy + rng.uniform(-jitter, jitter, yy.shape) * pitch
    return xx.ravel(), yy.ravel()


def dense_centre_lattice(rng, n: int, pitch: float, jitter: float, core: int) -> tuple[np.ndarray, np.ndarray]:
    """n x n jittered lattice whose central core x core points are replaced by
    a (2 core) x (2 core) jittered lattice at half the pitch."""
    m = np.arange(n) - n // 2
    yy, xx = np.meshgrid(m, m, indexing="ij")
    keep = ~((np.abs(xx + 0.5) < core / 2) & (np.abs(yy + 0.5) < core / 2))
    x0 = xx[keep] * pitch + rng.uniform(-jitter, jitter, keep.sum()) * pitch
    y0 = yy[keep] * pitch + rng.uniform(-jitter, jitter, keep.sum()) * pitch
    x1, y1 = jittered_lattice(rng, 2 * core, pitch / 2, jitter)
    return np.concatenate([x0, x1]), np.concatenate([y0, y1])


def graded_points(rng, n_side: int, half_extent: float, jitter: float) -> tuple[np.ndarray, np.ndarray]:
    """n_side^2 points whose local pitch grows from the centre to the edge.

    An index lattice t in (-1, 1)^2 is warped radially (Chebyshev norm
    rho = max(|t_x|, |t_y|)) by p = t * phi(rho) / rho with
    phi(rho) = (rho + rho^3) / 2: the radial pitch is 1/2 of the base pitch at
    the centre and 2x at the edge (a 4x grading).  Each point is jittered by
    U(+-jitter * local radial pitch).
    """
    t = -1.0 + (np.arange(n_side) + 0.5) * (2.0 / n_side)
    ty, tx = np.meshgrid(t, t, indexing="ij")
    rho = np.maximum(np.abs(tx), np.abs(ty))
    scale = 0.5 * (1.0 + rho * rho)                    # phi(rho) / rho
    px, py = tx * scale, ty * scale
    base = 2.0 * half_extent / n_side
    local = 0.5 * (1.0 + 3.0 * rho * rho) * base       # d phi / d rho * base pitch
    px = px * half_extent + rng.uniform(-jitter, jitter, px.shape) * local
    py = py * half_extent + rng.uniform(-jitter, jitter, py.shape) * local
    return px.ravel(), py.ravel()


def clustered_points(rng, m: int, half_extent: float, patches: int = 4,
                     sigma_frac: float = 0.1, cluster_share: float = 0.75) -> tuple[np.ndarray, np.ndarray]:
    """m points: cluster_share of them in Gaussian patches (sigma =
    sigma_frac * aperture, seeded centres within +-0.3 aperture), the rest
    uniform over the window."""
    aperture = 2.0 * half_extent
    mc = int(round(m * cluster_share))
    centres = rng.uniform(-0.3, 0.3, (patches, 2)) * aperture
    which = rng.integers(0, patches, mc)
    xc = centres[which, 0] + rng.normal(0.0, sigma_frac * aperture, mc)
    yc = centres[which, 1] + rng.normal(0.0, sigma_frac * aperture, mc)
    mu = m - mc
    xu = rng.uniform(-half_extent, half_extent, mu)
    yu = rng.uniform(-half_extent, half_extent, mu)
    x = np.concatenate([xc, xu])
    y = np.concatenate([yc, yu])
    perm = rng.permutation(m)
    return x[perm], y[perm]


def quadrant_lattice(n: int, pitch: float, scales=(0.9, 0.8, 0.7, 1.0)) -> tuple[np.ndarray, np.ndarray]:
    """n x n samples whose pitch differs per quadrant (first to fourth
    quadrant: scales[0..3] x pitch), laid outwards from the centre."""
    h = n // 2
    i = np.arange(h) + 0.5
    xs, ys = [], []
    signs = [(1, 1), (-1, 1), (-1, -1), (1, -1)]      # quadrants I..IV
    for (sx, sy), s in zip(signs, scales):
        yy, xx = np.meshgrid(i * s * pitch * sy, i * s * pitch * sx, indexing="ij")
        xs.append(xx.ravel())
        ys.append(yy.ravel())
    return np.concatenate(xs), np.concatenate(ys)


# ----------------------------------------------------------------------------
# The named workloads
# ----------------------------------------------------------------------------

def nuasm1_small(seed: int = 1001) -> Workload:
    """NU-ASM_1, 64 x 64 jittered source (10 um pitch, +-0.4 pitch jitter) with
    a 2x denser 32 x 32 core replacing the central 16 x 16 points (M = 4864),
    uniform 64 x 64 destination at 10 um, lambda 633 nm, z 5 cm, on axis."""
    rng = np.random.default_rng(seed)
    n, pitch = 64, 10e-6
    x, y = dense_centre_lattice(rng, n, pitch, 0.4, 16)
    x, y = clamp_window(x, n, pitch), clamp_window(y, n, pitch)
    c = random_phasor(rng, len(x))
    return Workload("nuasm1_n64_m4864", "asm", 1, n, pitch, 633e-9, 0.05, x=x, y=y, values=c)


def paper_experiment(seed: int = 1006) -> Workload:
    """The paper's NU-ASM_1 experiment geometry: 256 x 256 source samples whose
    pitch is 0.9/0.8/0.7/1.0 x 5 um in quadrants I-IV (weights: each sample's
    area relative to 5 um x 5 um), uniform 256 x 256 destination at 5 um,
    lambda 500 nm, z 8 mm, N' = 512.  Amplitude U[0, 1) and phase
    U[-pi/2, pi/2) stand in for the paper's two test images."""
    rng = np.random.default_rng(seed)
    n, pitch = 256, 5e-6
    x, y = quadrant_lattice(n, pitch)
    scale = np.select([(x > 0) & (y > 0), (x < 0) & (y > 0), (x < 0) & (y < 0)], [0.9, 0.8, 0.7], 1.0)
    c = rng.uniform(0.0, 1.0, n * n) * np.exp(1j * rng.uniform(-0.5 * np.pi, 0.5 * np.pi, n * n))
    return Workload(f"nuasm1_paper_n{n}_m{n * n}", "asm", 1, n, pitch, 500e-9, 8e-3, x=x, y=y, values=c,
                    weights=scale ** 2)


def nuasm2_graded(seed: int = 1002, n: int = 1024, pitch: float = 8e-6) -> Workload:
    """NU-ASM_2, uniform n x n source at 8 um holding a binary-amplitude
    random-phase pattern; n^2 destination points whose pitch grades 4 -> 16 um
    from the centre to the edge (+-0.3 local-pitch jitter); lambda 532 nm,
    z 20 cm, off-axis offset (1 mm, 0)."""
    rng = np.random.default_rng(seed)
    half = 0.5 * n * pitch
    x, y = graded_points(rng, n, half, 0.3)
    x, y = clamp_window(x, n, pitch), clamp_window(y, n, pitch)
    u1 = random_phasor(rng, (n, n), amp="binary")
    return Workload(f"nuasm2_n{n}_m{len(x)}", "asm", 2, n, pitch, 532e-9, 0.20,
                    ox=1e-3, oy=0.0, x=x, y=y, values=u1)


def fresnel_clustered(seed: int = 1003, type_: int = 2, n: int = 2048, m: int | None = None,
                      pitch: float = 4e-6, w0: float = 0.5e-3) -> Workload:
    """NU-FRE, n x n plane at 4 um, m points (default n^2) with 3/4 of them in
    4 Gaussian patches (sigma 0.1 aperture) over a uniform background,
    lambda 633 nm, z 1 m, Gaussian-beam input with waist w0."""
    rng = np.random.default_rng(seed)
    m = n * n if m is None else m
    half = 0.5 * n * pitch
    x, y = clustered_points(rng, m, half)
    x, y = clamp_window(x, n, pitch), clamp_window(y, n, pitch)
    if type_ == 1:
        vals = gaussian_beam(x, y, w0)
    else:
        g = (np.arange(n) - n // 2) * pitch
        gy, gx = np.meshgrid(g, g, indexing="ij")
        vals = gaussian_beam(gx, gy, w0)
    return Workload(f"nufre{type_}_n{n}_m{m}", "fresnel", type_, n, pitch, 633e-9, 1.0,
                    x=x, y=y, values=vals, extra={"w0": w0})


def mixed_plane(seed: int, plane: int) -> Workload:
    """One plane of the mixed batch: N in {256, 512, 1024, 2048}, type 1 or 2
    alternating, z ~ U[1, 50] cm, lambda in {450, 532, 633} nm, M/N^2
    log-uniform in [0.25, 4], jittered-lattice or clustered points."""
    rng = np.random.default_rng(seed + plane)
    n = int(rng.choice([256, 512, 1024, 2048]))
    type_ = 1 + (plane % 2)
    z = float(rng.uniform(0.01, 0.50))
    lam = float(rng.choice([450e-9, 532e-9, 633e-9]))
    pitch = 8e-6
    ratio = float(np.exp(rng.uniform(np.log(0.25), np.log(4.0))))
    m = max(1, int(ratio * n * n))
    half = 0.5 * n * pitch
    if rng.random() < 0.5:
        side = max(1, int(round(np.sqrt(m))))
        x, y = jittered_lattice(rng, side, 2 * half / side, 0.4)
    else:
        x, y = clustered_points(rng, m, half)
    x, y = clamp_window(x, n, pitch), clamp_window(y, n, pitch)
    if type_ == 1:
        vals = random_phasor(rng, len(x))
    else:
        vals = random_phasor(rng, (n, n))
    return Workload(f"mixed{plane}_n{n}_t{type_}_m{len(x)}", "asm", type_, n, pitch, lam, z,
                    x=x, y=y, values=vals)


def serving_point_set(seed: int, k: int, max_points: int = 16_000_000) -> Workload:
    """Point set k of the serving workload: N in {512, 1024, 2048, 4096},
    M/N^2 log-uniform in [1/4, 1] (at most max_points), jittered-lattice or
    clustered points, 8 um pitch.  Wavelength and distance belong to the
    requests, not to the set."""
    rng = np.random.default_rng(seed + 100 + k)
    n = int(rng.choice([512, 1024, 2048, 4096]))
    pitch = 8e-6
    m = min(max_points, max(1, int(np.exp(rng.uniform(np.log(0.25), 0.0)) * n * n)))
    half = 0.5 * n * pitch
    if rng.random() < 0.5:
        side = max(1, int(np.sqrt(m)))
        x, y = jittered_lattice(rng, side, 2 * half / side, 0.4)
    else:
        x, y = clustered_points(rng, m, half)
    x, y = clamp_window(x, n, pitch), clamp_window(y, n, pitch)
    return Workload(f"serve_set{k}_n{n}_m{len(x)}", "asm", 0, n, pitch, 0.0, 0.0, x=x, y=y, values=None)


def serving_trace(seed: int, count: int, sets: int) -> list:
    """count requests: (point-set index, type 1/2, z ~ U[1, 50] cm, lambda in
    {450, 532, 633} nm, unit-mean exponential gap before the arrival)."""
    rng = np.random.default_rng(seed + 7)
    out = []
    for _ in range(count):
        out.append((int(rng.integers(0, sets)), int(rng.integers(1, 3)), float(rng.uniform(0.01, 0.50)),
                    float(rng.choice([450e-9, 532e-9, 633e-9])), float(rng.exponential(1.0))))
    return out
