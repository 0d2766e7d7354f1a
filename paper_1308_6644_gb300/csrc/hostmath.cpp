// Plan-time host mathematics for the NU-ASM / NU-FRE library: parameter
// validation, the Rect band of Eq. 4, the NUFFT kernel and its deconvolution,
// the per-axis transfer-function tables (Eq. 4 separable part, Eq. 5) and the
// FFT twiddles.  Everything here runs once per plan in FP64 (double-double
// where a phase can exceed 1e5 cycles).
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nuasm_internal.h"

namespace nuasm {

namespace {

using cd = std::complex<double>;
constexpr double kTwoPi = 6.283185307179586476925286766559;

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) ++l; return l; }

// exp(2 pi i c) for a phase c in cycles with |c| <= 1/2 (callers reduce first)
cd cis(double c) { double a = kTwoPi * c; return cd(std::cos(a), std::sin(a)); }

// exp(2 pi i num/den) for integers, reduced exactly
cd cis_ratio(int64_t num, int64_t den) {
    int64_t r = num % den;
    if (r < 0) r += den;
    if (2 * r > den) r -= den;
    return cis(double(r) / double(den));
}

double frac(double c) { return c - std::nearbyint(c); }

// z / lambda reduced mod 1 with a double-double quotient: the phase of
// exp(ikz) reaches 1e6 cycles, beyond what one rounded FP64 division resolves
// at the 1e-10 level.
double z_over_lambda_frac(double z, double lam) {
    double q = z / lam;
    double r = std::fma(-q, lam, z);          // exact remainder z - q lambda
    double ql = r / lam;
    return frac(q) + ql;
}

// Exponential-of-semicircle kernel phi(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1)),
// supported on |t| <= w/2 (Barnett, Magland, af Klinteberg 2019).
double es_kernel(double t, int w, double beta) {
    double s = 2.0 * t / w;
    if (std::fabs(s) > 1.0) return 0.0;
    return std::exp(beta * (std::sqrt(1.0 - s * s) - 1.0));
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the three-term recurrence).
void gauss_legendre(int n, double* x, double* wt) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// In-place radix-2 FFT (forward, exp(-2 pi i k n / L)), FP64, twiddles computed
// directly from the index so that no rounding accumulates.
void fft_host(std::vector<cd>* a) {
    const int64_t L = int64_t(a->size());
    std::vector<cd>& v = *a;
    for (int64_t i = 1, j = 0; i < L; ++i) {
        int64_t bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(v[i], v[j]);
    }
    std::vector<cd> roots(L / 2);
    for (int64_t t = 0; t < L / 2; ++t) roots[t] = cis_ratio(-t, L);
    for (int64_t len = 2; len <= L; len <<= 1) {
        int64_t step = L / len;
        for (int64_t i = 0; i < L; i += len)
            for (int64_t k = 0; k < len / 2; ++k) {
                cd u = v[i + k], t = v[i + k + len / 2] * roots[k * step];
                v[i + k] = u + t;
                v[i + k + len / 2] = u - t;
            }
    }
}

// Band of Eq. 4 along one axis as a frequency interval (see nuasm.h).
void band_limits(int n, double pitch, double lam, double z, double o, double* lo, double* hi) {
    const double s = n * pitch;
    if (z == 0.0) {
        if (std::fabs(o) <= s) { *lo = -INFINITY; *hi = INFINITY; }
        else { *lo = INFINITY; *hi = -INFINITY; }
        return;
    }
    const double sg = z > 0 ? 1.0 : -1.0;
    auto ginv = [&](double t) { return sg * t / (lam * std::sqrt(z * z + t * t)); };
    double a = ginv(o - s), b = ginv(o + s);
    *lo = a < b ? a : b;
    *hi = a < b ? b : a;
}

bool in_band(const nuasm_params_t& p, int np, int k, int axis) {
    if (p.kind != NUASM_KIND_ASM) return true;
    if (!p.band_auto) {
        double c = axis == 0 ? p.c_m : p.c_n;
        double w = axis == 0 ? p.w_m : p.w_n;
        return std::fabs(double(k) - c) <= w / 2.0;
    }
    double lo, hi;
    band_limits(p.n, p.pitch, p.lambda, p.z, axis == 0 ? p.ox : p.oy, &lo, &hi);
    double f = double(k) / (double(np) * p.pitch);
    return f >= lo && f <= hi;
}

}  // namespace

// ---------------------------------------------------------------- shared per-mode helpers
// (heap-free, so that the no-allocation solve can use them too)

// Gaussian kernel exp(-beta t^2), |t| <= w/2 (Greengard and Lee's gridding kernel)
double gaussian_kernel(double t, int w, double beta) {
    if (std::fabs(t) > 0.5 * w) return 0.0;
    return std::exp(-beta * t * t);
}

double kernel_value(const Geometry& g, double t) {
    return g.kernel == NUASM_KERNEL_GAUSSIAN ? gaussian_kernel(t, g.w, g.beta) : es_kernel(t, g.w, g.beta);
}

void make_quad(const Geometry& g, KernelQuad* qd) {
    qd->n = 2 * g.w + 48;
    double gx[KernelQuad::kMax], gw[KernelQuad::kMax];
    gauss_legendre(qd->n, gx, gw);
    for (int i = 0; i < qd->n; ++i) {
        qd->t[i] = (gx[i] + 1.0) * g.w / 4.0;              // [0, w/2]
        qd->f[i] = gw[i] * g.w / 4.0 * kernel_value(g, qd->t[i]);
    }
}

double phihat_at(const KernelQuad& qd, double nu) {
    double acc = 0.0;
    for (int i = 0; i < qd.n; ++i) acc += qd.f[i] * std::cos(kTwoPi * nu * qd.t[i]);
    return 2.0 * acc;
}

void asm_axis_factor(const nuasm_params_t& p, int np, int k, int axis, double* re, double* im) {
    *re = 0.0;
    *im = 0.0;
    if (!in_band(p, np, k, axis)) return;
    const double o = axis == 0 ? p.ox : p.oy;
    const double f = double(k) / (double(np) * p.pitch);
    const cd v = cis(frac(o * f - 0.5 * p.z * p.lambda * f * f));   // cycles
    *re = v.real();
    *im = v.imag();
}

void table_entry(const nuasm_params_t& p, const Geometry& g, int q, int type, double phihat, double hs_re,
                 double hs_im, double* re, double* im) {
    const int np = g.np;
    if (type == 3) {
        // type 1 forward then type 2 back: window phases and (-1)^k cancel
        const double dec = 1.0 / (phihat * phihat * np);
        *re = hs_re * dec;
        *im = hs_im * dec;
        return;
    }
    const int k = q < np / 2 ? q : q - np;
    const double dec = ((k & 1) ? -1.0 : 1.0) / phihat / np;
    const cd win1 = cis_ratio(-int64_t(k) * g.Lo, g.G);      // window origin on the 2N' grid
    const cd ctr1 = cis_ratio(-int64_t(k) * (g.n / 2), np);   // centred plane indices
    const cd f = (type == 1 ? win1 * ctr1 : std::conj(win1) * std::conj(ctr1)) * dec * cd(hs_re, hs_im);
    *re = f.real();
    *im = f.imag();
}

void constant_factor(const nuasm_params_t& p, double* re, double* im) {
    cd cst = cis(frac(z_over_lambda_frac(p.z, p.lambda)));
    if (p.kind == NUASM_KIND_FRESNEL) cst /= cd(0.0, p.lambda * p.z);
    *re = cst.real();
    *im = cst.imag();
}

void twiddle(int i, int G, double* re, double* im) {
    const cd v = cis_ratio(-i, G);
    *re = v.real();
    *im = v.imag();
}

double nonsep_rmax(const nuasm_params_t& p, const Geometry& g) {
    if (p.kind != NUASM_KIND_ASM || p.z == 0.0) return 0.0;
    const int np = g.np;
    double sx = 0.0, sy = 0.0;   // largest kept lambda^2 f^2 per axis
    for (int q = 0; q < np; ++q) {
        const int k = q < np / 2 ? q : q - np;
        const double f = double(k) / (double(np) * p.pitch);
        const double sv = p.lambda * p.lambda * f * f;
        if (in_band(p, np, k, 0) && sv > sx) sx = sv;
        if (in_band(p, np, k, 1) && sv > sy) sy = sv;
    }
    const double sm = sx + sy;
    const double qm = sm >= 1.0 ? 1.0 : sm / (1.0 + std::sqrt(1.0 - sm));
    return std::fabs(p.z / (2.0 * p.lambda)) * qm * qm;
}

bool kernel_shape(double tol, int prec, int kernel, int* w, double* beta) {
    if (!(tol > 0)) tol = prec == NUASM_PREC_F64 ? 1e-12 : 1e-6;
    int ww;
    if (kernel == NUASM_KERNEL_GAUSSIAN) {
        // aliasing exp(-pi^2 s^2) balanced against truncation exp(-w^2 / (8 s^2))
        // at s^2 = w / (2 sqrt(2) pi): error about exp(-1.11 w)
        ww = int(std::ceil(-std::log(tol) / 1.11 - 1e-9));
        if (ww < 2) ww = 2;
        *w = ww;
        *beta = std::sqrt(2.0) * M_PI / ww;   // 1 / (2 s^2)
        return ww <= kPolyMaxW;               // 26 taps: tol >= 3e-13
    }
    ww = int(std::ceil(-std::log10(tol) - 1e-9)) + 1;
    if (ww < 2) ww = 2;
    if (ww > 16) ww = 16;
    *w = ww;
    *beta = 2.30 * ww;   // shape parameter for upsampling factor 2
    return true;
}

nuasm_status validate(const nuasm_params_t& p0, int64_t m, nuasm_params_t* out) {
    nuasm_params_t p = p0;
    if (p.kind != NUASM_KIND_ASM && p.kind != NUASM_KIND_FRESNEL) return NUASM_EINVAL;
    if (p.prec != NUASM_PREC_F32_F64PHASE && p.prec != NUASM_PREC_F64) return NUASM_EINVAL;
    if (p.kernel != NUASM_KERNEL_ES && p.kernel != NUASM_KERNEL_GAUSSIAN) return NUASM_EINVAL;
    if (m < 0 || m > (int64_t(1) << 29)) return m < 0 ? NUASM_EINVAL : NUASM_EUNSUPPORTED;
    if (p.n < 2 || (p.n & 1)) return NUASM_EINVAL;
    if (!std::isfinite(p.pitch) || !(p.pitch > 0)) return NUASM_EINVAL;
    if (!std::isfinite(p.lambda) || !(p.lambda > 0)) return NUASM_EINVAL;
    if (!std::isfinite(p.z) || !std::isfinite(p.ox) || !std::isfinite(p.oy)) return NUASM_EINVAL;
    if (p.kind == NUASM_KIND_FRESNEL && p.z == 0.0) return NUASM_EINVAL;
    if (p.band_auto != 0 && p.band_auto != 1) return NUASM_EINVAL;
    if (!p.band_auto && p.kind == NUASM_KIND_ASM) {
        if (!std::isfinite(p.c_m) || !std::isfinite(p.c_n) || !std::isfinite(p.w_m) ||
            !std::isfinite(p.w_n) || p.w_m < 0 || p.w_n < 0)
            return NUASM_EINVAL;
    }
    if (std::isnan(p.tol) || p.tol < 0 || p.tol > 0.1) return NUASM_EINVAL;
    if (p.tol == 0) p.tol = p.prec == NUASM_PREC_F64 ? 1e-12 : 1e-6;
    if (p.tol < 1e-15) return NUASM_EINVAL;
    {
        int w;
        double beta;
        if (!kernel_shape(p.tol, p.prec, p.kernel, &w, &beta)) return NUASM_EUNSUPPORTED;
    }
    if (p.tile != 0 && p.tile != 16 && p.tile != 32 && p.tile != 64) return NUASM_EINVAL;
    if (p.interp_chunk != 0 && p.interp_chunk < 64) return NUASM_EINVAL;
    if (p.spread_chunk < -1 || (p.spread_chunk > 0 && p.spread_chunk < 32)) return NUASM_EINVAL;
    {
        int w;
        double beta;
        kernel_shape(p.tol, p.prec, p.kernel, &w, &beta);
        if (p.tile != 0 && p.tile < w - 1) return NUASM_EUNSUPPORTED;   // taps would reach two tiles away
    }
    if (p.n_pad != 0 && (p.n_pad < 2 * p.n || (p.n_pad & 1))) return NUASM_EINVAL;
    // what this build implements: power-of-two planes 16 <= N and N', N' <= 8192
    // (F32) / 4096 (F64); other even sizes are valid problems it does not run
    if (!is_pow2(p.n) || p.n < 16 || (p.n_pad != 0 && !is_pow2(p.n_pad))) return NUASM_EUNSUPPORTED;
    if (p.n_pad == 0) p.n_pad = 2 * p.n;
    const int np_max = p.prec == NUASM_PREC_F64 ? 4096 : 8192;
    if (p.n_pad > np_max) return NUASM_EUNSUPPORTED;
    *out = p;
    return NUASM_OK;
}

void band_range(const nuasm_params_t& p, int out[4]) {
    const int np = p.n_pad ? p.n_pad : 2 * p.n;
    for (int axis = 0; axis < 2; ++axis) {
        int lo = np / 2, hi = -np / 2 - 1;   // empty
        for (int k = -np / 2; k < np / 2; ++k)
            if (in_band(p, np, k, axis)) {
                if (k < lo) lo = k;
                if (k > hi) hi = k;
            }
        out[2 * axis] = lo;
        out[2 * axis + 1] = hi;
    }
}

Geometry make_geometry(const nuasm_params_t& p) {
    Geometry g{};
    g.n = p.n;
    g.np = p.n_pad;
    g.G = 2 * p.n_pad;
    g.logn = ilog2(p.n);
    g.lognp = ilog2(p.n_pad);
    g.kernel = p.kernel;
    kernel_shape(p.tol, p.prec, p.kernel, &g.w, &g.beta);
    g.h = (g.w + 1) / 2;
    g.W = 2 * p.n + 2 * g.h;
    g.Wp = (g.W + 31) & ~31;
    g.Lo = p.n_pad - p.n - g.h;
    // default tile: the largest side that still gives at least 608 tiles
    // (four CTAs per SM on 152 SMs), else the smallest
    g.T = p.tile;
    if (!g.T) {
        g.T = 16;
        for (int t : {64, 32}) {
            const int per_axis = (g.W + t - 1) / t;
            if (per_axis * per_axis >= 608) {
                g.T = t;
                break;
            }
        }
    }
    // a point's taps may reach only the next tile on each axis: w - 1 <= T
    while (g.T < g.w - 1) g.T *= 2;
    g.ntx = (g.W + g.T - 1) / g.T;
    g.ntiles = g.ntx * g.ntx;
    band_range(p, g.band);
    return g;
}

void phihat_table(const Geometry& g, double* out) {
    KernelQuad qd;
    make_quad(g, &qd);
    const int np = g.np;
    for (int q = 0; q < np; ++q) {
        const int k = q < np / 2 ? q : q - np;
        out[q] = phihat_at(qd, double(k) / g.G);
    }
}

void build_tables(const nuasm_params_t& p, const Geometry& g, HostTables* t, const double* phihat,
                  bool with_twiddles) {
    const int np = g.np, G = g.G;
    t->t1x = new double[2 * np];
    t->t1y = new double[2 * np];
    t->t2x = new double[2 * np];
    t->t2y = new double[2 * np];
    t->t3x = new double[2 * np];
    t->t3y = new double[2 * np];
    t->s = new double[np];
    t->tw = with_twiddles ? new double[2 * G] : nullptr;

    // deconvolution 1/phihat(k/G) by Gauss-Legendre quadrature of the truncated kernel
    // (geometry only: callers that keep it pass it in)
    std::vector<double> ph_own;
    if (!phihat) {
        ph_own.resize(np);
        phihat_table(g, ph_own.data());
        phihat = ph_own.data();
    }
    // separable transfer-function factor per axis (Eq. 4 or Eq. 5)
    std::vector<cd> hx(np), hy(np);
    for (int axis = 0; axis < 2; ++axis) {
        std::vector<cd>& hs = axis == 0 ? hx : hy;
        if (p.kind == NUASM_KIND_ASM) {
            for (int q = 0; q < np; ++q) {
                const int k = q < np / 2 ? q : q - np;
                double re, im;
                asm_axis_factor(p, np, k, axis, &re, &im);
                hs[q] = cd(re, im);
            }
        } else {
            // Hx(k) = pitch * sum_{m in [-N'/2, N'/2)} exp(i pi (m pitch + o)^2/(lambda z)) exp(-2 pi i k m / N')
            const double o = axis == 0 ? p.ox : p.oy;
            std::vector<cd> chirp(np);
            for (int i = 0; i < np; ++i) {
                const double xm = double(i - np / 2) * p.pitch + o;
                chirp[i] = cis(frac(xm * xm / (2.0 * p.lambda * p.z)));
            }
            fft_host(&chirp);
            for (int q = 0; q < np; ++q) {
                const int k = q < np / 2 ? q : q - np;
                hs[q] = p.pitch * ((k & 1) ? -1.0 : 1.0) * chirp[q];
            }
        }
    }
    double cre, cim;
    constant_factor(p, &cre, &cim);
    const cd cst(cre, cim);
    for (int q = 0; q < np; ++q) {
        const int k = q < np / 2 ? q : q - np;
        const double ph = phihat[q];
        const cd hyc = hy[q] * cst;
        // the arithmetic of table_entry, with the mode's phase factors formed once
        const double dec = ((k & 1) ? -1.0 : 1.0) / ph / np;
        const cd win1 = cis_ratio(-int64_t(k) * g.Lo, g.G);
        const cd ctr1 = cis_ratio(-int64_t(k) * (g.n / 2), np);
        const cd a1 = win1 * ctr1, a2 = std::conj(win1) * std::conj(ctr1);
        auto put = [](double* dst, int i, const cd& v) {
            dst[2 * i] = v.real();
            dst[2 * i + 1] = v.imag();
        };
        put(t->t1x, q, a1 * dec * hx[q]);
        put(t->t1y, q, a1 * dec * hyc);
        put(t->t2x, q, a2 * dec * hx[q]);
        put(t->t2y, q, a2 * dec * hyc);
        const double dec3 = 1.0 / (ph * ph * np);
        put(t->t3x, q, cd(hx[q].real() * dec3, hx[q].imag() * dec3));
        put(t->t3y, q, cd(hyc.real() * dec3, hyc.imag() * dec3));
        const double f = double(k) / (double(np) * p.pitch);
        t->s[q] = p.lambda * p.lambda * f * f;
    }
    t->rc = p.z / (2.0 * p.lambda);
    t->rmax = nonsep_rmax(p, g);
    fit_kernel_poly(g, &t->poly);
    if (t->tw)
        for (int i = 0; i < G; ++i) twiddle(i, G, &t->tw[2 * i], &t->tw[2 * i + 1]);
}

namespace {
int log2_of(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
}  // namespace

size_t table_bytes(const Geometry& g, bool f64, bool with_twiddles) {
    const size_t eb = f64 ? 16 : 8, sb = f64 ? sizeof(double) : 2 * sizeof(float);
    const size_t tw = with_twiddles ? size_t(g.G) + size_t(twp_entries(f64, log2_of(g.np))) : 0;
    return 6 * size_t(g.np) * eb + size_t(g.np) * sb + tw * eb;
}

void pack_twp(const double* tw, int logl, bool f64, void* dst) {
    size_t idx = 0;
    for (int le = 3; le <= 4; ++le) {
        const int nfull = logl / le, rem = logl % le, npass = nfull + (rem ? 1 : 0);
        for (int i = 1; i < npass; ++i) {
            const int lr = i < nfull ? le : rem, ns = 1 << (i * le);
            const int cnt = twp_per_k(f64, lr), sh = logl + 1 - i * le - lr;
            for (int k = 0; k < ns; ++k)
                for (int n = 0; n < cnt; ++n, ++idx) {
                    const int pw = f64 ? n + 1 : (n == 0 ? 1 : (lr == 2 ? 2 : 4));
                    const size_t t = size_t(k * pw) << sh;
                    if (f64) {
                        double* d = static_cast<double*>(dst);
                        d[2 * idx] = tw[2 * t];
                        d[2 * idx + 1] = tw[2 * t + 1];
                    } else {
                        float* d = static_cast<float*>(dst);
                        d[2 * idx] = float(tw[2 * t]);
                        d[2 * idx + 1] = float(tw[2 * t + 1]);
                    }
                }
        }
    }
}

// Device image of the tables: T1x T1y T2x T2y T3x T3y (complex, plan precision),
// s (double, or float hi/lo pairs), then the twiddles when present.
void pack_tables(const HostTables& t, const Geometry& g, bool f64, bool with_twiddles, void* dst) {
    const int np = g.np;
    const size_t eb = f64 ? 16 : 8;
    char* out = static_cast<char*>(dst);
    auto put_c = [&](size_t off, const double* src, int count) {
        if (f64) std::memcpy(out + off, src, sizeof(double) * 2 * count);
        else {
            float* d = reinterpret_cast<float*>(out + off);
            for (int i = 0; i < 2 * count; ++i) d[i] = float(src[i]);
        }
    };
    const double* six[6] = {t.t1x, t.t1y, t.t2x, t.t2y, t.t3x, t.t3y};
    for (int i = 0; i < 6; ++i) put_c(size_t(i) * np * eb, six[i], np);
    const size_t soff = 6 * size_t(np) * eb;
    if (f64) std::memcpy(out + soff, t.s, sizeof(double) * np);
    else {
        float* d = reinterpret_cast<float*>(out + soff);
        for (int i = 0; i < np; ++i) {
            const float hi = float(t.s[i]);
            d[2 * i] = hi;
            d[2 * i + 1] = float(t.s[i] - double(hi));
        }
    }
    if (with_twiddles && t.tw) {
        const size_t toff = soff + size_t(np) * (f64 ? sizeof(double) : 2 * sizeof(float));
        put_c(toff, t.tw, g.G);
        pack_twp(t.tw, log2_of(np), f64, out + toff + size_t(g.G) * eb);
    }
}

int choose_nonsep_mode(const nuasm_params_t& p, double rmax) {
    if (p.kind != NUASM_KIND_ASM || p.z == 0.0) return 0;
    if (p.prec == NUASM_PREC_F64 || rmax <= 0.5) return 1;
    return 2;
}

// Chebyshev interpolation of each tap phi(i + f - w/2), f in [0, 1), at
// Chebyshev nodes of x = 2f - 1, converted to monomial coefficients in x (the
// coefficients stay O(1), so Horner's rule is as accurate as direct
// evaluation of the exponential: FP32 at degree w + 1, FP64 at kPoly64Deg).
template <typename Poly, typename T>
void fit_poly(const Geometry& g, int d, Poly* kp) {
    std::memset(kp, 0, sizeof(*kp));
    if (d > kPolyMaxD - 1) d = kPolyMaxD - 1;
    kp->deg = d;
    const int K = 2 * d + 2;
    double xn[2 * kPolyMaxD + 2];
    for (int k = 0; k < K; ++k) xn[k] = std::cos(M_PI * (k + 0.5) / K);
    // monomial coefficients of the Chebyshev polynomials T_0..T_d
    double Tm[kPolyMaxD][kPolyMaxD] = {};
    Tm[0][0] = 1.0;
    if (d >= 1) Tm[1][1] = 1.0;
    for (int j = 2; j <= d; ++j)
        for (int m = 0; m <= d; ++m)
            Tm[j][m] = (m > 0 ? 2.0 * Tm[j - 1][m - 1] : 0.0) - Tm[j - 2][m];
    for (int i = 0; i < g.w && i < kPolyMaxW; ++i) {
        double cheb[kPolyMaxD] = {};
        for (int k = 0; k < K; ++k) {
            const double f = 0.5 * (xn[k] + 1.0);
            const double val = kernel_value(g, i + f - 0.5 * g.w);
            for (int j = 0; j <= d; ++j) cheb[j] += val * std::cos(j * M_PI * (k + 0.5) / K);
        }
        for (int j = 0; j <= d; ++j) cheb[j] *= (j == 0 ? 1.0 : 2.0) / K;
        for (int m = 0; m <= d; ++m) {
            double acc = 0.0;
            for (int j = m; j <= d; ++j) acc += cheb[j] * Tm[j][m];
            kp->c[i][m] = T(acc);
        }
    }
}

void fit_kernel_poly(const Geometry& g, KernelPoly* kp) { fit_poly<KernelPoly, float>(g, g.w + 1, kp); }
void fit_kernel_poly64(const Geometry& g, KernelPoly64* kp) { fit_poly<KernelPoly64, double>(g, kPoly64Deg, kp); }

void split_kernel_poly64(const KernelPoly64& kp, KernelPolyDF* out) {
    for (int i = 0; i < kPolyMaxW; ++i)
        for (int k = 0; k < kPolyMaxD; ++k) {
            const float hi = float(kp.c[i][k]);
            out->c[i][k] = float2{hi, float(kp.c[i][k] - double(hi))};
        }
}

void free_tables(HostTables* t) {
    delete[] t->t1x; delete[] t->t1y; delete[] t->t2x; delete[] t->t2y; delete[] t->t3x; delete[] t->t3y;
    delete[] t->s; delete[] t->tw;
    std::memset(t, 0, sizeof(*t));
}

}  // namespace nuasm
