// FFT passes of the NU-ASM / NU-FRE pipeline.
//
// Every transform here has length N' (the padded plane size).  The length-2N'
// transforms of the oversampled NUFFT grid are split into their even and odd
// halves, each an N'-point transform:
//   forward (window -> modes, type 1):  B(2k')   = FFT_N'[x(n) + x(n+N')](k'),
//                                       B(2k'+1) = FFT_N'[(x(n) - x(n+N')) e^{-2 pi i n/2N'}](k');
//   inverse (modes -> window, type 2):  y(2u')   = IFFT_N'[Y(q)](u'),
//                                       y(2u'+1) = IFFT_N'[Y(q) e^{2 pi i p(q)/2N'}](u'),
// where p(q) is the 2N'-grid bin of natural N'-bin q.  Only the modes
// k in [-N'/2, N'/2) and the window rows [0, W) are ever produced.
//
// Type 1 (Eq. 6):  window --col_fwd_fold--> A (N' x W) --row_t1--> B (N' x N)
//                  --col_inv--> u2 (N x N).  row_t1 fuses the forward row
//                  transform, the deconvolution, H (Eq. 4 / Eq. 5) and the
//                  inverse row transform.
// Type 2 (Eq. 9):  u1 --col_fwd--> B (N' x N) --row_t2--> A (N' x W)
//                  --col_inv_fold--> window.
//
// The non-separable part of the ASM phase is evaluated per mode:
//   z sqrt(1/lambda^2 - |f|^2) = z/lambda - (z lambda/2)|f|^2 - (z/(2 lambda)) q^2,
//   q = s / (1 + sqrt(1 - s)),  s = lambda^2 |f|^2,
// an exact rearrangement whose first two terms are separable (folded into the
// per-axis tables in FP64 on the host) and whose last term is small; it is
// computed in FP64 (F64 plans) or double-float FP32 (F32 plans), reduced mod 1
// and passed to sincospi.  Evanescent modes (s >= 1) are zeroed.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft_engine.cuh"
#include "nuasm_internal.h"

namespace nuasm {

namespace {

constexpr int kE = 16;   // elements per thread in every engine

// --------------------------------------------------------------- non-separable ASM factor
__device__ __forceinline__ float2 asm_nonsep(const float2* __restrict__ s, int qx, int qy, float rc_hi,
                                             float rc_lo) {
    const float2 a = __ldg(&s[qx]), b = __ldg(&s[qy]);
    df sv = df_add({a.x, a.y}, {b.x, b.y});
    if (sv.hi >= 1.f) return make_float2(0.f, 0.f);
    df one_m = df_add({1.f, 0.f}, {-sv.hi, -sv.lo});
    df root = df_sqrt(one_m);
    df den = df_add({1.f, 0.f}, root);
    df q = df_div(sv, den);
    df r = df_mul({rc_hi, rc_lo}, df_mul(q, q));
    float ri = rintf(r.hi);
    float fr = (r.hi - ri) + r.lo;        // exact leading difference, then the tail
    float sn, cs;
    sincospif(-2.f * fr, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ double2 asm_nonsep(const double* __restrict__ s, int qx, int qy, double rc,
                                              double /*unused*/) {
    const double sv = __ldg(&s[qx]) + __ldg(&s[qy]);
    if (sv >= 1.0) return make_double2(0.0, 0.0);
    const double q = sv / (1.0 + sqrt(1.0 - sv));
    const double r = rc * q * q;
    const double fr = r - rint(r);
    double sn, cs;
    sincospi(-2.0 * fr, &sn, &cs);
    return make_double2(cs, sn);
}

template <typename V> struct STable;
template <> struct STable<float2> { using type = float2; };
template <> struct STable<double2> { using type = double; };

struct RowArgs {
    int n, np, W, Wp, logNp, logG;
    int rows_per_cta, log_rows;
    int asm_kind;          // 1: ASM non-separable factor; 0: Fresnel (rank one)
    double rc;             // z / (2 lambda)
    float rc_hi, rc_lo;
};

__device__ __forceinline__ float2 nonsep(const float2* __restrict__ s, int qx, int qy, const RowArgs& a) {
    return asm_nonsep(s, qx, qy, a.rc_hi, a.rc_lo);
}
__device__ __forceinline__ double2 nonsep(const double* __restrict__ s, int qx, int qy, const RowArgs& a) {
    return asm_nonsep(s, qx, qy, a.rc, 0.0);
}


// --------------------------------------------------------------- type-1 row pass
// One CTA = `rows_per_cta` rows r of A (ky bin r): forward 2N' transform of the
// window row restricted to the kept modes (two folded N'-point FFTs), multiply
// by T1x(kx) T1y(ky) E(kx, ky), inverse N'-point FFT, keep the N outputs.
template <typename V>
__global__ void __launch_bounds__(512) row_t1_kernel(const V* __restrict__ A, V* __restrict__ B,
                                                     const V* __restrict__ tx, const V* __restrict__ ty,
                                                     const typename STable<V>::type* __restrict__ s,
                                                     const V* __restrict__ tw, RowArgs a) {
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    const int np = a.np, rows = a.rows_per_cta;
    V* M = S + spad_size<V>(np * rows);
    const int r0 = blockIdx.x * rows;
    const int W = a.W, Wp = a.Wp, half = np / 2;

    auto x_at = [&](int c, int p) -> V {
        return p < W ? A[size_t(r0 + c) * Wp + p] : CTraits<V>::zero();
    };
    for (int sgn = 0; sgn < 2; ++sgn) {
        auto load = [&](int p, int c) -> V {
            V u = x_at(c, p), t = x_at(c, p + np);
            if (sgn == 0) return cadd(u, t);
            return cmul(csub(u, t), __ldg(&tw[p]));
        };
        auto store = [&](int pk, int c, V v) {
            const int pb = 2 * pk + sgn;
            if (pb < half) M[c * np + pb] = v;
            else if (pb >= 3 * half) M[c * np + pb - np] = v;
        };
        block_fft<V, -1, kE, true>(S, a.logNp, a.log_rows, tw, a.logG, load, store);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * np; idx += blockDim.x) {
        const int c = idx >> a.logNp, q = idx & (np - 1);
        const int r = r0 + c;
        V f = cmul(__ldg(&tx[q]), __ldg(&ty[r]));
        if (a.asm_kind && (f.x != 0 || f.y != 0)) f = cmul(f, nonsep(s, q, r, a));
        M[idx] = cmul(M[idx], f);
    }
    __syncthreads();
    auto load = [&](int p, int c) -> V { return M[c * np + p]; };
    auto store = [&](int p, int c, V v) {
        if (p < a.n) B[size_t(r0 + c) * a.n + p] = v;
    };
    block_fft<V, +1, kE, true>(S, a.logNp, a.log_rows, tw, a.logG, load, store);
}

// --------------------------------------------------------------- type-2 row pass
// One CTA = rows r of B (ky bin r, N values): forward N'-point FFT, multiply
// by T2x T2y E, then the inverse 2N' transform onto the window row (even and
// odd outputs as two N'-point FFTs), keeping the W window entries.
template <typename V>
__global__ void __launch_bounds__(512) row_t2_kernel(const V* __restrict__ B, V* __restrict__ A,
                                                     const V* __restrict__ tx, const V* __restrict__ ty,
                                                     const typename STable<V>::type* __restrict__ s,
                                                     const V* __restrict__ tw, RowArgs a) {
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    const int np = a.np, rows = a.rows_per_cta;
    V* M = S + spad_size<V>(np * rows);
    const int r0 = blockIdx.x * rows;
    const int n = a.n, W = a.W, Wp = a.Wp, half = np / 2;
    {
        auto load = [&](int p, int c) -> V {
            return p < n ? B[size_t(r0 + c) * n + p] : CTraits<V>::zero();
        };
        auto store = [&](int p, int c, V v) { M[c * np + p] = v; };
        block_fft<V, -1, kE, true>(S, a.logNp, a.log_rows, tw, a.logG, load, store);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * np; idx += blockDim.x) {
        const int c = idx >> a.logNp, q = idx & (np - 1);
        const int r = r0 + c;
        V f = cmul(__ldg(&tx[q]), __ldg(&ty[r]));
        if (a.asm_kind && (f.x != 0 || f.y != 0)) f = cmul(f, nonsep(s, q, r, a));
        M[idx] = cmul(M[idx], f);
    }
    __syncthreads();
    for (int sgn = 0; sgn < 2; ++sgn) {
        auto load = [&](int q, int c) -> V {
            V y = M[c * np + q];
            if (sgn == 0) return y;
            const int pg = q < half ? q : q + np;
            return cmul(y, cconj(__ldg(&tw[pg])));
        };
        auto store = [&](int k, int c, V v) {
            const int u = 2 * k + sgn;
            if (u < W) A[size_t(r0 + c) * Wp + u] = v;
        };
        block_fft<V, +1, kE, true>(S, a.logNp, a.log_rows, tw, a.logG, load, store);
    }
}

// --------------------------------------------------------------- column passes
struct ColArgs {
    int n, np, W, Wp, logNp, logG;
    int cols_per_cta, log_cols;
    int ncols;             // columns to transform
};

enum ColMode { COL_FWD_FOLD = 0, COL_INV = 1, COL_FWD = 2, COL_INV_FOLD = 3 };

// One CTA = C adjacent columns (blockIdx.x) and, for the folded modes, one
// half (blockIdx.y: 0 even, 1 odd).
template <typename V, int MODE>
__global__ void __launch_bounds__(512) col_kernel(const V* __restrict__ src, V* __restrict__ dst,
                                                  const V* __restrict__ tw, ColArgs a) {
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    const int col0 = blockIdx.x * a.cols_per_cta;
    const int sgn = blockIdx.y;
    const int np = a.np, half = np / 2, W = a.W, Wp = a.Wp, n = a.n;
    const V zero = CTraits<V>::zero();
    if (MODE == COL_FWD_FOLD) {
        // src: window (W x Wp); dst: A (N' x Wp), kept modes in natural N'-bin rows
        auto load = [&](int p, int c) -> V {
            const int col = col0 + c;
            if (col >= W) return zero;
            V u = p < W ? src[size_t(p) * Wp + col] : zero;
            V t = p + np < W ? src[size_t(p + np) * Wp + col] : zero;
            if (sgn == 0) return cadd(u, t);
            return cmul(csub(u, t), __ldg(&tw[p]));
        };
        auto store = [&](int pk, int c, V v) {
            const int col = col0 + c;
            const int pb = 2 * pk + sgn;
            int r = -1;
            if (pb < half) r = pb;
            else if (pb >= 3 * half) r = pb - np;
            if (r >= 0 && col < W) dst[size_t(r) * Wp + col] = v;
        };
        block_fft<V, -1, kE, false>(S, a.logNp, a.log_cols, tw, a.logG, load, store);
    } else if (MODE == COL_INV) {
        // src: B (N' x N); dst: u2 (N x N)
        auto load = [&](int p, int c) -> V { return src[size_t(p) * n + col0 + c]; };
        auto store = [&](int p, int c, V v) {
            if (p < n) dst[size_t(p) * n + col0 + c] = v;
        };
        block_fft<V, +1, kE, false>(S, a.logNp, a.log_cols, tw, a.logG, load, store);
    } else if (MODE == COL_FWD) {
        // src: u1 (N x N); dst: B (N' x N)
        auto load = [&](int p, int c) -> V { return p < n ? src[size_t(p) * n + col0 + c] : zero; };
        auto store = [&](int p, int c, V v) { dst[size_t(p) * n + col0 + c] = v; };
        block_fft<V, -1, kE, false>(S, a.logNp, a.log_cols, tw, a.logG, load, store);
    } else {
        // src: A (N' x Wp); dst: window (W x Wp)
        auto load = [&](int q, int c) -> V {
            const int col = col0 + c;
            if (col >= W) return zero;
            V y = src[size_t(q) * Wp + col];
            if (sgn == 0) return y;
            const int pg = q < half ? q : q + np;
            return cmul(y, cconj(__ldg(&tw[pg])));
        };
        auto store = [&](int k, int c, V v) {
            const int col = col0 + c;
            const int u = 2 * k + sgn;
            if (u < W && col < W) dst[size_t(u) * Wp + col] = v;
        };
        block_fft<V, +1, kE, false>(S, a.logNp, a.log_cols, tw, a.logG, load, store);
    }
}

int ilog2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

RowArgs row_args(const nuasm_plan_s* P) {
    const Geometry& g = P->g;
    RowArgs a{};
    a.n = g.n; a.np = g.np; a.W = g.W; a.Wp = g.Wp;
    a.logNp = g.lognp; a.logG = g.lognp + 1;
    // at least 128 threads per CTA: rows_per_cta * N' / 16 >= 128
    int rows = 2048 / g.np;
    if (rows < 1) rows = 1;
    if (rows > g.np) rows = g.np;
    a.rows_per_cta = rows;
    a.log_rows = ilog2i(rows);
    a.asm_kind = P->p.kind == NUASM_KIND_ASM ? 1 : 0;
    a.rc = P->rc;
    a.rc_hi = float(P->rc);
    a.rc_lo = float(P->rc - double(a.rc_hi));
    return a;
}

template <typename V> size_t row_smem(const RowArgs& a) {
    return (spad_size<V>(a.np * a.rows_per_cta) + size_t(a.np) * a.rows_per_cta) * sizeof(V);
}

ColArgs col_args(const nuasm_plan_s* P, int ncols) {
    const Geometry& g = P->g;
    ColArgs a{};
    a.n = g.n; a.np = g.np; a.W = g.W; a.Wp = g.Wp;
    a.logNp = g.lognp; a.logG = g.lognp + 1;
    const int budget = P->f64 ? 4096 : 8192;    // elements per CTA (64 KB)
    int c = budget / g.np;
    if (c > 16) c = 16;
    if (c < 1) c = 1;
    a.cols_per_cta = c;
    a.log_cols = ilog2i(c);
    a.ncols = ncols;
    return a;
}

template <typename V> size_t col_smem(const ColArgs& a) {
    return size_t(spad_size<V>(a.np * a.cols_per_cta)) * sizeof(V);
}

template <typename K> cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

template <typename V, int MODE>
cudaError_t launch_col(const nuasm_plan_s* P, const void* src, void* dst, int ncols, int halves,
                       cudaStream_t st) {
    ColArgs a = col_args(P, ncols);
    const size_t sm = col_smem<V>(a);
    cudaError_t e = set_smem(col_kernel<V, MODE>, sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + a.cols_per_cta - 1) / a.cols_per_cta, halves);
    const int threads = (a.np * a.cols_per_cta) / kE;
    col_kernel<V, MODE><<<grid, threads, sm, st>>>(static_cast<const V*>(src), static_cast<V*>(dst),
                                                   static_cast<const V*>(P->d.tw), a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_fwd_fold(const nuasm_plan_s* P, cudaStream_t s) {
    if (P->f64) return launch_col<double2, COL_FWD_FOLD>(P, P->d.win, P->d.bufA, P->g.W, 2, s);
    return launch_col<float2, COL_FWD_FOLD>(P, P->d.win, P->d.bufA, P->g.W, 2, s);
}

cudaError_t launch_col_inv(const nuasm_plan_s* P, void* u2, cudaStream_t s) {
    if (P->f64) return launch_col<double2, COL_INV>(P, P->d.bufB, u2, P->g.n, 1, s);
    return launch_col<float2, COL_INV>(P, P->d.bufB, u2, P->g.n, 1, s);
}

cudaError_t launch_col_fwd(const nuasm_plan_s* P, const void* u1, cudaStream_t s) {
    if (P->f64) return launch_col<double2, COL_FWD>(P, u1, P->d.bufB, P->g.n, 1, s);
    return launch_col<float2, COL_FWD>(P, u1, P->d.bufB, P->g.n, 1, s);
}

cudaError_t launch_col_inv_fold(const nuasm_plan_s* P, cudaStream_t s) {
    if (P->f64) return launch_col<double2, COL_INV_FOLD>(P, P->d.bufA, P->d.win, P->g.W, 2, s);
    return launch_col<float2, COL_INV_FOLD>(P, P->d.bufA, P->d.win, P->g.W, 2, s);
}

template <typename V>
static cudaError_t launch_row_impl(const nuasm_plan_s* P, int type, cudaStream_t st) {
    RowArgs a = row_args(P);
    const size_t sm = row_smem<V>(a);
    using ST = typename STable<V>::type;
    const int threads = (a.np * a.rows_per_cta) / kE;
    const int blocks = a.np / a.rows_per_cta;
    const V* tw = static_cast<const V*>(P->d.tw);
    const ST* s = static_cast<const ST*>(P->d.s);
    cudaError_t e;
    if (type == 1) {
        e = set_smem(row_t1_kernel<V>, sm);
        if (e != cudaSuccess) return e;
        row_t1_kernel<V><<<blocks, threads, sm, st>>>(static_cast<const V*>(P->d.bufA),
                                                      static_cast<V*>(P->d.bufB),
                                                      static_cast<const V*>(P->d.t1x),
                                                      static_cast<const V*>(P->d.t1y), s, tw, a);
    } else {
        e = set_smem(row_t2_kernel<V>, sm);
        if (e != cudaSuccess) return e;
        row_t2_kernel<V><<<blocks, threads, sm, st>>>(static_cast<const V*>(P->d.bufB),
                                                      static_cast<V*>(P->d.bufA),
                                                      static_cast<const V*>(P->d.t2x),
                                                      static_cast<const V*>(P->d.t2y), s, tw, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_row_t1(const nuasm_plan_s* P, cudaStream_t s) {
    return P->f64 ? launch_row_impl<double2>(P, 1, s) : launch_row_impl<float2>(P, 1, s);
}

cudaError_t launch_row_t2(const nuasm_plan_s* P, cudaStream_t s) {
    return P->f64 ? launch_row_impl<double2>(P, 2, s) : launch_row_impl<float2>(P, 2, s);
}

}  // namespace nuasm
