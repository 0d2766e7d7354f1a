// FFT passes of the NU-ASM / NU-FRE pipeline (kernel templates; instantiated
// per precision and per N' in passes_{row,col}_{f32,f64}.cu).
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
// The non-separable part of the ASM phase:
//   z sqrt(1/lambda^2 - |f|^2) = z/lambda - (z lambda/2)|f|^2 - (z/(2 lambda)) q^2,
//   q = s / (1 + sqrt(1 - s)),  s = lambda^2 |f|^2,
// an exact rearrangement whose first two terms are separable (folded into the
// per-axis tables in FP64 on the host) and whose last term r is small.  A plan
// tabulates E = exp(-2 pi i r) once in FP64 over |kx|, |ky| in [0, N'/2]
// (E depends on |f|^2 only); without the table (served requests, the
// allocation-free solve) r is computed per mode in FP64 (F64 plans), with FP32
// fast-math intrinsics when the largest |r| is at most 1/2 cycle (phase error
// below 2e-6 rad), else in double-float FP32 reduced mod 1 and passed to
// sincospi.  Evanescent modes (s >= 1) are zeroed either way.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "fft_engine.cuh"
#include "nuasm_internal.h"
#include "tma.cuh"

namespace nuasm {
namespace passes {

// --------------------------------------------------------------- launch configuration
template <typename V> struct Prec;
#ifndef NUASM_ROW_REGS
#define NUASM_ROW_REGS 64   // FP32 register budget per thread that sets the row passes' CTAs per SM
#endif
#ifndef NUASM_COL_BUDGET
#define NUASM_COL_BUDGET 8192   // FP32 column passes: complex elements per CTA (columns = budget / N')
#endif
// FP64 passes run at the FP64 pipe's pace, so small planes want many CTAs:
// measured on the N' = 128 plane (C1), 2^9 elements per row-pass CTA and 512
// per column-pass CTA against 2^11 and 4096: row_t1 57 -> 33 us, the column
// passes 24 -> 16 and 17 -> 11 us (N' = 512: 440 -> 412 us per solve); the
// same configuration as before at N' = 4096
#ifndef NUASM_COL_BUDGET64
#define NUASM_COL_BUDGET64 512    // FP64 column passes: complex elements per CTA
#endif
#ifndef NUASM_ROW_LOGBUDGET64
#define NUASM_ROW_LOGBUDGET64 9   // FP64 row passes: log2 of the complex elements per CTA
#endif
template <> struct Prec<float2> {
    static constexpr bool f64 = false;
    static constexpr int col_e = 16, col_budget = NUASM_COL_BUDGET;   // elements per thread / per CTA
    static constexpr int col_cmax = 16;                               // columns per CTA at most
    static constexpr int row_logbudget = 11;                          // rows per CTA = 2^11 / N'
    static constexpr int regs = 64;
    static constexpr int row_regs = NUASM_ROW_REGS;
};
template <> struct Prec<double2> {
    static constexpr bool f64 = true;
    static constexpr int col_e = 8, col_budget = NUASM_COL_BUDGET64, col_cmax = 16;
    static constexpr int row_logbudget = NUASM_ROW_LOGBUDGET64;
    static constexpr int regs = 128;
    static constexpr int row_regs = 128;
};

// double-float passes of FP64 plans: the FP64 row configuration (16-byte
// elements, as complex128); column CTAs of up to NUASM_DF_COL_BUDGET elements
// and NUASM_DF_COL_CMAX columns, NUASM_DF_COL_E elements per thread
#ifndef NUASM_DF_COL_E
#define NUASM_DF_COL_E 8
#endif
#ifndef NUASM_DF_COL_BUDGET
#define NUASM_DF_COL_BUDGET 8192
#endif
#ifndef NUASM_DF_COL_CMAX
#define NUASM_DF_COL_CMAX 4
#endif
template <> struct Prec<dfc> : Prec<double2> {
    static constexpr int col_e = NUASM_DF_COL_E, col_budget = NUASM_DF_COL_BUDGET, col_cmax = NUASM_DF_COL_CMAX;
};

template <typename V, int LOGNP> struct RowCfg {
    static constexpr int NP = 1 << LOGNP;
    static constexpr int LB = Prec<V>::row_logbudget;
    static constexpr int LOGROWS = LOGNP >= LB ? 0 : (LB - LOGNP > LOGNP ? LOGNP : LB - LOGNP);
    static constexpr int ROWS = 1 << LOGROWS;
    // merged even/odd engines (two sequences per row in one pass sequence)
    static constexpr bool MERGE = !Prec<V>::f64 && LOGNP <= 12;
    static constexpr int EF = (!Prec<V>::f64 && LOGNP >= 13) ? 16 : 8;   // single-sequence engines
    static constexpr int EM = 16;                                         // merged engines
    static constexpr int P = (NP * ROWS) / EF;
    static constexpr int MINB = (65536 / (P * Prec<V>::row_regs)) > 0 ? 65536 / (P * Prec<V>::row_regs) : 1;
    static constexpr int SEQ = MERGE ? 2 * ROWS : ROWS;                  // sequences in the work buffer
    // The mode buffer M (NP x ROWS) between the forward and inverse transforms
    // lives inside the work buffer when the engines are merged (the forward
    // transform's last pass writes it after its last read of the buffer, the
    // inverse one's first pass reads it all before its first write); the
    // sequential engines read it twice, so it gets its own space.
    static size_t smem() {
        return (size_t(spad_size<V>(NP * SEQ)) + (MERGE ? size_t(0) : size_t(NP) * ROWS)) * sizeof(V);
    }
};

#ifndef NUASM_COL_FWD_BUDGET
#define NUASM_COL_FWD_BUDGET NUASM_COL_BUDGET   // FP32 budget of the type-2 forward column pass
#endif
template <typename V, int LOGNP, int MODE = 0> struct ColCfg {
    static constexpr int NP = 1 << LOGNP;
    static constexpr int E = Prec<V>::col_e;
    static constexpr int BUDGET = (MODE == 2 && !Prec<V>::f64) ? NUASM_COL_FWD_BUDGET : Prec<V>::col_budget;
    static constexpr int CRAW = BUDGET / NP;
    static constexpr int C = CRAW > Prec<V>::col_cmax ? Prec<V>::col_cmax : (CRAW < 1 ? 1 : CRAW);
    static constexpr int LOGC = Log2<C>::v;
    static constexpr int P = (NP * C) / E;
    static constexpr int MINB = (65536 / (P * Prec<V>::regs)) > 0 ? 65536 / (P * Prec<V>::regs) : 1;
    static size_t smem() { return size_t(spad_size<V>(NP * C)) * sizeof(V); }
};

template <typename V> struct STable;
template <> struct STable<float2> { using type = float2; };
template <> struct STable<double2> { using type = double; };
template <> struct STable<dfc> { using type = double; };

// Global-memory element type of a pass's register type and the conversions
// between them: the identity, except for double-float registers over FP64
// arrays (scale s: the arrays hold the values times 2^s, so that a CTA's data
// stays in the float range).
template <typename V> struct Mem {
    using type = V;
    static constexpr bool scaled = false;
    __device__ static V ld(V x, int) { return x; }
    __device__ static V st(V v, int) { return v; }
};
template <> struct Mem<dfc> {
    using type = double2;
    static constexpr bool scaled = true;
    __device__ static dfc ld(double2 x, int sc) { return dfc{dfr_split(x.x, sc), dfr_split(x.y, sc)}; }
    __device__ static double2 st(dfc v, int sc) { return make_double2(dfr_to_double(v.x, sc), dfr_to_double(v.y, sc)); }
};
template <typename V> using MemT = typename Mem<V>::type;

__device__ __forceinline__ bool nonzero(float2 v) { return v.x != 0.f || v.y != 0.f; }
__device__ __forceinline__ bool nonzero(double2 v) { return v.x != 0.0 || v.y != 0.0; }
__device__ __forceinline__ bool nonzero(dfc v) { return v.x.hi != 0.f || v.y.hi != 0.f; }

// exponent k with 2^k <= |x| < 2^(k+1) (-1023 for zeros and subnormals)
__device__ __forceinline__ int dexp2(double x) {
    return (int(static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff) - 1023;
}

// The CTA's scale for double-float registers: the largest exponent among the
// n elements at stride 1 of the rows r0 .. r0 + rows - 1 of an FP64 array
// (row pitch `pitch`), clamped to the normal range; 0 for other types.  All
// threads call it; it synchronises the block.
template <typename V>
__device__ __forceinline__ int cta_scale(const MemT<V>* __restrict__ x, int r0, int rows, int n, int pitch) {
    if constexpr (!Mem<V>::scaled) {
        return 0;
    } else {
        __shared__ int emax;
        if (threadIdx.x == 0) emax = -1023;
        __syncthreads();
        int em = -1023;
        for (int i = threadIdx.x; i < rows * n; i += blockDim.x) {
            const int row = i / n, p = i - row * n;
            const double2 v = x[size_t(r0 + row) * pitch + p];
            em = max(em, max(dexp2(v.x), dexp2(v.y)));
        }
        em = __reduce_max_sync(0xffffffffu, em);
        if ((threadIdx.x & 31) == 0) atomicMax(&emax, em);
        __syncthreads();
        return min(max(emax, -1022), 1023);
    }
}

struct RowArgs {
    int n, W, Wp;
    int nonsep;            // 0: none (Fresnel, z = 0); 1: plain (FP32 or FP64); 2: double-float FP32
    double rc;             // z / (2 lambda)
    float rc_hi, rc_lo;
    const void* etab;      // E(|kx|, |ky|) table of the plan precision, or null (E evaluated per mode)
    const void* etab2;     // type 2: T2x(kx) E(|kx|, |ky|), rows of N' entries, or null
    int ep;                // entries per table row
    int np;                // N'
};

struct ColArgs {
    int n, W, Wp;
};

// --------------------------------------------------------------- non-separable ASM factor
__device__ __forceinline__ float2 nonsep_factor(float2 sa, float2 sb, const RowArgs& a) {
    float fr;
    if (a.nonsep == 1) {
        // |r| <= 1/2 cycle: fast-math evaluation, phase error below 2e-6 rad
        const float sv = sa.x + sb.x;
        if (sv >= 1.f) return make_float2(0.f, 0.f);
        const float t = 1.f - sv;
        const float q = __fdividef(sv, 1.f + t * rsqrtf(t));
        const float r = a.rc_hi * q * q;
        float sn, cs;
        __sincosf(-6.28318530717958647692f * (r - rintf(r)), &sn, &cs);
        return make_float2(cs, sn);
    } else {
        df sv = df_add({sa.x, sa.y}, {sb.x, sb.y});
        if (sv.hi >= 1.f) return make_float2(0.f, 0.f);
        df root = df_sqrt(df_add({1.f, 0.f}, {-sv.hi, -sv.lo}));
        df q = df_div(sv, df_add({1.f, 0.f}, root));
        df r = df_mul({a.rc_hi, a.rc_lo}, df_mul(q, q));
        fr = (r.hi - rintf(r.hi)) + r.lo;
    }
    float sn, cs;
    sincospif(-2.f * fr, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ double2 nonsep_factor(double sa, double sb, const RowArgs& a) {
    const double sv = sa + sb;
    if (sv >= 1.0) return make_double2(0.0, 0.0);
    const double q = sv / (1.0 + sqrt(1.0 - sv));
    const double r = a.rc * q * q;
    double sn, cs;
    sincospi(-2.0 * (r - rint(r)), &sn, &cs);
    return make_double2(cs, sn);
}

// Tx(q) Ty(r) E(q, r): the per-mode factor applied between the row transforms.
// A row's Ty(r) and s(r) (or its row of the E table) are loaded once per row
// (RowConst) and passed in.  E depends on |f|^2 only, so the table holds the
// quadrant |kx|, |ky| in [0, N'/2]; natural bin q maps to |k| = min(q, N' - q).
template <typename V> struct RowConst {
    V ty;
    typename STable<V>::type s;
    const MemT<V>* erow;
};

template <typename V>
__device__ __forceinline__ RowConst<V> row_const(int r, const MemT<V>* __restrict__ ty,
                                                 const typename STable<V>::type* __restrict__ s, const RowArgs& a) {
    const MemT<V>* erow = nullptr;
    if (a.etab) erow = static_cast<const MemT<V>*>(a.etab) + size_t(min(r, a.np - r)) * a.ep;
    return RowConst<V>{Mem<V>::ld(__ldg(&ty[r]), 0), __ldg(&s[r]), erow};
}

template <typename V>
__device__ __forceinline__ V mode_factor(int q, const RowConst<V>& rc, const MemT<V>* __restrict__ tx,
                                         const typename STable<V>::type* __restrict__ s, const RowArgs& a) {
    V f = cmul(Mem<V>::ld(__ldg(&tx[q]), 0), rc.ty);
    if (rc.erow) {
        f = cmul(f, Mem<V>::ld(__ldg(&rc.erow[min(q, a.np - q)]), 0));   // both loads in flight together
    } else if (a.nonsep && nonzero(f)) {
        f = cmul(f, Mem<V>::ld(nonsep_factor(__ldg(&s[q]), rc.s, a), 0));
    }
    return f;
}

template <typename V>
__device__ __forceinline__ V mode_factor(int q, int r, const MemT<V>* __restrict__ tx, const MemT<V>* __restrict__ ty,
                                         const typename STable<V>::type* __restrict__ s, const RowArgs& a) {
    return mode_factor<V>(q, row_const<V>(r, ty, s, a), tx, s, a);
}

// Copy the E-table rows of the CTA's rows r0 .. r0 + ROWS - 1 to shared memory at
// `dst` (ep entries per row) with cp.async (the caller commits the group and
// waits for it).  Returns false (nothing issued) when
// the plan has no table or `dst` is not 16-byte aligned; the decision is the
// same for every thread of the block.
template <typename V, int ROWS>
__device__ __forceinline__ bool stage_erows(V* dst, int r0, const RowArgs& a) {
    using M = MemT<V>;
    if (!a.etab || (reinterpret_cast<uintptr_t>(dst) & 15)) return false;
    const int chunks = int((size_t(a.ep) * sizeof(M)) / 16);   // ep * sizeof(M) is a multiple of 16
    for (int i = threadIdx.x; i < ROWS * chunks; i += blockDim.x) {
        const int c = i / chunks, k = i - c * chunks;
        const int rr = min(r0 + c, a.np - r0 - c);
        const char* src = static_cast<const char*>(a.etab) + size_t(rr) * a.ep * sizeof(M) + 16 * size_t(k);
        cp_async16(reinterpret_cast<char*>(dst) + size_t(c) * a.ep * sizeof(M) + 16 * size_t(k), src);
    }
    return true;
}

// the factor of mode q in the CTA's row `row` (ROWS == 1: the constants held in registers)
template <typename V, int ROWS>
__device__ __forceinline__ V row_factor(int q, int row, int r0, const RowConst<V>& rc0, const MemT<V>* __restrict__ tx,
                                        const MemT<V>* __restrict__ ty, const typename STable<V>::type* __restrict__ s,
                                        const RowArgs& a) {
    if constexpr (ROWS == 1) return mode_factor<V>(q, rc0, tx, s, a);
    else return mode_factor<V>(q, r0 + row, tx, ty, s, a);
}

// --------------------------------------------------------------- type-1 row pass
// One CTA = ROWS rows r of A (ky bin r): forward 2N' transform of the window
// row restricted to the kept modes (two folded N'-point FFTs), multiply by
// T1x(kx) T1y(ky) E(kx, ky), inverse N'-point FFT, keep the N outputs.
template <typename V, int LOGNP>
__global__ void __launch_bounds__(RowCfg<V, LOGNP>::P, RowCfg<V, LOGNP>::MINB)
    row_t1_kernel(const MemT<V>* __restrict__ A, MemT<V>* __restrict__ B, const MemT<V>* __restrict__ tx,
                  const MemT<V>* __restrict__ ty, const typename STable<V>::type* __restrict__ s,
                  const V* __restrict__ tw, RowArgs a) {
    using Cf = RowCfg<V, LOGNP>;
    constexpr int NP = Cf::NP, ROWS = Cf::ROWS, HALF = NP / 2;
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    V* M = Cf::MERGE ? S : S + spad_size<V>(NP * Cf::SEQ);
    const int r0 = blockIdx.x * ROWS;
    const int W = a.W, Wp = a.Wp;
    const V zero = CTraits<V>::zero();
    pdl_allow_next();
    const RowConst<V> rc0 = row_const<V>(r0, ty, s, a);
    pdl_wait();   // A comes from the previous kernel
    const int sc = cta_scale<V>(A, r0, ROWS, W, Wp);

    constexpr int R0 = Cf::MERGE ? Cf::EM : Cf::EF;   // first-pass radix of the forward engines
    [[maybe_unused]] const int a_n = a.np * Wp;   // extent of A (N' x Wp)
    auto folded = [&](int row, int p, int sgn) -> V {
        const MemT<V>* x = A + (r0 + row) * Wp;
        const V u = p < W && NUASM_IN_RANGE((r0 + row) * Wp + p, a_n, dbg::kRowLoad) ? Mem<V>::ld(x[p], sc) : zero;
        const V t = p + NP < W && NUASM_IN_RANGE((r0 + row) * Wp + p + NP, a_n, dbg::kRowLoad)
                        ? Mem<V>::ld(x[p + NP], sc) : zero;
        return sgn == 0 ? cadd(u, t) : cmul(csub(u, t), half_bin<V, -1, LOGNP, R0>(tw, p));
    };
    auto put = [&](int row, int pk, int sgn, V v) {
        const int pb = 2 * pk + sgn;
        const int q = pb < HALF ? pb : (pb >= 3 * HALF ? pb - NP : -1);
        if (q >= 0 && NUASM_IN_RANGE(row * NP + q, ROWS * NP, dbg::kRowModes))
            M[row * NP + q] = cmul(v, row_factor<V, ROWS>(q, row, r0, rc0, tx, ty, s, a));
    };
    if constexpr (Cf::MERGE) {
        block_fft<V, -1, Cf::EM, LOGNP, Cf::LOGROWS + 1, false>(
            S, tw, [&](int p, int cs) { return folded(cs >> 1, p, cs & 1); },
            [&](int pk, int cs, V v) { put(cs >> 1, pk, cs & 1, v); });
    } else {
#pragma unroll 1
        for (int sgn = 0; sgn < 2; ++sgn)
            block_fft<V, -1, Cf::EF, LOGNP, Cf::LOGROWS, true>(
                S, tw, [&](int p, int c) { return folded(c, p, sgn); },
                [&](int pk, int c, V v) { put(c, pk, sgn, v); });
    }
    __syncthreads();
    const int n = a.n;
    block_fft<V, +1, Cf::EF, LOGNP, Cf::LOGROWS, true, Cf::MERGE>(
        S, tw, [&](int p, int c) { return NUASM_IN_RANGE(c * NP + p, ROWS * NP, dbg::kRowModes) ? M[c * NP + p] : zero; },
        [&](int p, int c, V v) {
            if (p < n && NUASM_IN_RANGE((r0 + c) * n + p, a.np * n, dbg::kRowStore))
                B[(r0 + c) * n + p] = Mem<V>::st(v, sc);
        });
}

// --------------------------------------------------------------- type-2 row pass
// One CTA = ROWS rows r of B (ky bin r, N values): forward N'-point FFT,
// multiply by T2x T2y E, then the inverse 2N' transform onto the window row
// (even and odd outputs as two N'-point FFTs), keeping the W window entries.
template <typename V, int LOGNP>
__global__ void __launch_bounds__(RowCfg<V, LOGNP>::P, RowCfg<V, LOGNP>::MINB)
    row_t2_kernel(const MemT<V>* __restrict__ B, MemT<V>* __restrict__ A, const MemT<V>* __restrict__ tx,
                  const MemT<V>* __restrict__ ty, const typename STable<V>::type* __restrict__ s,
                  const V* __restrict__ tw, RowArgs a) {
    using Cf = RowCfg<V, LOGNP>;
    constexpr int NP = Cf::NP, ROWS = Cf::ROWS, HALF = NP / 2;
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    V* M = Cf::MERGE ? S : S + spad_size<V>(NP * Cf::SEQ);
    const int r0 = blockIdx.x * ROWS;
    const int n = a.n, W = a.W, Wp = a.Wp;
    const V zero = CTraits<V>::zero();
    pdl_allow_next();
    const RowConst<V> rc0 = row_const<V>(r0, ty, s, a);
    // With merged inverse engines S holds 2 ROWS sequences and the forward
    // transform uses the first ROWS: the E rows are staged behind them while it
    // runs (waited for after its first pass, whose successors synchronise),
    // clear of M, which its last pass writes at the start of S.
    static_assert(LOGNP > 3, "the staged E rows need a forward transform of at least two passes");
    // Where the plan has the combined T2x E table, its rows (N' entries,
    // Tx folded in) are staged instead and the epilogue needs no Tx load.
    V* Es = S + ((spad_size<V>(NP * ROWS) + 1) & ~1);
    int staged = 0;   // 0: nothing staged, 1: E rows, 2: T2x E rows
    if constexpr (Cf::MERGE) {
        if (a.etab2 && !(reinterpret_cast<uintptr_t>(Es) & 15)) {
            constexpr int chunks = int((size_t(NP) * sizeof(V)) / 16);
            for (int i = threadIdx.x; i < ROWS * chunks; i += Cf::P) {
                const int c = i / chunks, k = i - c * chunks;
                const int rr = min(r0 + c, NP - r0 - c);
                cp_async16(reinterpret_cast<char*>(Es) + (size_t(c) * NP * sizeof(V)) + 16 * size_t(k),
                           static_cast<const char*>(a.etab2) + (size_t(rr) * NP * sizeof(V)) + 16 * size_t(k));
            }
            staged = 2;
        } else if (stage_erows<V, ROWS>(Es, r0, a)) {
            staged = 1;
        }
        if (staged) cp_async_commit();
    }
    pdl_wait();   // B comes from the previous kernel
    const int sc = cta_scale<V>(B, r0, ROWS, n, n);
    block_fft<V, -1, Cf::EF, LOGNP, Cf::LOGROWS, true>(
        S, tw,
        [&](int p, int c) {
            return p < n && NUASM_IN_RANGE((r0 + c) * n + p, a.np * n, dbg::kRowLoad)
                       ? Mem<V>::ld(B[(r0 + c) * n + p], sc) : zero;
        },
        [&](int p, int c, V v) {
            V f;
            const V t = ROWS == 1 ? rc0.ty : Mem<V>::ld(__ldg(&ty[r0 + c]), 0);
            if (staged == 2) {
                f = cmul(Es[c * NP + p], t);
            } else if (staged == 1) {
                const MemT<V>* Em = reinterpret_cast<const MemT<V>*>(Es);
                f = cmul(cmul(Mem<V>::ld(__ldg(&tx[p]), 0), t), Mem<V>::ld(Em[c * a.ep + min(p, NP - p)], 0));
            } else {
                f = row_factor<V, ROWS>(p, c, r0, rc0, tx, ty, s, a);
            }
            if (NUASM_IN_RANGE(c * NP + p, ROWS * NP, dbg::kRowModes)) M[c * NP + p] = cmul(v, f);
        },
        [&] {
            if (staged) cp_async_wait_all();
        });
    __syncthreads();
    // pre-twiddle of the odd outputs: conj(tw[pg]), pg the 2N'-grid bin of q, is
    // exp(i pi q / N') with a minus sign for q >= N'/2
    constexpr int R0I = Cf::MERGE ? Cf::EM : Cf::EF;   // first-pass radix of the inverse engines
    auto get = [&](int row, int q, int sgn) -> V {
        const V y = NUASM_IN_RANGE(row * NP + q, ROWS * NP, dbg::kRowModes) ? M[row * NP + q] : zero;
        if (sgn == 0) return y;
        const V f = half_bin<V, +1, LOGNP, R0I>(tw, q);
        return cmul(y, q < HALF ? f : CTraits<V>::make(-f.x, -f.y));
    };
    auto put = [&](int row, int k, int sgn, V v) {
        const int u = 2 * k + sgn;
        if (u < W && NUASM_IN_RANGE((r0 + row) * Wp + u, a.np * Wp, dbg::kRowStore))
            A[(r0 + row) * Wp + u] = Mem<V>::st(v, sc);
    };
    if constexpr (Cf::MERGE) {
        block_fft<V, +1, Cf::EM, LOGNP, Cf::LOGROWS + 1, false, true>(
            S, tw, [&](int q, int cs) { return get(cs >> 1, q, cs & 1); },
            [&](int k, int cs, V v) { put(cs >> 1, k, cs & 1, v); });
    } else {
#pragma unroll 1
        for (int sgn = 0; sgn < 2; ++sgn)
            block_fft<V, +1, Cf::EF, LOGNP, Cf::LOGROWS, true>(
                S, tw, [&](int q, int c) { return get(c, q, sgn); },
                [&](int k, int c, V v) { put(c, k, sgn, v); });
    }
}

// --------------------------------------------------------------- type-3 row pass
// NU-ASM_3 / NU-FRE_3: one CTA = ROWS rows r of A (ky bin r, W window
// entries): forward 2N' transform restricted to the kept modes (folded halves,
// as in row_t1), multiply by T3x T3y E, inverse 2N' transform back onto the
// window row (even/odd halves, as in row_t2), written over the input row (all
// reads happen in the first forward pass, before any write).
template <typename V, int LOGNP>
__global__ void __launch_bounds__(RowCfg<V, LOGNP>::P, RowCfg<V, LOGNP>::MINB)
    row_t3_kernel(MemT<V>* __restrict__ A, const MemT<V>* __restrict__ tx, const MemT<V>* __restrict__ ty,
                  const typename STable<V>::type* __restrict__ s, const V* __restrict__ tw, RowArgs a) {
    using Cf = RowCfg<V, LOGNP>;
    constexpr int NP = Cf::NP, ROWS = Cf::ROWS, HALF = NP / 2;
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    V* M = Cf::MERGE ? S : S + spad_size<V>(NP * Cf::SEQ);
    const int r0 = blockIdx.x * ROWS;
    const int W = a.W, Wp = a.Wp;
    const V zero = CTraits<V>::zero();
    pdl_allow_next();
    const RowConst<V> rc0 = row_const<V>(r0, ty, s, a);
    pdl_wait();   // A comes from the previous kernel
    const int sc = cta_scale<V>(A, r0, ROWS, W, Wp);
    constexpr int R0 = Cf::MERGE ? Cf::EM : Cf::EF;   // first-pass radix of the engines
    [[maybe_unused]] const int a_n = a.np * Wp;   // extent of A (N' x Wp)
    auto folded = [&](int row, int p, int sgn) -> V {
        const MemT<V>* x = A + (r0 + row) * Wp;
        const V u = p < W && NUASM_IN_RANGE((r0 + row) * Wp + p, a_n, dbg::kRowLoad) ? Mem<V>::ld(x[p], sc) : zero;
        const V t = p + NP < W && NUASM_IN_RANGE((r0 + row) * Wp + p + NP, a_n, dbg::kRowLoad)
                        ? Mem<V>::ld(x[p + NP], sc) : zero;
        return sgn == 0 ? cadd(u, t) : cmul(csub(u, t), half_bin<V, -1, LOGNP, R0>(tw, p));
    };
    auto put_mode = [&](int row, int pk, int sgn, V v) {
        const int pb = 2 * pk + sgn;
        const int q = pb < HALF ? pb : (pb >= 3 * HALF ? pb - NP : -1);
        if (q >= 0 && NUASM_IN_RANGE(row * NP + q, ROWS * NP, dbg::kRowModes))
            M[row * NP + q] = cmul(v, row_factor<V, ROWS>(q, row, r0, rc0, tx, ty, s, a));
    };
    auto get_mode = [&](int row, int q, int sgn) -> V {
        const V y = NUASM_IN_RANGE(row * NP + q, ROWS * NP, dbg::kRowModes) ? M[row * NP + q] : zero;
        if (sgn == 0) return y;
        const V f = half_bin<V, +1, LOGNP, R0>(tw, q);
        return cmul(y, q < HALF ? f : CTraits<V>::make(-f.x, -f.y));
    };
    auto put_row = [&](int row, int k, int sgn, V v) {
        const int u = 2 * k + sgn;
        if (u < W && NUASM_IN_RANGE((r0 + row) * Wp + u, a_n, dbg::kRowStore))
            A[(r0 + row) * Wp + u] = Mem<V>::st(v, sc);
    };
    if constexpr (Cf::MERGE) {
        block_fft<V, -1, Cf::EM, LOGNP, Cf::LOGROWS + 1, false>(
            S, tw, [&](int p, int cs) { return folded(cs >> 1, p, cs & 1); },
            [&](int pk, int cs, V v) { put_mode(cs >> 1, pk, cs & 1, v); });
        __syncthreads();
        block_fft<V, +1, Cf::EM, LOGNP, Cf::LOGROWS + 1, false, true>(
            S, tw, [&](int q, int cs) { return get_mode(cs >> 1, q, cs & 1); },
            [&](int k, int cs, V v) { put_row(cs >> 1, k, cs & 1, v); });
    } else {
#pragma unroll 1
        for (int sgn = 0; sgn < 2; ++sgn)
            block_fft<V, -1, Cf::EF, LOGNP, Cf::LOGROWS, true>(
                S, tw, [&](int p, int c) { return folded(c, p, sgn); },
                [&](int pk, int c, V v) { put_mode(c, pk, sgn, v); });
        __syncthreads();
#pragma unroll 1
        for (int sgn = 0; sgn < 2; ++sgn)
            block_fft<V, +1, Cf::EF, LOGNP, Cf::LOGROWS, true>(
                S, tw, [&](int q, int c) { return get_mode(c, q, sgn); },
                [&](int k, int c, V v) { put_row(c, k, sgn, v); });
    }
}

// --------------------------------------------------------------- column passes
enum ColMode { COL_FWD_FOLD = 0, COL_INV = 1, COL_FWD = 2, COL_INV_FOLD = 3 };

// One CTA = C adjacent columns (blockIdx.x) and, for the folded modes, one
// half (blockIdx.y: 0 even, 1 odd).
template <typename V, int LOGNP, int MODE>
__global__ void __launch_bounds__(ColCfg<V, LOGNP, MODE>::P, ColCfg<V, LOGNP, MODE>::MINB)
    col_kernel(const MemT<V>* __restrict__ src, MemT<V>* __restrict__ dst, const V* __restrict__ tw, ColArgs a) {
    using Cf = ColCfg<V, LOGNP, MODE>;
    constexpr int NP = Cf::NP, HALF = NP / 2, C = Cf::C;
    extern __shared__ unsigned char smem_raw[];
    V* S = reinterpret_cast<V*>(smem_raw);
    const int col0 = blockIdx.x * C;
    const int sgn = blockIdx.y;
    const int W = a.W, Wp = a.Wp, n = a.n;
    const V zero = CTraits<V>::zero();
    // extents of src and dst (elements) for the checks of the debug library
    [[maybe_unused]] const int src_n = MODE == COL_FWD_FOLD ? W * Wp : MODE == COL_INV ? NP * n
                                     : MODE == COL_FWD ? n * n : NP * Wp;
    [[maybe_unused]] const int dst_n = MODE == COL_FWD_FOLD ? NP * Wp : MODE == COL_INV ? n * n
                                     : MODE == COL_FWD ? NP * n : W * Wp;
    pdl_allow_next();
    pdl_wait();   // src comes from the previous kernel (no-op for the first kernel of a chain)
    // double-float passes: the CTA's scale over the source rows and columns it reads
    int sc = 0;
    if constexpr (Mem<V>::scaled) {
        const bool win_cols = MODE == COL_FWD_FOLD || MODE == COL_INV_FOLD;   // window-wide arrays
        const int cols = win_cols ? W : n, pitch = win_cols ? Wp : n;
        const int rows = MODE == COL_FWD_FOLD ? W : MODE == COL_FWD ? n : NP;
        sc = cta_scale<V>(src + col0, 0, rows, min(C, cols - col0), pitch);
    }
    auto ld = [&](int i) -> V { return NUASM_IN_RANGE(i, src_n, dbg::kColLoad) ? Mem<V>::ld(src[i], sc) : zero; };
    auto st = [&](int i, V v) {
        if (NUASM_IN_RANGE(i, dst_n, dbg::kColStore)) dst[i] = Mem<V>::st(v, sc);
    };
    if constexpr (MODE == COL_FWD_FOLD) {
        // src: window (W x Wp); dst: A (N' x Wp), kept modes in natural N'-bin rows
        block_fft<V, -1, Cf::E, LOGNP, Cf::LOGC, false>(
            S, tw,
            [&](int p, int c) -> V {
                const int col = col0 + c;
                if (col >= W) return zero;
                const V u = p < W ? ld(p * Wp + col) : zero;
                const V t = p + NP < W ? ld((p + NP) * Wp + col) : zero;
                return sgn == 0 ? cadd(u, t) : cmul(csub(u, t), half_bin<V, -1, LOGNP, Cf::E>(tw, p));
            },
            [&](int pk, int c, V v) {
                const int col = col0 + c;
                const int pb = 2 * pk + sgn;
                const int r = pb < HALF ? pb : (pb >= 3 * HALF ? pb - NP : -1);
                if (r >= 0 && col < W) st(r * Wp + col, v);
            });
    } else if constexpr (MODE == COL_INV) {
        // src: B (N' x N); dst: u2 (N x N)
        block_fft<V, +1, Cf::E, LOGNP, Cf::LOGC, false>(
            S, tw, [&](int p, int c) { return ld(p * n + col0 + c); },
            [&](int p, int c, V v) {
                if (p < n) st(p * n + col0 + c, v);
            });
    } else if constexpr (MODE == COL_FWD) {
        // src: u1 (N x N); dst: B (N' x N)
        block_fft<V, -1, Cf::E, LOGNP, Cf::LOGC, false>(
            S, tw, [&](int p, int c) { return p < n ? ld(p * n + col0 + c) : zero; },
            [&](int p, int c, V v) { st(p * n + col0 + c, v); });
    } else {
        // src: A (N' x Wp); dst: window (W x Wp)
        block_fft<V, +1, Cf::E, LOGNP, Cf::LOGC, false>(
            S, tw,
            [&](int q, int c) -> V {
                const int col = col0 + c;
                if (col >= W) return zero;
                const V y = ld(q * Wp + col);
                if (sgn == 0) return y;
                const V f = half_bin<V, +1, LOGNP, Cf::E>(tw, q);
                return cmul(y, q < HALF ? f : CTraits<V>::make(-f.x, -f.y));
            },
            [&](int k, int c, V v) {
                const int col = col0 + c;
                const int u = 2 * k + sgn;
                if (u < W && col < W) st(u * Wp + col, v);
            });
    }
}

// --------------------------------------------------------------- TMA column passes (FP32)
// Persistent variant of col_kernel: each CTA walks column strips s, s + G, ...
// One elected thread loads a strip (C columns x all needed rows) into a raw
// shared buffer with 2-D TMA boxes of C x BOXR elements completed on an
// mbarrier; rows and columns outside the array arrive as zeros, which provides
// the zero padding and the window clipping for free.  The FFT's first pass
// reads the raw buffer; right after that pass the next strip's load is issued,
// so it overlaps the remaining passes.  The folded modes compute both halves
// from one load.  Waits are bounded: a wait that gives up sets bit 2 of the
// plan's error word, waits once more for its own copy and the CTA returns.
// Tuning knobs: columns per TMA strip (NUASM_TMA_C) and the column modes that
// use the TMA pipeline (bit MODE of NUASM_TMA_MODES up to N' = 2048, of
// NUASM_TMA_MODES_WIDE beyond; measured: at N' = 2048 the unfolded passes are
// faster without TMA, at N' = 4096 with it).
#ifndef NUASM_TMA_C
#define NUASM_TMA_C 4
#endif
#ifndef NUASM_TMA_MODES
#define NUASM_TMA_MODES 0x9        // N' <= 2048
#endif
#ifndef NUASM_TMA_MODES_WIDE
#define NUASM_TMA_MODES_WIDE 0xF   // N' >= 4096: the unfolded passes have 1024+ strips too
#endif
#ifndef NUASM_TMA_HALF_TAIL
#define NUASM_TMA_HALF_TAIL 1      // a last partial round of strips runs as half strips
#endif

#ifndef NUASM_TMA_STORE
#define NUASM_TMA_STORE 1          // 1: outputs staged in shared memory and written with bulk tensor stores
#endif

template <int LOGNP, int MODE> struct TmaColCfg {
    using Base = ColCfg<float2, LOGNP>;
    static constexpr int NP = Base::NP;
    static constexpr int C = Base::C < NUASM_TMA_C ? Base::C : NUASM_TMA_C;
    static constexpr int LOGC = Log2<C>::v;
    // up to N' = 2048 the folded modes transform both halves of every column
    // at once (sequence cs = 2 c + half, 2C sequences per strip, twice the
    // warps); beyond, 1024 threads would spill, so the halves run in turn
    static constexpr bool FOLDED = MODE == COL_FWD_FOLD || MODE == COL_INV_FOLD;
    static constexpr bool MERGED = FOLDED && LOGNP <= 11;
    static constexpr int SEQ = MERGED ? 2 * C : C;
    static constexpr int LOGSEQ = Log2<SEQ>::v;
    static constexpr int E = Base::E;
    static constexpr int P = (NP * SEQ) / E;
    static constexpr int BOXR = NP < 256 ? NP : 256;
    static constexpr int RAW_ROWS = MODE == COL_FWD_FOLD ? NP + BOXR : NP;
    static constexpr size_t RAW_BYTES = size_t(RAW_ROWS) * C * sizeof(float2);
    static constexpr size_t WORK_BYTES = ((size_t(spad_size<float2>(NP * SEQ)) * sizeof(float2)) + 127) & ~size_t(127);
    // Bulk stores: the output is viewed as {columns, PLANES, rows / PLANES}
    // (the folded modes interleave their two halves by row: plane = half) and
    // written in boxes of BOXZ rows, instead of 8-byte stores per thread that
    // each cover half a 32-byte sector at C = 2.  A strip that runs one
    // transform stages its output in the work buffer itself (the last pass has
    // read it by then); the halves of a folded strip run in turn and stage in a
    // buffer of their own.  Measured: the N' = 4096 folded passes 143 ->
    // 120 us and 150 -> 127 us on the 4M-point plane; the merged N' = 2048
    // fold 34.7 -> 36.8 us (its staging in the work buffer holds the next
    // strip's first pass until the stores have read it), so it keeps
    // per-thread stores.
    static constexpr bool STORE = NUASM_TMA_STORE != 0 && !MERGED;
    static constexpr bool OWN_STAGE = STORE && FOLDED;
    static constexpr size_t STAGE_BYTES = OWN_STAGE ? size_t(NP) * C * sizeof(float2) : 0;
    static constexpr int PLANES = FOLDED ? 2 : 1;
    static constexpr int BOXZ = NP < 256 ? NP : 256;
    static constexpr size_t SMEM = 128 + RAW_BYTES + WORK_BYTES + STAGE_BYTES + 16;
    static size_t smem() { return SMEM; }
    static constexpr bool FITS = SMEM <= 227u * 1024u;
    // CTAs per SM that shared memory allows (228 KB per SM, 1 KB reserved per
    // CTA): registers are capped only as far as that occupancy needs
    static constexpr int BY_SMEM = int((228u * 1024u) / (SMEM + 1024u));
    static constexpr int BY_REGS = 65536 / (P * 64);
    static constexpr int MINB = BY_SMEM < 1 ? 1 : (BY_SMEM < BY_REGS ? BY_SMEM : (BY_REGS < 1 ? 1 : BY_REGS));
};

// Work items: `nfull` strips of C columns, then half strips of C/2 columns
// for the columns of a last partial round (the host passes nfull as a whole
// number of rounds of the grid when that leaves a partial round).  A half
// strip loads the same C-wide box (the columns beyond its own are not used)
// and transforms its C/2 columns with half the elements per thread, so a last
// round that would keep part of the GPU busy for a full strip's time takes
// half of it on all of the GPU.  `omap` and `omap_h` are the output's store
// views with boxes C and C/2 columns wide; `nz` is the number of output rows
// (per plane) that the stores cover.
template <int LOGNP, int MODE>
__global__ void __launch_bounds__(TmaColCfg<LOGNP, MODE>::P, TmaColCfg<LOGNP, MODE>::MINB)
    col_tma_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap omap,
                   const __grid_constant__ CUtensorMap omap_h, float2* __restrict__ dst,
                   const float2* __restrict__ tw, ColArgs a, int nfull, int nitems, int nboxes, int nz,
                   int* __restrict__ err) {
    using Cf = TmaColCfg<LOGNP, MODE>;
    constexpr int NP = Cf::NP, HALF = NP / 2, C = Cf::C, BOXR = Cf::BOXR, BOXZ = Cf::BOXZ;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float2* raw = reinterpret_cast<float2*>(base);
    float2* S = reinterpret_cast<float2*>(base + Cf::RAW_BYTES);
    float2* O = reinterpret_cast<float2*>(base + Cf::RAW_BYTES + Cf::WORK_BYTES);   // own staging, if any
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + Cf::RAW_BYTES + Cf::WORK_BYTES + Cf::STAGE_BYTES);
    const int tid = threadIdx.x;
    const int W = a.W, Wp = a.Wp, n = a.n;
    const float2 zero = make_float2(0.f, 0.f);
    // extents for the checks of the debug library: the raw strip, the staging
    // buffers and dst (elements)
    [[maybe_unused]] constexpr int RAW_N = Cf::RAW_ROWS * C, O_N = Cf::OWN_STAGE ? NP * C : 0, S_N = spad_size<float2>(NP * Cf::SEQ);
    [[maybe_unused]] const int dst_n = MODE == COL_FWD_FOLD ? NP * Wp : MODE == COL_INV ? n * n
                                     : MODE == COL_FWD ? NP * n : W * Wp;
    auto rd = [&](int i) -> float2 { return NUASM_IN_RANGE(i, RAW_N, dbg::kColRaw) ? raw[i] : zero; };
    [[maybe_unused]] auto st = [&](int i, float2 v) {
        if (NUASM_IN_RANGE(i, dst_n, dbg::kColStore)) dst[i] = v;
    };
    [[maybe_unused]] auto stage_o = [&](int i, float2 v) {
        if (NUASM_IN_RANGE(i, O_N, dbg::kColStage)) O[i] = v;
    };
    [[maybe_unused]] auto stage_s = [&](int i, float2 v) {
        if (NUASM_IN_RANGE(i, S_N, dbg::kColStage)) S[i] = v;
    };
    pdl_allow_next();
    if (tid == 0) tma::mbar_init(bar, 1);
    pdl_wait();   // the strips come from the previous kernel
    if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");   // its writes, for the TMA reads
    __syncthreads();
    auto col0_of = [&](int item) { return item < nfull ? item * C : nfull * C + (item - nfull) * (C / 2); };
    auto issue = [&](int item) {
        tma::mbar_expect_tx(bar, uint32_t(nboxes) * BOXR * C * uint32_t(sizeof(float2)));
        for (int b = 0; b < nboxes; ++b) tma::load_2d(raw + b * BOXR * C, &map, col0_of(item), b * BOXR, bar);
    };
    if (tid == 0 && int(blockIdx.x) < nitems) issue(blockIdx.x);
    uint32_t parity = 0;
    // one item of CC columns (CC = C or C/2) with EE elements per thread
    auto run_item = [&](auto cc_tag, auto prefetch, int col0) {
        constexpr int CC = decltype(cc_tag)::value;
        constexpr int EE = Cf::E * CC / C;
        constexpr int LOGCC = Log2<CC>::v;
        [[maybe_unused]] constexpr int LOGSEQ = Cf::MERGED ? LOGCC + 1 : LOGCC;
        // staged output of the item's transform: plane `plane`, rows [0, nz) --
        // make the staged data visible to the bulk copies and issue them
        [[maybe_unused]] auto flush = [&](const float2* stage, int plane) {
            tma::store_fence();
            __syncthreads();
            if (tid == 0) {
                const CUtensorMap* om = CC == C ? &omap : &omap_h;
                for (int z0 = 0; z0 < nz; z0 += BOXZ) tma::store_3d(om, col0, plane, z0, stage + z0 * CC);
                tma::store_commit();
            }
        };
        // the second half of a non-merged folded strip rewrites the staging
        // buffer: its reads by the first half's stores end before the barriers
        // that follow its first pass
        [[maybe_unused]] auto second_half_hook = [&] {
            if (tid == 0) tma::store_wait_read();
            prefetch();
        };
        if constexpr (MODE == COL_FWD_FOLD) {
            // raw: window rows [0, NP + BOXR) of C columns (zero beyond the window);
            // half 0 transforms x(p) + x(p + N'), half 1 (x(p) - x(p + N')) w^p
            auto fold = [&](int p, int c, int sgn) -> float2 {
                // rows p + N' < W lie within the first BOXR rows past N' (W - N' = 2h <= 16)
                const float2 u = rd(p * C + c), t = p < BOXR ? rd((p + NP) * C + c) : zero;
                const float sg = sgn ? -1.f : 1.f;
                const float2 v = make_float2(fmaf(sg, t.x, u.x), fmaf(sg, t.y, u.y));
                return sgn ? cmul(v, half_bin<float2, -1, LOGNP, EE>(tw, p)) : v;
            };
            // output row r = 2 pk + sgn (first quarter of the bins) or 2 pk + sgn - N' (last quarter)
            auto put = [&](int pk, int c, int sgn, float2 v) {
                const int pb = 2 * pk + sgn;
                const int r = pb < HALF ? pb : (pb >= 3 * HALF ? pb - NP : -1);
                if constexpr (Cf::STORE) {
                    if (r >= 0) stage_o((r >> 1) * CC + c, v);   // plane sgn, row r >> 1
                } else {
                    const int col = col0 + c;
                    if (r >= 0 && col < W) st(r * Wp + col, v);
                }
            };
            if constexpr (Cf::MERGED) {
                block_fft<float2, -1, EE, LOGNP, LOGSEQ, false>(
                    S, tw, [&](int p, int cs) { return fold(p, cs >> 1, cs & 1); },
                    [&](int pk, int cs, float2 v) { put(pk, cs >> 1, cs & 1, v); }, prefetch);
            } else {
                auto nothing = [] {};
#pragma unroll 1
                for (int sgn = 0; sgn < 2; ++sgn) {
                    auto load = [&](int p, int c) { return fold(p, c, sgn); };
                    auto store = [&](int pk, int c, float2 v) { put(pk, c, sgn, v); };
                    if (sgn == 0) block_fft<float2, -1, EE, LOGNP, LOGCC, false>(S, tw, load, store, nothing);
                    else if constexpr (Cf::STORE)
                        block_fft<float2, -1, EE, LOGNP, LOGCC, false>(S, tw, load, store, second_half_hook);
                    else block_fft<float2, -1, EE, LOGNP, LOGCC, false>(S, tw, load, store, prefetch);
                    if constexpr (Cf::STORE) flush(O, sgn);
                }
            }
        } else if constexpr (MODE == COL_INV_FOLD) {
            // raw: rows [0, N') of A, C columns (zero beyond the window's columns);
            // half 1 is pre-twiddled for the odd outputs
            auto get = [&](int q, int c, int sgn) -> float2 {
                const float2 y = rd(q * C + c);
                if (sgn == 0) return y;
                const float2 f = half_bin<float2, +1, LOGNP, EE>(tw, q);
                return cmul(y, q < HALF ? f : make_float2(-f.x, -f.y));
            };
            // output row u = 2 k + sgn
            auto put = [&](int k, int c, int sgn, float2 v) {
                if constexpr (Cf::STORE) {
                    stage_o(k * CC + c, v);   // plane sgn, row k
                } else {
                    const int col = col0 + c;
                    const int u = 2 * k + sgn;
                    if (u < W && col < W) st(u * Wp + col, v);
                }
            };
            if constexpr (Cf::MERGED) {
                block_fft<float2, +1, EE, LOGNP, LOGSEQ, false>(
                    S, tw, [&](int q, int cs) { return get(q, cs >> 1, cs & 1); },
                    [&](int k, int cs, float2 v) { put(k, cs >> 1, cs & 1, v); }, prefetch);
            } else {
                auto nothing = [] {};
#pragma unroll 1
                for (int sgn = 0; sgn < 2; ++sgn) {
                    auto load = [&](int q, int c) { return get(q, c, sgn); };
                    auto store = [&](int k, int c, float2 v) { put(k, c, sgn, v); };
                    if (sgn == 0) block_fft<float2, +1, EE, LOGNP, LOGCC, false>(S, tw, load, store, nothing);
                    else if constexpr (Cf::STORE)
                        block_fft<float2, +1, EE, LOGNP, LOGCC, false>(S, tw, load, store, second_half_hook);
                    else block_fft<float2, +1, EE, LOGNP, LOGCC, false>(S, tw, load, store, prefetch);
                    if constexpr (Cf::STORE) flush(O, sgn);
                }
            }
        } else if constexpr (MODE == COL_INV) {
            block_fft<float2, +1, EE, LOGNP, LOGCC, false>(
                S, tw, [&](int p, int c) { return rd(p * C + c); },
                [&](int p, int c, float2 v) {
                    if constexpr (Cf::STORE) stage_s(p * CC + c, v);
                    else if (p < n && col0 + c < n) st(p * n + col0 + c, v);
                },
                prefetch);
            if constexpr (Cf::STORE) flush(S, 0);
        } else {
            block_fft<float2, -1, EE, LOGNP, LOGCC, false>(
                S, tw, [&](int p, int c) { return p < n ? rd(p * C + c) : zero; },
                [&](int p, int c, float2 v) {
                    if constexpr (Cf::STORE) stage_s(p * CC + c, v);
                    else if (col0 + c < n) st(p * n + col0 + c, v);
                },
                prefetch);
            if constexpr (Cf::STORE) flush(S, 0);
        }
    };
    // before a wait gives up and the CTA returns: its own copies in flight end first
    auto give_up = [&] {
        if (tid == 0) {
            atomicOr(err, 2);
            tma::mbar_wait(bar, parity);
            if constexpr (Cf::STORE) tma::store_wait_all();
        }
    };
    // the full strips, then (nfull being a whole number of rounds) the half strips
    int s = blockIdx.x;
    for (; s < nfull; s += gridDim.x) {
        // the previous strip's stores have read the staged output before this strip's first pass rewrites it
        if (Cf::STORE && tid == 0) tma::store_wait_read();
        const bool ok = tma::mbar_wait(bar, parity);
        if (__syncthreads_or(!ok)) {
            give_up();
            return;
        }
        parity ^= 1;
        const int next = s + gridDim.x;
        auto prefetch = [&] {
            if (tid == 0 && next < nitems) issue(next);
        };
        run_item(std::integral_constant<int, C>{}, prefetch, s * C);
    }
    if constexpr (C >= 4) {   // half strips start on an even column (16-byte TMA coordinate)
        for (; s < nitems; s += gridDim.x) {
            if (Cf::STORE && tid == 0) tma::store_wait_read();
            const bool ok = tma::mbar_wait(bar, parity);
            if (__syncthreads_or(!ok)) {
                give_up();
                return;
            }
            parity ^= 1;
            const int next = s + gridDim.x;
            auto prefetch = [&] {
                if (tid == 0 && next < nitems) issue(next);
            };
            run_item(std::integral_constant<int, C / 2>{}, prefetch, col0_of(s));
        }
    }
    if (Cf::STORE && tid == 0) tma::store_wait_all();
}

// --------------------------------------------------------------- launchers
template <typename K> cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

inline RowArgs row_args(const nuasm_plan_s* P) {
    RowArgs a{};
    a.n = P->g.n;
    a.W = P->g.W;
    a.Wp = P->g.Wp;
    a.nonsep = P->nonsep_mode;
    a.rc = P->rc;
    a.rc_hi = float(P->rc);
    a.rc_lo = float(P->rc - double(a.rc_hi));
    a.etab = P->d.etab;
    a.etab2 = P->d.etab2;
    a.ep = P->etab_pitch;
    a.np = P->g.np;
    return a;
}

template <typename V, int LOGNP>
cudaError_t launch_row(const nuasm_plan_s* P, int type, cudaStream_t st) {
    using Cf = RowCfg<V, LOGNP>;
    using ST = typename STable<V>::type;
    using M = MemT<V>;
    const RowArgs a = row_args(P);
    const size_t sm = Cf::smem();
    // double-float passes read the plan's twiddles as float pairs
    const V* tw = static_cast<const V*>(Mem<V>::scaled ? P->d.tw_df : P->d.tw);
    if (!tw) return cudaErrorInvalidValue;
    const ST* s = static_cast<const ST*>(P->d.s);
    const int blocks = Cf::NP / Cf::ROWS;
    cudaError_t e;
    if (type == 1) {
        if ((e = set_smem(row_t1_kernel<V, LOGNP>, sm)) != cudaSuccess) return e;
        e = launch_chained(row_t1_kernel<V, LOGNP>, dim3(blocks), dim3(Cf::P), sm, st,
                           static_cast<const M*>(P->d.bufA), static_cast<M*>(P->d.bufB),
                           static_cast<const M*>(P->d.t1x), static_cast<const M*>(P->d.t1y), s, tw, a);
    } else if (type == 3) {
        if ((e = set_smem(row_t3_kernel<V, LOGNP>, sm)) != cudaSuccess) return e;
        e = launch_chained(row_t3_kernel<V, LOGNP>, dim3(blocks), dim3(Cf::P), sm, st, static_cast<M*>(P->d.bufA),
                           static_cast<const M*>(P->d.t3x), static_cast<const M*>(P->d.t3y), s, tw, a);
    } else {
        if ((e = set_smem(row_t2_kernel<V, LOGNP>, sm)) != cudaSuccess) return e;
        e = launch_chained(row_t2_kernel<V, LOGNP>, dim3(blocks), dim3(Cf::P), sm, st,
                           static_cast<const M*>(P->d.bufB), static_cast<M*>(P->d.bufA),
                           static_cast<const M*>(P->d.t2x), static_cast<const M*>(P->d.t2y), s, tw, a);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename V, int LOGNP, int MODE>
cudaError_t launch_col(const nuasm_plan_s* P, const void* src, void* dst, int ncols, int halves, cudaStream_t st) {
    using Cf = ColCfg<V, LOGNP, MODE>;
    const ColArgs a{P->g.n, P->g.W, P->g.Wp};
    const size_t sm = Cf::smem();
    cudaError_t e = set_smem(col_kernel<V, LOGNP, MODE>, sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + Cf::C - 1) / Cf::C, halves);
    using M = MemT<V>;
    // double-float passes read the plan's twiddles as float pairs
    const V* tw = static_cast<const V*>(Mem<V>::scaled ? P->d.tw_df : P->d.tw);
    if (!tw) return cudaErrorInvalidValue;
    if constexpr (MODE == COL_FWD) {   // first kernel of the type-2 chain
        col_kernel<V, LOGNP, MODE><<<grid, Cf::P, sm, st>>>(static_cast<const M*>(src), static_cast<M*>(dst), tw, a);
    } else {
        e = launch_chained(col_kernel<V, LOGNP, MODE>, grid, dim3(Cf::P), sm, st, static_cast<const M*>(src),
                           static_cast<M*>(dst), tw, a);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// TMA variant (FP32, at least two columns per strip); returns cudaErrorNotSupported
// when the source array breaks the TMA alignment rules, so the caller can fall back.
template <int LOGNP, int MODE>
cudaError_t launch_col_tma(const nuasm_plan_s* P, const void* src, void* dst, int ncols, int src_cols,
                           int src_rows, int src_pitch, int load_rows, cudaStream_t st) {
    using Cf = TmaColCfg<LOGNP, MODE>;
    constexpr int modes = LOGNP >= 12 ? NUASM_TMA_MODES_WIDE : NUASM_TMA_MODES;
    if constexpr (Cf::C < 2 || Cf::NP < 512 || !((modes >> MODE) & 1) || !Cf::FITS) {
        return cudaErrorNotSupported;
    } else {
        CUtensorMap map, omap, omap_h;
        if (!encode_map_8b(&map, src, src_cols, src_rows, src_pitch, Cf::C, Cf::BOXR)) return cudaErrorNotSupported;
        // the output's store view: {columns, planes, rows per plane}, row pitch
        const Geometry& g = P->g;
        int ocols = g.n, orows = Cf::NP, opitch = g.n, nz = Cf::NP;
        if constexpr (MODE == COL_FWD_FOLD) {
            ocols = g.W, orows = Cf::NP / 2, opitch = g.Wp, nz = orows;
        } else if constexpr (MODE == COL_INV_FOLD) {
            if (g.W & 1) return cudaErrorNotSupported;   // the window's rows pair up as (2k, 2k + 1)
            ocols = g.W, orows = g.W / 2, opitch = g.Wp, nz = orows < Cf::NP ? orows : Cf::NP;
        } else if constexpr (MODE == COL_INV) {
            orows = g.n, nz = g.n;
        }
        if constexpr (Cf::STORE) {
            constexpr int hc = Cf::C >= 4 ? Cf::C / 2 : Cf::C;
            if (!encode_store_map_8b(&omap, dst, ocols, Cf::PLANES, orows, opitch, Cf::C, 1, Cf::BOXZ) ||
                !encode_store_map_8b(&omap_h, dst, ocols, Cf::PLANES, orows, opitch, hc, 1, Cf::BOXZ))
                return cudaErrorNotSupported;
        } else {
            omap = map;
            omap_h = map;
        }
        const size_t sm = Cf::smem();
        cudaError_t e = set_smem(col_tma_kernel<LOGNP, MODE>, sm);
        if (e != cudaSuccess) return e;
        static std::atomic<int> resident{0};   // persistent grid: resident CTAs on the whole GPU
        int ctas = resident.load(std::memory_order_relaxed);
        if (ctas == 0) {
            int dev = 0, nsm = 0, per = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, col_tma_kernel<LOGNP, MODE>, Cf::P, sm)) !=
                cudaSuccess)
                return e;
            ctas = nsm * (per > 0 ? per : 1);
            resident.store(ctas, std::memory_order_relaxed);
        }
        const int nstrips = (ncols + Cf::C - 1) / Cf::C;
        const int nboxes = (load_rows + Cf::BOXR - 1) / Cf::BOXR;
        const int grid = nstrips < ctas ? nstrips : ctas;
        // a last partial round of strips runs as half strips over the whole grid
        int nfull = nstrips, nitems = nstrips;
        // (C >= 4: a half strip's first column, the TMA x coordinate, must stay even)
        if (NUASM_TMA_HALF_TAIL && Cf::C >= 4 && nstrips > grid && nstrips % grid != 0) {
            nfull = (nstrips / grid) * grid;
            const int tail = ncols - nfull * Cf::C, hc = Cf::C / 2;
            nitems = nfull + (tail + hc - 1) / hc;
            if ((hc & 1) || ((nfull * Cf::C) & 1)) return cudaErrorNotSupported;   // an odd TMA x: never issued
        }
        const ColArgs a{P->g.n, P->g.W, P->g.Wp};
        if constexpr (MODE == COL_FWD) {   // first kernel of the type-2 chain
            col_tma_kernel<LOGNP, MODE><<<grid, Cf::P, sm, st>>>(map, omap, omap_h, static_cast<float2*>(dst),
                                                                 static_cast<const float2*>(P->d.tw), a, nfull,
                                                                 nitems, nboxes, nz, P->d.err);
        } else {
            e = launch_chained(col_tma_kernel<LOGNP, MODE>, dim3(grid), dim3(Cf::P), sm, st, map, omap, omap_h,
                               static_cast<float2*>(dst), static_cast<const float2*>(P->d.tw), a, nfull, nitems,
                               nboxes, nz, P->d.err);
            if (e != cudaSuccess) return e;
        }
        return cudaGetLastError();
    }
}

// all FFT stages of one precision and one N'
template <typename V, int LOGNP> struct Stages {
    static constexpr bool kTma = sizeof(V) == 8;
    template <int MODE>
    static cudaError_t col(const nuasm_plan_s* P, const void* src, void* dst, int ncols, int src_cols, int src_rows,
                           int src_pitch, int load_rows, cudaStream_t s) {
        if constexpr (kTma) {
            const cudaError_t e = launch_col_tma<LOGNP, MODE>(P, src, dst, ncols, src_cols, src_rows, src_pitch,
                                                              load_rows, s);
            if (e != cudaErrorNotSupported) return e;
        }
        const int halves = (MODE == COL_FWD_FOLD || MODE == COL_INV_FOLD) ? 2 : 1;
        return launch_col<V, LOGNP, MODE>(P, src, dst, ncols, halves, s);
    }
    static cudaError_t col_fwd_fold(const nuasm_plan_s* P, cudaStream_t s) {
        const Geometry& g = P->g;
        return col<COL_FWD_FOLD>(P, P->d.win, P->d.bufA, g.W, g.W, g.W, g.Wp, g.np + (g.np < 256 ? g.np : 256), s);
    }
    static cudaError_t col_inv(const nuasm_plan_s* P, void* u2, cudaStream_t s) {
        const Geometry& g = P->g;
        return col<COL_INV>(P, P->d.bufB, u2, g.n, g.n, g.np, g.n, g.np, s);
    }
    static cudaError_t col_fwd(const nuasm_plan_s* P, const void* u1, cudaStream_t s) {
        const Geometry& g = P->g;
        return col<COL_FWD>(P, u1, P->d.bufB, g.n, g.n, g.n, g.n, g.n, s);
    }
    static cudaError_t col_inv_fold(const nuasm_plan_s* P, cudaStream_t s) {
        const Geometry& g = P->g;
        return col<COL_INV_FOLD>(P, P->d.bufA, P->d.win, g.W, g.W, g.np, g.Wp, g.np, s);
    }
    static cudaError_t row(const nuasm_plan_s* P, int type, cudaStream_t s) { return launch_row<V, LOGNP>(P, type, s); }
};

// dispatch on log2 N' (5 .. LOGMAX) at run time
template <typename V, int LOGMAX, class F> cudaError_t dispatch(int lognp, F&& f) {
    switch (lognp) {
        case 5: return f(Stages<V, 5>{});
        case 6: return f(Stages<V, 6>{});
        case 7: return f(Stages<V, 7>{});
        case 8: return f(Stages<V, 8>{});
        case 9: return f(Stages<V, 9>{});
        case 10: return f(Stages<V, 10>{});
        case 11: return f(Stages<V, 11>{});
        case 12: return f(Stages<V, 12>{});
        case 13:
            if constexpr (LOGMAX >= 13) return f(Stages<V, 13>{});
            else return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace passes
}  // namespace nuasm
