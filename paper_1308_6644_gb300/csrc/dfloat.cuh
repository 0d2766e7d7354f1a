// Double-float real and complex types for the FFT passes of FP64 plans
// (FFT engine arithmetic on the FP32 pipe).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace nuasm {

// ---------------------------------------------------------------- double-float complex
// A real hi + lo of two floats (about 47 significant bits) and a complex of
// two of them, for FFT passes of FP64 plans on the FP32 pipe.  Sums use the
// two-sum of the high parts with the low parts added to its error term, and
// products the FMA error of the high parts; both renormalise once.
struct dfr {
    float hi, lo;
    dfr() = default;
    __host__ __device__ constexpr dfr(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit dfr(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
};
__host__ __device__ constexpr dfr operator-(dfr a) { return dfr(-a.hi, -a.lo); }
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = s + e;
    return dfr(h, e - (h - s));
}
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
    const float h = p + e;
    return dfr(h, e - (h - p));
}
// k a for a small integer k (the FFT engine's direction signs)
__device__ __forceinline__ dfr operator*(int k, dfr a) {
    return k == 1 ? a : k == -1 ? -a : dfr(float(k), 0.f) * a;
}
struct __align__(16) dfc {
    dfr x, y;
};
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc cmul(dfc a, dfc b) { return dfc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dfc cconj(dfc a) { return dfc{a.x, -a.y}; }
template <> struct CTraits<dfc> {
    using real = dfr;
    static constexpr int pad_shift = 3;   // 16-byte elements, as complex128
    __device__ static dfc zero() { return dfc{dfr(0.f, 0.f), dfr(0.f, 0.f)}; }
    __device__ static dfc make(dfr a, dfr b) { return dfc{a, b}; }
};

// read-only cached load of a table entry (complex types of 8 or 16 bytes, reals)
template <typename T> __device__ __forceinline__ T ldgv(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfc ldgv<dfc>(const dfc* p) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    return dfc{dfr(q.x, q.y), dfr(q.z, q.w)};
}

// 2^k as a double for k in [-1022, 1023]
__device__ __forceinline__ double dfr_pow2(int k) {
    return __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}

// x 2^-s (s in [-1022, 1023]) as a double-float by integer operations on the
// bits: hi the leading 24 significant bits of x (truncated), lo the next 23,
// relative error below 2^-46.  The caller picks s so that the result stays
// within the float range.  A subnormal x is first scaled by 2^-s in FP64
// (exact while the product is normal); zeros and values below 2^-100 after
// the scaling give zero, infinities and NaNs give themselves in hi.
__device__ __forceinline__ dfr dfr_split(double x, int s) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    int ex = int(b >> 52) & 0x7ff;
    if (ex == 0x7ff) return dfr(__double2float_rn(x), 0.f);
    if (ex == 0) {   // zero or subnormal
        if ((b << 1) == 0 || s > -923) return dfr(0.f, 0.f);   // zero, or below 2^-100 of 2^s
        b = static_cast<unsigned long long>(__double_as_longlong(x * dfr_pow2(-s)));
        ex = int(b >> 52) & 0x7ff;
        s = 0;
    }
    const int e = ex - 1023 - s;
    if (e < -100) return dfr(0.f, 0.f);
    const unsigned sign = unsigned(b >> 32) & 0x80000000u;
    const unsigned hb = sign | (unsigned(e + 127) << 23) | unsigned((b >> 29) & 0x7fffffu);
    const unsigned r = unsigned(b) & 0x1fffffffu;   // the 29 mantissa bits below hi
    const unsigned lb = unsigned(e - 23 + 127) << 23;
    const float lo = __uint_as_float(lb | (r >> 6)) - __uint_as_float(lb);   // (r >> 6) 2^(e - 46), exact
    return dfr(__uint_as_float(hb), sign ? -lo : lo);
}

// (hi + lo) 2^s as a double by integer operations (the 53 leading bits of
// the exact sum, truncated), for a normalised pair (|lo| below ulp(hi)); a
// result outside the normal double range (subnormal, or beyond the largest
// double) is formed in FP64 arithmetic instead.  Zeros and subnormal hi give
// zero; infinities and NaNs give themselves.
__device__ __forceinline__ double dfr_to_double(dfr a, int s) {
    const unsigned hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
    const int eh = int(hb >> 23) & 0xff;
    if (eh == 0) return 0.0;
    if (eh == 0xff) return double(a.hi);
    // |hi| = Mh 2^(eh - 150); X = Mh 2^39 in units of 2^(eh - 189)
    long long X = static_cast<long long>((hb & 0x7fffffu) | 0x800000u) << 39;
    const int el = int(lb >> 23) & 0xff;
    if (el != 0) {
        const long long L = static_cast<long long>((lb & 0x7fffffu) | 0x800000u);
        const int d = eh - el;   // lo's mantissa sits d bits below hi's
        const long long Ls = d <= 39 ? (d >= 0 ? L << (39 - d) : 0) : (d - 39 < 63 ? L >> (d - 39) : 0);
        X = ((hb ^ lb) >> 31) ? X - Ls : X + Ls;
    }
    const int lz = __clzll(X);                  // leading bit at 63 - lz
    const int E = eh - 126 - lz + s;            // unbiased exponent of the result
    if (E < -1022 || E > 1023) {                // s is within [-1022, 1023]: two exact halves
        const int s1 = s / 2;
        return ((double(a.hi) + double(a.lo)) * dfr_pow2(s1)) * dfr_pow2(s - s1);
    }
    const unsigned long long m = lz <= 11 ? static_cast<unsigned long long>(X) >> (11 - lz)
                                          : static_cast<unsigned long long>(X) << (lz - 11);
    const unsigned long long bits = (static_cast<unsigned long long>(hb >> 31) << 63) |
                                    (static_cast<unsigned long long>(E + 1023) << 52) | (m & 0xfffffffffffffull);
    return __longlong_as_double(static_cast<long long>(bits));
}

}  // namespace nuasm
