// Device-side helpers shared by the NU-ASM kernels: complex arithmetic on
// float2/double2, double-float (compensated FP32) arithmetic, padding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nuasm {

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

template <typename V> struct CTraits;
template <> struct CTraits<float2> {
    using real = float;
    static constexpr int pad_shift = 4;   // one pad slot per 16 elements (128 B)
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct CTraits<double2> {
    using real = double;
    static constexpr int pad_shift = 3;   // one pad slot per 8 elements (128 B)
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};

// multiply by -i (DIR = -1) or +i (DIR = +1)
template <int DIR, typename V> __device__ __forceinline__ V mul_i(V a) {
    using C = CTraits<V>;
    return DIR < 0 ? C::make(a.y, -a.x) : C::make(-a.y, a.x);
}

// shared-memory padding: one spare slot every 128 bytes breaks the power-of-two
// strides of the first Stockham pass across banks
template <typename V> __device__ __forceinline__ int spad(int q) {
    return q + (q >> CTraits<V>::pad_shift);
}
template <typename V> __host__ __device__ constexpr int spad_size(int n) {
    return n + (n >> (sizeof(V) == 8 ? 4 : 3)) + 1;
}

// ---------------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two floats (Dekker / Knuth error-free transforms).
struct df { float hi, lo; };

__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    df t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df df_div(df a, df b) {
    float q = a.hi / b.hi;
    // remainder a - q b, exact leading part through fma
    float r = fmaf(-q, b.hi, a.hi);
    r = r + a.lo - q * b.lo;
    float ql = r / b.hi;
    return df_fast_two_sum(q, ql);
}
__device__ __forceinline__ df df_sqrt(df a) {
    float y = sqrtf(a.hi);
    if (y == 0.f) return {0.f, 0.f};
    float e = fmaf(-y, y, a.hi) + a.lo;
    return df_fast_two_sum(y, e / (2.f * y));
}

}  // namespace nuasm
