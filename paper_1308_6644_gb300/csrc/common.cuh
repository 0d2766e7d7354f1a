// Device-side helpers shared by the NU-ASM kernels: complex arithmetic on
// float2/double2, double-float (compensated FP32) arithmetic, padding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nuasm {

// ---------------------------------------------------------------- programmatic dependent launch
// The kernels of an execute chain after the first can be launched with
// programmatic stream serialisation (launch_chained): every kernel lets the
// next one launch as soon as all of its own CTAs are running
// (pdl_allow_next), and the next one runs its prologue -- index arithmetic,
// plan-constant loads -- before pdl_wait(), which returns once the previous
// grid has completed and its writes are visible.  Nothing before pdl_wait()
// reads what the previous kernel writes or writes what it reads.  Without the
// launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// 16-byte asynchronous global -> shared copies (both addresses 16-byte aligned).
// The issuing thread waits with cp_async_wait_all; a barrier after that wait
// makes the data visible to the block.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Off by default: measured on the NU-ASM_2 N = 1024 chain it cost 3.5 us per
// solve (131.1 -> 134.6 us) and changed nothing at N = 2048 or in batches.
#ifndef NUASM_PDL
#define NUASM_PDL 0   // 1: launch_chained sets programmatic stream serialisation
#endif

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = NUASM_PDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- debug bounds checks
// The debug library (built with NUASM_DEBUG_BOUNDS=1) checks the shared- and
// global-memory indices and the TMA coordinates its kernels compute against
// the extents of the buffers they address, skips any access that would fall
// outside, and records per translation unit how many were skipped and the
// first one (site, index, extent); nuasm_debug_bounds reads and clears the
// records.  It stands in for a memory checker.  In the normal build every
// check is the constant true and compiles away.
#ifndef NUASM_DEBUG_BOUNDS
#define NUASM_DEBUG_BOUNDS 0
#endif
namespace dbg {
enum Site : int {
    kFftLoad = 1, kFftStore = 2, kTmaLoad = 3, kTmaStore = 4,
    kColLoad = 10, kColStore = 11, kColRaw = 12, kColStage = 13,
    kRowLoad = 20, kRowStore = 21, kRowModes = 22,
    kBinRec = 30, kSpreadRec = 31, kSpreadValue = 32, kSpreadPlane = 33, kSpreadWindow = 34,
    kInterpRec = 40, kInterpTile = 41, kInterpOut = 42,
};
struct Record {
    unsigned int hits;
    int site;
    long long index, limit;
};
using Reader = cudaError_t (*)(Record*, bool reset);
int add_reader(Reader r);   // diag.cu: every translation unit's reader
}  // namespace dbg
#if NUASM_DEBUG_BOUNDS
namespace dbg {
static __device__ Record rec_;   // one per translation unit
static __device__ __noinline__ bool miss(long long i, long long n, int site) {
    if (atomicAdd(&rec_.hits, 1u) == 0) {
        rec_.site = site;
        rec_.index = i;
        rec_.limit = n;
    }
    return false;
}
__device__ __forceinline__ bool in_range(long long i, long long n, int site) {
    return (i >= 0 && i < n) ? true : miss(i, n, site);
}
static cudaError_t read_rec(Record* out, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, rec_, sizeof(Record));
    if (e == cudaSuccess && reset) {
        const Record zero = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(rec_, &zero, sizeof(Record));
    }
    return e;
}
[[maybe_unused]] static const int registered_ = add_reader(&read_rec);
}  // namespace dbg
#define NUASM_IN_RANGE(i, n, site) ::nuasm::dbg::in_range((long long)(i), (long long)(n), (site))
#else
#define NUASM_IN_RANGE(i, n, site) true
#endif

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
template <typename V> __host__ __device__ __forceinline__ constexpr int spad(int q) {
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
