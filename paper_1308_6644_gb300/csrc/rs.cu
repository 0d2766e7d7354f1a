// Rayleigh-Sommerfeld diffraction (Eq. 10) as a direct sum on the GPU: the
// O(M1 M2) reference the paper compares NU-ASM and NU-FRE against.
//
//   u2(x2) = (1/2 pi) sum_j a_j c_j (z/r)(1 - i k r) exp(i k r) / r^2,
//   r = sqrt(|x2 + o - x1_j|^2 + z^2),  k = 2 pi / lambda,
//
// with a_j the area element of source sample j.  The phase is split as
// k r = 2 pi (frac(z/lambda) + (r - z)/lambda), r - z = rho^2 / (r + z), so
// FP32 keeps ~1e-5-cycle accuracy for the geometries of the paper's
// experiments; the FP64 variant evaluates everything in double precision.
// One thread owns one destination point; source samples stream through
// shared memory in tiles of the block size.
#include <cuda_runtime.h>

#include <cmath>

#include "nuasm_internal.h"

namespace nuasm {
namespace {

constexpr int kThreads = 256;

struct Src64 { double x, y, re, im; };

struct RsArgs {
    double lam, z, ox, oy, zfrac;
    int64_t m1, m2;
};

__global__ void __launch_bounds__(kThreads) rs_f32_kernel(const double* __restrict__ x1, const double* __restrict__ y1,
                                                          const float2* __restrict__ c, const double* __restrict__ area,
                                                          const double* __restrict__ x2, const double* __restrict__ y2,
                                                          float2* __restrict__ out, RsArgs a) {
    __shared__ float4 src[kThreads];   // x, y, re(a c), im(a c)
    const int64_t t = blockIdx.x * int64_t(kThreads) + threadIdx.x;
    const bool live = t < a.m2;
    const float px = live ? float(x2[t] + a.ox) : 0.f, py = live ? float(y2[t] + a.oy) : 0.f;
    const float z = float(a.z), z2 = z * z, il = float(1.0 / a.lam), zf = float(a.zfrac);
    const float k = float(2.0 * M_PI / a.lam);
    float ar = 0.f, ai = 0.f;
    for (int64_t base = 0; base < a.m1; base += kThreads) {
        const int64_t j = base + threadIdx.x;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < a.m1) {
            const float2 v = c[j];
            const float w = float(area[j]);
            s = make_float4(float(x1[j]), float(y1[j]), v.x * w, v.y * w);
        }
        __syncthreads();
        src[threadIdx.x] = s;
        __syncthreads();
        const int cnt = int(a.m1 - base < kThreads ? a.m1 - base : kThreads);
        for (int q = 0; q < cnt; ++q) {
            const float4 sq = src[q];
            const float dx = px - sq.x, dy = py - sq.y;
            const float rho2 = fmaf(dx, dx, dy * dy);
            const float r = sqrtf(rho2 + z2);
            float ph = zf + (rho2 / (r + z)) * il;
            ph -= rintf(ph);
            float sn, cs;
            sincospif(2.f * ph, &sn, &cs);
            const float amp = z / (r * r * r);
            const float kr = k * r;
            // (1 - i k r)(cs + i sn) = (cs + kr sn) + i (sn - kr cs)
            const float kre = amp * fmaf(kr, sn, cs), kim = amp * fmaf(-kr, cs, sn);
            ar = fmaf(sq.z, kre, fmaf(-sq.w, kim, ar));
            ai = fmaf(sq.z, kim, fmaf(sq.w, kre, ai));
        }
    }
    if (live) out[t] = make_float2(ar * float(0.5 / M_PI), ai * float(0.5 / M_PI));
}

__global__ void __launch_bounds__(kThreads) rs_f64_kernel(const double* __restrict__ x1, const double* __restrict__ y1,
                                                          const double2* __restrict__ c, const double* __restrict__ area,
                                                          const double* __restrict__ x2, const double* __restrict__ y2,
                                                          double2* __restrict__ out, RsArgs a) {
    __shared__ Src64 src[kThreads];
    const int64_t t = blockIdx.x * int64_t(kThreads) + threadIdx.x;
    const bool live = t < a.m2;
    const double px = live ? x2[t] + a.ox : 0.0, py = live ? y2[t] + a.oy : 0.0;
    const double z = a.z, z2 = z * z, il = 1.0 / a.lam, k = 2.0 * M_PI / a.lam;
    double ar = 0.0, ai = 0.0;
    for (int64_t base = 0; base < a.m1; base += kThreads) {
        const int64_t j = base + threadIdx.x;
        Src64 s{0.0, 0.0, 0.0, 0.0};
        if (j < a.m1) {
            const double2 v = c[j];
            s = Src64{x1[j], y1[j], v.x * area[j], v.y * area[j]};
        }
        __syncthreads();
        src[threadIdx.x] = s;
        __syncthreads();
        const int cnt = int(a.m1 - base < kThreads ? a.m1 - base : kThreads);
        for (int q = 0; q < cnt; ++q) {
            const Src64 sq = src[q];
            const double dx = px - sq.x, dy = py - sq.y;
            const double rho2 = dx * dx + dy * dy;
            const double r = sqrt(rho2 + z2);
            double ph = a.zfrac + (rho2 / (r + z)) * il;
            ph -= rint(ph);
            double sn, cs;
            sincospi(2.0 * ph, &sn, &cs);
            const double amp = z / (r * r * r), kr = k * r;
            const double kre = amp * (cs + kr * sn), kim = amp * (sn - kr * cs);
            ar += sq.re * kre - sq.im * kim;
            ai += sq.re * kim + sq.im * kre;
        }
    }
    if (live) out[t] = make_double2(ar * (0.5 / M_PI), ai * (0.5 / M_PI));
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace nuasm

extern "C" nuasm_status nuasm_rs_direct(const nuasm_params_t* p, int64_t m1, const double* x1, const double* y1,
                                        const void* c, const double* area, int64_t m2, const double* x2,
                                        const double* y2, void* out, void* stream) {
    using namespace nuasm;
    if (!p || m1 < 0 || m2 < 0) return NUASM_EINVAL;
    if (!std::isfinite(p->lambda) || !(p->lambda > 0) || !std::isfinite(p->z) || !(p->z > 0) ||
        !std::isfinite(p->ox) || !std::isfinite(p->oy))
        return NUASM_EINVAL;
    if (p->prec != NUASM_PREC_F32_F64PHASE && p->prec != NUASM_PREC_F64) return NUASM_EINVAL;
    if (m2 == 0) return NUASM_OK;
    if (!x2 || !y2 || !out || (m1 > 0 && (!x1 || !y1 || !c || !area))) return NUASM_EINVAL;
    const void* ptrs[] = {x2, y2, out};
    for (const void* q : ptrs)
        if (!on_device(q)) return NUASM_EINVAL;
    if (m1 > 0) {
        const void* sp[] = {x1, y1, c, area};
        for (const void* q : sp)
            if (!on_device(q)) return NUASM_EINVAL;
    }
    // z / lambda reduced mod 1 from a double-double quotient
    const double q = p->z / p->lambda;
    const double ql = std::fma(-q, p->lambda, p->z) / p->lambda;
    RsArgs a{p->lambda, p->z, p->ox, p->oy, (q - std::nearbyint(q)) + ql, m1, m2};
    const int64_t blocks = (m2 + kThreads - 1) / kThreads;
    if (blocks > (int64_t(1) << 31) - 1) return NUASM_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->prec == NUASM_PREC_F64)
        rs_f64_kernel<<<unsigned(blocks), kThreads, 0, st>>>(x1, y1, static_cast<const double2*>(c), area, x2, y2,
                                                             static_cast<double2*>(out), a);
    else
        rs_f32_kernel<<<unsigned(blocks), kThreads, 0, st>>>(x1, y1, static_cast<const float2*>(c), area, x2, y2,
                                                             static_cast<float2*>(out), a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}
