// Precision dispatch of the FFT stages (kernels in passes.cuh, instantiated in
// passes_{row,col}_{f32,f64}.cu).
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "nuasm_internal.h"
#include "tma.cuh"

namespace nuasm {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return encode;
}
}  // namespace

bool encode_store_map_8b(CUtensorMap* map, void* base, int cols, int planes, int rows, int pitch, int box_cols,
                         int box_planes, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode || !base || (reinterpret_cast<uintptr_t>(base) & 15) || ((int64_t(pitch) * 8) & 15)) return false;
    if (box_cols < 2 || box_cols > 256 || ((box_cols * 8) & 15) || box_planes < 1 || box_planes > planes ||
        box_rows < 1 || box_rows > 256 || cols < 1 || planes < 1 || rows < 1)
        return false;
    const cuuint64_t dims[3] = {cuuint64_t(cols), cuuint64_t(planes), cuuint64_t(rows)};
    const cuuint64_t strides[2] = {cuuint64_t(pitch) * 8u, cuuint64_t(pitch) * 8u * cuuint64_t(planes)};
    const cuuint32_t box[3] = {cuuint32_t(box_cols), cuuint32_t(box_planes), cuuint32_t(box_rows)};
    const cuuint32_t estride[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_map_8b(CUtensorMap* map, const void* base, int cols, int rows, int pitch, int box_cols, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode || !base || (reinterpret_cast<uintptr_t>(base) & 15) || ((int64_t(pitch) * 8) & 15)) return false;
    if (box_cols < 2 || box_cols > 256 || box_rows < 1 || box_rows > 256 || ((box_cols * 8) & 15)) return false;
    const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(pitch) * 8u};
    const cuuint32_t box[2] = {cuuint32_t(box_cols), cuuint32_t(box_rows)};
    const cuuint32_t estride[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t row_f32(const nuasm_plan_s* P, int type, cudaStream_t s);
cudaError_t row_f64(const nuasm_plan_s* P, int type, cudaStream_t s);
cudaError_t col_f32(const nuasm_plan_s* P, int mode, const void* ext, cudaStream_t s);
cudaError_t col_f64(const nuasm_plan_s* P, int mode, const void* ext, cudaStream_t s);

namespace {
cudaError_t col(const nuasm_plan_s* P, int mode, const void* ext, cudaStream_t s) {
    return P->f64 ? col_f64(P, mode, ext, s) : col_f32(P, mode, ext, s);
}
}  // namespace

// modes follow passes::ColMode: 0 forward fold, 1 inverse, 2 forward, 3 inverse fold
cudaError_t launch_col_fwd_fold(const nuasm_plan_s* P, cudaStream_t s) { return col(P, 0, nullptr, s); }
cudaError_t launch_col_inv(const nuasm_plan_s* P, void* u2, cudaStream_t s) { return col(P, 1, u2, s); }
cudaError_t launch_col_fwd(const nuasm_plan_s* P, const void* u1, cudaStream_t s) { return col(P, 2, u1, s); }
cudaError_t launch_col_inv_fold(const nuasm_plan_s* P, cudaStream_t s) { return col(P, 3, nullptr, s); }
cudaError_t launch_row_t1(const nuasm_plan_s* P, cudaStream_t s) {
    return P->f64 ? row_f64(P, 1, s) : row_f32(P, 1, s);
}
cudaError_t launch_row_t2(const nuasm_plan_s* P, cudaStream_t s) {
    return P->f64 ? row_f64(P, 2, s) : row_f32(P, 2, s);
}
cudaError_t launch_row_t3(const nuasm_plan_s* P, cudaStream_t s) {
    return P->f64 ? row_f64(P, 3, s) : row_f32(P, 3, s);
}

// The non-separable part of the ASM phase (Eq. 4), E = exp(-2 pi i rc Q(s)^2),
// Q(s) = s / (1 + sqrt(1 - s)), s = lambda^2 |f|^2, tabulated once per plan in
// FP64 for |kx| = a and |ky| = b in [0, N'/2] (s = c (a^2 + b^2),
// c = (lambda / (N' pitch))^2); evanescent modes (s >= 1) hold 0.  Row b holds
// `pitch` entries (N'/2 + 1 rounded up to even, so rows start 16-byte aligned).
size_t etab_elems(const Geometry& g, int* pitch) {
    const int half = g.np / 2;
    *pitch = (half + 2) & ~1;
    return size_t(half + 1) * size_t(*pitch);
}

namespace {
template <typename V>
__global__ void etab_kernel(V* __restrict__ out, int half, int pitch, double c, double rc) {
    const int64_t total = int64_t(half + 1) * pitch;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int b = int(i / pitch), a = int(i - int64_t(b) * pitch);
        double re = 0.0, im = 0.0;
        if (a <= half) {
            const double sv = c * (double(a) * a + double(b) * b);
            if (sv < 1.0) {
                const double q = sv / (1.0 + sqrt(1.0 - sv));
                const double r = rc * q * q;
                sincospi(-2.0 * (r - rint(r)), &im, &re);
            }
        }
        out[i] = CTraits<V>::make(re, im);
    }
}
}  // namespace

namespace {
__global__ void etab2_kernel(float2* __restrict__ out, const float2* __restrict__ etab, const float2* __restrict__ tx,
                             int np, int pitch) {
    const int64_t total = int64_t(np / 2 + 1) * np;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int b = int(i / np), q = int(i - int64_t(b) * np);
        out[i] = cmul(tx[q], etab[size_t(b) * pitch + min(q, np - q)]);
    }
}
}  // namespace

cudaError_t build_etab2(const nuasm_plan_s* P, cudaStream_t s) {
    if (!P->d.etab || !P->d.etab2 || P->f64) return cudaErrorInvalidValue;
    const int np = P->g.np;
    const size_t n = size_t(np / 2 + 1) * np;
    const int threads = 256;
    const int blocks = int(std::min<size_t>((n + threads - 1) / threads, size_t(152) * 8));
    etab2_kernel<<<blocks, threads, 0, s>>>(static_cast<float2*>(P->d.etab2), static_cast<const float2*>(P->d.etab),
                                            static_cast<const float2*>(P->d.t2x), np, P->etab_pitch);
    return cudaGetLastError();
}

cudaError_t build_etab(const nuasm_plan_s* P, cudaStream_t s) {
    int pitch = 0;
    const size_t n = etab_elems(P->g, &pitch);
    if (!P->d.etab || pitch != P->etab_pitch) return cudaErrorInvalidValue;
    const double k = P->p.lambda / (double(P->g.np) * P->p.pitch);
    const int threads = 256;
    const int blocks = int(std::min<size_t>((n + threads - 1) / threads, size_t(152) * 8));
    if (P->f64)
        etab_kernel<<<blocks, threads, 0, s>>>(static_cast<double2*>(P->d.etab), P->g.np / 2, pitch, k * k, P->rc);
    else
        etab_kernel<<<blocks, threads, 0, s>>>(static_cast<float2*>(P->d.etab), P->g.np / 2, pitch, k * k, P->rc);
    return cudaGetLastError();
}

}  // namespace nuasm
