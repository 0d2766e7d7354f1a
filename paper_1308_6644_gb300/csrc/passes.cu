// Precision dispatch of the FFT stages (kernels in passes.cuh, instantiated in
// passes_{row,col}_{f32,f64}.cu).
#include <cudaTypedefs.h>

#include <mutex>

#include "nuasm_internal.h"
#include "tma.cuh"

namespace nuasm {

bool encode_map_8b(CUtensorMap* map, const void* base, int cols, int rows, int pitch, int box_cols, int box_rows) {
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

}  // namespace nuasm
