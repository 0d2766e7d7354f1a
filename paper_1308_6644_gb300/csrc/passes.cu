// Precision dispatch of the FFT stages (kernels in passes.cuh, instantiated in
// passes_{row,col}_{f32,f64}.cu).
#include "nuasm_internal.h"

namespace nuasm {

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

}  // namespace nuasm
