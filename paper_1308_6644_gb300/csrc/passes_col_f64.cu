// Column-pass instantiations (double2) for every supported N'.
#include "passes.cuh"

namespace nuasm {

cudaError_t col_f64(const nuasm_plan_s* P, int mode, const void* ext, cudaStream_t s) {
    return passes::dispatch<double2, 12>(P->g.lognp, [&](auto st) -> cudaError_t {
        using S = decltype(st);
        switch (mode) {
            case passes::COL_FWD_FOLD: return S::col_fwd_fold(P, s);
            case passes::COL_INV: return S::col_inv(P, const_cast<void*>(ext), s);
            case passes::COL_FWD: return S::col_fwd(P, ext, s);
            default: return S::col_inv_fold(P, s);
        }
    });
}

}  // namespace nuasm
