// Column-pass instantiations of FP64 plans for every supported N': from
// N' = 512 up in double-float arithmetic (dfc, on the FP32 pipe) over the
// plan's FP64 arrays, below in FP64 (double2), as the row passes.
// NUASM_F64_DF_COLS=0 keeps FP64 throughout.
#include "passes.cuh"

#ifndef NUASM_F64_DF_COLS
#define NUASM_F64_DF_COLS 1
#endif

namespace nuasm {

cudaError_t col_f64(const nuasm_plan_s* P, int mode, const void* ext, cudaStream_t s) {
    using R = std::conditional_t<NUASM_F64_DF_COLS != 0, dfc, double2>;
    auto run = [&](auto st) -> cudaError_t {
        using S = decltype(st);
        switch (mode) {
            case passes::COL_FWD_FOLD: return S::col_fwd_fold(P, s);
            case passes::COL_INV: return S::col_inv(P, const_cast<void*>(ext), s);
            case passes::COL_FWD: return S::col_fwd(P, ext, s);
            default: return S::col_inv_fold(P, s);
        }
    };
    switch (P->g.lognp) {
        case 5: return run(passes::Stages<double2, 5>{});
        case 6: return run(passes::Stages<double2, 6>{});
        case 7: return run(passes::Stages<double2, 7>{});
        case 8: return run(passes::Stages<double2, 8>{});
        case 9: return run(passes::Stages<R, 9>{});
        case 10: return run(passes::Stages<R, 10>{});
        case 11: return run(passes::Stages<R, 11>{});
        case 12: return run(passes::Stages<R, 12>{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nuasm
