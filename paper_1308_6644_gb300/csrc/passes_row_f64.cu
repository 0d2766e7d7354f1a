// Row-pass instantiations of FP64 plans: every supported N' is compiled here
// so that the radix schedule, the rows per CTA and the launch bounds are
// constants.  From N' = 512 up the passes compute in double-float arithmetic
// (dfc, on the FP32 pipe) over the plan's FP64 arrays; below, where a pass
// has few rows and is bound by the latency of its dependent operations
// rather than by their rate, in FP64 (double2).  NUASM_F64_DF_ROWS=0 keeps
// FP64 throughout.
#include "passes.cuh"

#ifndef NUASM_F64_DF_ROWS
#define NUASM_F64_DF_ROWS 1
#endif

namespace nuasm {

cudaError_t row_f64(const nuasm_plan_s* P, int type, cudaStream_t s) {
    using R = std::conditional_t<NUASM_F64_DF_ROWS != 0, dfc, double2>;
    auto run = [&](auto st) -> cudaError_t { return decltype(st)::row(P, type, s); };
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
