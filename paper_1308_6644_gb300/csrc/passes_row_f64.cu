// Row-pass instantiations (double2): every supported N' is compiled here so that
// the radix schedule, the rows per CTA and the launch bounds are constants.
#include "passes.cuh"

namespace nuasm {

cudaError_t row_f64(const nuasm_plan_s* P, int type, cudaStream_t s) {
    return passes::dispatch<double2, 12>(P->g.lognp, [&](auto st) -> cudaError_t { return decltype(st)::row(P, type, s); });
}

}  // namespace nuasm
