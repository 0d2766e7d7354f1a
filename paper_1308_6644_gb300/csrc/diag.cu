// Diagnostic entry point for the bounded-wait failure path (declared in
// include/nuasm.h).  One CTA waits on an mbarrier that no thread or copy will
// ever complete, with the same bounded try-wait loop the TMA column passes
// use; when the bound runs out it sets bit 2 of the error word, exactly as a
// stalled copy would, and returns.  Nothing is in flight, so there is nothing
// else to wait for or release.
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "nuasm_internal.h"
#include "tma.cuh"

namespace nuasm {
namespace dbg {
namespace {
std::vector<Reader>& readers() {
    static std::vector<Reader> r;   // filled during static initialisation, read afterwards
    return r;
}
}  // namespace
int add_reader(Reader r) {
    readers().push_back(r);
    return int(readers().size());
}
}  // namespace dbg
}  // namespace nuasm

namespace {

__global__ void bounded_wait_kernel(int spins, int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    nuasm::tma::mbar_init(&bar, 1);   // expects one arrival that never comes
    if (!nuasm::tma::mbar_wait(&bar, 0, spins)) atomicOr(err, 2);
}

nuasm_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

}  // namespace

extern "C" nuasm_status nuasm_debug_bounded_wait(int32_t spins, void* stream) {
    if (spins < 1 || spins > nuasm::tma::kSpinLimit) return NUASM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = nullptr;
    cudaError_t e = nuasm::xmalloc_async(reinterpret_cast<void**>(&err), sizeof(int), st);
    if (e != cudaSuccess) return status_of(e);
    int host = 0;
    e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 32, 0, st>>>(spins, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    nuasm::xfree_async(err, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) return status_of(e);
    return (host & 2) ? NUASM_ETIMEOUT : NUASM_OK;
}

// The same wait with a plan's own error word as the flag it sets: what a
// column pass whose copy never arrived leaves behind, without a stalled copy
// (nothing else is in flight).  The plan's next execute call reports it.
extern "C" nuasm_status nuasm_debug_plan_wait(nuasm_plan_t plan, int32_t spins, void* stream) {
    if (!plan || spins < 1 || spins > nuasm::tma::kSpinLimit) return NUASM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bounded_wait_kernel<<<1, 32, 0, st>>>(spins, plan->d.err);
    cudaError_t e = cudaGetLastError();
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    return status_of(e);
}

// Bounds records of the debug library (see the debug bounds checks in
// common.cuh): the number of accesses the kernels skipped as out of range
// since the last reset, summed over translation units, and the first one.
extern "C" nuasm_status nuasm_debug_bounds(int64_t* hits, int32_t* site, int64_t* index, int64_t* limit,
                                           int32_t reset) {
    if (!hits) return NUASM_EINVAL;
#if !NUASM_DEBUG_BOUNDS
    (void)site;
    (void)index;
    (void)limit;
    (void)reset;
    *hits = -1;
    return NUASM_EUNSUPPORTED;
#else
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return status_of(e);
    int64_t total = 0;
    bool first = true;
    for (nuasm::dbg::Reader rd : nuasm::dbg::readers()) {
        nuasm::dbg::Record r{};
        if ((e = rd(&r, reset != 0)) != cudaSuccess) return status_of(e);
        total += r.hits;
        if (r.hits && first) {
            first = false;
            if (site) *site = r.site;
            if (index) *index = r.index;
            if (limit) *limit = r.limit;
        }
    }
    if (first) {
        if (site) *site = 0;
        if (index) *index = 0;
        if (limit) *limit = 0;
    }
    *hits = total;
    return NUASM_OK;
#endif
}
