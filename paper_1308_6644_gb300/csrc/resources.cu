// Resource acquisition of the library: every device, pool and pinned host
// allocation, and every stream, event and graph instantiation, goes through
// these wrappers.  They keep a count of the acquisitions alive and carry a
// test hook that makes the k-th acquisition from now fail as if the device
// had run out of memory, so that the clean-up paths of nuasm_plan,
// nuasm_batch_create and the server can be exercised without exhausting a
// GPU (nuasm_debug_fail_alloc / nuasm_debug_live_resources in nuasm.h).
#include <cuda_runtime.h>

#include <atomic>

#include "nuasm_internal.h"

namespace nuasm {

namespace {

std::atomic<int64_t> g_fail_at{0};   // 0: off; k: the k-th acquisition from now fails
std::atomic<int64_t> g_live{0};      // acquisitions not yet released

}  // namespace

bool acquire_fails() {
    int64_t k = g_fail_at.load(std::memory_order_relaxed);
    while (k > 0) {
        if (g_fail_at.compare_exchange_weak(k, k - 1, std::memory_order_relaxed))
            return k == 1;   // this acquisition took the count from 1 to 0
    }
    return false;
}

void live_add(int64_t d) { g_live.fetch_add(d, std::memory_order_relaxed); }

cudaError_t xmalloc(void** p, size_t bytes) {
    *p = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) live_add(1);
    return e;
}

cudaError_t xmalloc_async(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e == cudaSuccess) live_add(1);
    return e;
}

cudaError_t xmalloc_pool(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s) {
    *p = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    if (e == cudaSuccess) live_add(1);
    return e;
}

cudaError_t xmalloc_host(void** p, size_t bytes, unsigned flags) {
    *p = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaHostAlloc(p, bytes ? bytes : 16, flags);
    if (e == cudaSuccess) live_add(1);
    return e;
}

void xfree(void* p) {
    if (!p) return;
    cudaFree(p);
    live_add(-1);
}

void xfree_async(void* p, cudaStream_t s) {
    if (!p) return;
    cudaFreeAsync(p, s);
    live_add(-1);
}

void xfree_host(void* p) {
    if (!p) return;
    cudaFreeHost(p);
    live_add(-1);
}

cudaError_t xstream_create(cudaStream_t* s) {
    *s = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    if (e == cudaSuccess) live_add(1);
    return e;
}

void xstream_destroy(cudaStream_t s) {
    if (!s) return;
    cudaStreamDestroy(s);
    live_add(-1);
}

cudaError_t xevent_create(cudaEvent_t* ev, unsigned flags) {
    *ev = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaEventCreateWithFlags(ev, flags);
    if (e == cudaSuccess) live_add(1);
    return e;
}

void xevent_destroy(cudaEvent_t ev) {
    if (!ev) return;
    cudaEventDestroy(ev);
    live_add(-1);
}

cudaError_t xgraph_instantiate(cudaGraphExec_t* exec, cudaGraph_t graph) {
    *exec = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
    if (e == cudaSuccess) live_add(1);
    return e;
}

void xgraph_exec_destroy(cudaGraphExec_t exec) {
    if (!exec) return;
    cudaGraphExecDestroy(exec);
    live_add(-1);
}

cudaError_t xpool_create(cudaMemPool_t* pool, const cudaMemPoolProps* props) {
    *pool = nullptr;
    if (acquire_fails()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMemPoolCreate(pool, props);
    if (e == cudaSuccess) live_add(1);
    return e;
}

cudaError_t xpool_destroy(cudaMemPool_t pool) {
    if (!pool) return cudaSuccess;
    const cudaError_t e = cudaMemPoolDestroy(pool);
    live_add(-1);
    return e;
}

}  // namespace nuasm

extern "C" {

nuasm_status nuasm_debug_fail_alloc(int64_t k) {
    if (k < 0) return NUASM_EINVAL;
    nuasm::g_fail_at.store(k, std::memory_order_relaxed);
    return NUASM_OK;
}

nuasm_status nuasm_debug_live_resources(int64_t* count) {
    if (!count) return NUASM_EINVAL;
    *count = nuasm::g_live.load(std::memory_order_relaxed);
    return NUASM_OK;
}

}  // extern "C"
