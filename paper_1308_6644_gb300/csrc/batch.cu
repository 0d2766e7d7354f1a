// Batches of planes recorded into one CUDA graph (declared in include/nuasm.h).
//
// Creation groups the items by the plan whose workspace they write, assigns
// the groups to lanes longest-first (greedy LPT on an estimate of each
// plane's HBM bytes and kernel taps), and captures every plane's launch chain
// on its lane's stream between a fork and a join event of an internal origin
// stream.  Execution is one cudaGraphLaunch.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "nuasm_internal.h"

using namespace nuasm;

struct nuasm_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int lanes = 0;
    int64_t kernels = 0;
    std::vector<nuasm_plan_s*> plans;   // plans whose workspace and error word the graph uses
};

namespace {

constexpr int kMaxLanes = 64;
constexpr int kMaxItems = 65536;

// Work estimate of one solve: grid traffic of the five passes plus the taps.
double plane_cost(const nuasm_plan_s* P, int64_t points) {
    const Geometry& g = P->g;
    const double eb = P->f64 ? 16.0 : 8.0;
    const double grid = eb * (2.0 * ws_win_elems(g) + 2.0 * ws_bufA_elems(g) + 2.0 * ws_bufB_elems(g) +
                              double(g.n) * g.n);
    return grid + double(points) * (24.0 + 2.0 * g.w * g.w);
}

nuasm_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

struct Streams {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> ev;
    ~Streams() {
        for (cudaEvent_t e : ev) xevent_destroy(e);
        for (cudaStream_t q : s) xstream_destroy(q);
    }
};

}  // namespace

extern "C" {

nuasm_status nuasm_batch_create(nuasm_batch_t* out, const nuasm_batch_item_t* items, int32_t count, int32_t lanes) {
    if (!out) return NUASM_EINVAL;
    *out = nullptr;
    if (!items || count < 1 || count > kMaxItems || lanes < 0 || lanes > kMaxLanes) return NUASM_EINVAL;
    if (lanes == 0) lanes = 8;

    // validate and group by the plan whose workspace the item writes
    std::vector<nuasm_plan_s*> owners;
    std::vector<int> group(count);
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) {
        const nuasm_batch_item_t& it = items[i];
        nuasm_plan_s* P = it.plan;
        if (!P || !P->d.win || it.type < 1 || it.type > 3) return NUASM_EINVAL;
        if (it.type == 3) {
            if (!it.dst || !same_problem(P->p, it.dst->p)) return NUASM_EINVAL;
        } else if (it.dst) {
            return NUASM_EINVAL;
        }
        const int64_t m_in = it.type == 2 ? int64_t(P->g.n) * P->g.n : P->m;
        const int64_t m_out = it.type == 1 ? int64_t(P->g.n) * P->g.n : (it.type == 2 ? P->m : it.dst->m);
        if ((m_in > 0 && (!it.in || !device_accessible(it.in))) ||
            (m_out > 0 && (!it.out || !device_accessible(it.out))))
            return NUASM_EINVAL;
        auto f = std::find(owners.begin(), owners.end(), P);
        group[i] = int(f - owners.begin());
        if (f == owners.end()) owners.push_back(P);
        cost[i] = plane_cost(P, it.type == 3 ? P->m + it.dst->m : P->m);
    }

    // longest-processing-time-first assignment of the groups to lanes
    const int ng = int(owners.size());
    std::vector<double> gcost(ng, 0.0);
    for (int i = 0; i < count; ++i) gcost[group[i]] += cost[i];
    std::vector<int> order(ng);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gcost[a] > gcost[b]; });
    const int nl = std::min(lanes, ng);
    std::vector<double> load(nl, 0.0);
    std::vector<int> lane_of(ng);
    for (int gi : order) {
        const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
        lane_of[gi] = l;
        load[l] += gcost[gi];
    }

    Streams S;
    cudaStream_t origin = nullptr;
    cudaError_t e = xstream_create(&origin);
    if (e != cudaSuccess) return status_of(e);
    S.s.push_back(origin);
    for (int l = 0; l < nl; ++l) {
        cudaStream_t q = nullptr;
        if ((e = xstream_create(&q)) != cudaSuccess) return status_of(e);
        S.s.push_back(q);
    }
    for (int l = 0; l <= nl; ++l) {
        cudaEvent_t ev = nullptr;
        if ((e = xevent_create(&ev)) != cudaSuccess) return status_of(e);
        S.ev.push_back(ev);
    }

    if ((e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return status_of(e);
    cudaError_t ce = cudaEventRecord(S.ev[0], origin);
    for (int l = 0; l < nl && ce == cudaSuccess; ++l) {
        cudaStream_t q = S.s[1 + l];
        ce = cudaStreamWaitEvent(q, S.ev[0], 0);
        for (int i = 0; i < count && ce == cudaSuccess; ++i) {
            if (lane_of[group[i]] != l) continue;
            const nuasm_batch_item_t& it = items[i];
            nuasm_plan_s view = *it.plan;   // no per-stage events inside a graph
            view.prof = false;
            if (it.type == 1) ce = chain_type1(&view, it.in, it.out, q);
            else if (it.type == 2) ce = chain_type2(&view, it.in, it.out, q);
            else ce = chain_type3(&view, it.dst, it.in, it.out, q);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(S.ev[1 + l], q);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(origin, S.ev[1 + l], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(origin, &graph);
    if (ce != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return status_of(ce != cudaSuccess ? ce : e);
    }
    cudaGraphExec_t exec = nullptr;
    if ((e = xgraph_instantiate(&exec, graph)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return status_of(e);
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    int64_t kernels = 0;
    if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }

    nuasm_batch_s* B = new (std::nothrow) nuasm_batch_s();
    if (!B) {
        xgraph_exec_destroy(exec);
        cudaGraphDestroy(graph);
        return NUASM_ENOMEM;
    }
    B->graph = graph;
    B->exec = exec;
    B->lanes = nl;
    B->kernels = kernels;
    try {
        B->plans = owners;
    } catch (...) {
        xgraph_exec_destroy(exec);
        cudaGraphDestroy(graph);
        delete B;
        return NUASM_ENOMEM;
    }
    *out = B;
    return NUASM_OK;
}

nuasm_status nuasm_batch_execute(nuasm_batch_t batch, void* stream) {
    if (!batch) return NUASM_EINVAL;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NUASM_ECUDA;
    }
    // a bounded device wait of an earlier launch gave up (host-mapped error words; reported once)
    bool timed_out = false;
    for (nuasm_plan_s* P : batch->plans)
        if (P->d.h_err && (*static_cast<volatile int*>(P->d.h_err) & 2)) {
            __atomic_fetch_and(P->d.h_err, ~2, __ATOMIC_SEQ_CST);
            timed_out = true;
        }
    if (timed_out) return NUASM_ETIMEOUT;
    return status_of(cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream)));
}

nuasm_status nuasm_batch_info(nuasm_batch_t batch, int32_t* lanes, int64_t* kernels) {
    if (!batch || !lanes || !kernels) return NUASM_EINVAL;
    *lanes = batch->lanes;
    *kernels = batch->kernels;
    return NUASM_OK;
}

nuasm_status nuasm_batch_destroy(nuasm_batch_t batch) {
    if (!batch) return NUASM_OK;
    const cudaError_t e = cudaDeviceSynchronize();
    xgraph_exec_destroy(batch->exec);
    cudaGraphDestroy(batch->graph);
    delete batch;
    return status_of(e);
}

}  // extern "C"
