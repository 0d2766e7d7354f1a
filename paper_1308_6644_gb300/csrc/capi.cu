// C ABI of the NU-ASM / NU-FRE library (declared in include/nuasm.h).
//
// Plan: validate -> host FP64 tables (band of Eq. 4, Fresnel tables of Eq. 5,
// deconvolution, twiddles) -> device allocations (tables, workspace, staging)
// -> point binning on the device.  Execute: stream-ordered launches only.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nuasm_internal.h"

#ifndef NUASM_ETAB2
#define NUASM_ETAB2 1   // FP32 plans also tabulate T2x E for the type-2 row pass
#endif

using namespace nuasm;

namespace nuasm {

bool device_accessible(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the non-sticky error of a foreign pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool same_problem(const nuasm_params_t& a, const nuasm_params_t& b) {
    bool same = a.n == b.n && a.n_pad == b.n_pad && a.pitch == b.pitch && a.lambda == b.lambda && a.z == b.z &&
                a.ox == b.ox && a.oy == b.oy && a.band_auto == b.band_auto && a.kind == b.kind &&
                a.prec == b.prec && a.tol == b.tol && a.kernel == b.kernel && a.tile == b.tile;
    if (same && !a.band_auto)
        same = a.c_m == b.c_m && a.c_n == b.c_n && a.w_m == b.w_m && a.w_n == b.w_n;
    return same;
}

}  // namespace nuasm

namespace {

nuasm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

#define NUASM_TRY(expr)                                    \
    do {                                                   \
        cudaError_t e__ = (expr);                          \
        if (e__ != cudaSuccess) return cuda_status(e__);   \
    } while (0)

size_t elt_bytes(const nuasm_plan_s* P) { return P->f64 ? 16 : 8; }

// ---------------------------------------------------------------- profiling ring
struct ProfRing {
    static constexpr int kCap = 64;
    cudaEvent_t start[kCap], stop[kCap];
    int head = 0, count = 0;
    bool created = false;
};

struct PlanExtra {
    ProfRing ring[NUASM_STAGE_COUNT];
};

}  // namespace

static PlanExtra* extra_of(nuasm_plan_s* P) { return static_cast<PlanExtra*>(P->prof_state); }

namespace {

void ring_consume_oldest(nuasm_plan_s* P, int stage) {
    ProfRing& r = extra_of(P)->ring[stage];
    const int idx = (r.head - r.count + ProfRing::kCap) % ProfRing::kCap;
    float ms = 0.f;
    if (cudaEventSynchronize(r.stop[idx]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, r.start[idx], r.stop[idx]) == cudaSuccess) {
        P->prof_ms[stage] += ms;
        P->prof_n[stage] += 1;
    }
    r.count -= 1;
}

// One stage of an execute chain: an NVTX range on the host thread (named as
// nuasm_stage_name; free when no tool is attached) and, when the plan's
// profiling is on, CUDA events around the stage on its stream.
struct StageScope {
    nuasm_plan_s* P;
    int stage;
    cudaStream_t st;
    int slot = -1;
    StageScope(nuasm_plan_s* p, int s, cudaStream_t stream) : P(p), stage(s), st(stream) {
        nvtxRangePushA(nuasm_stage_name(s));
        if (!P->prof) return;
        ProfRing& r = extra_of(P)->ring[stage];
        if (!r.created) {
            for (int i = 0; i < ProfRing::kCap; ++i) {
                cudaEventCreate(&r.start[i]);
                cudaEventCreate(&r.stop[i]);
            }
            r.created = true;
        }
        if (r.count == ProfRing::kCap) ring_consume_oldest(P, stage);
        slot = r.head;
        cudaEventRecord(r.start[slot], st);
    }
    ~StageScope() {
        nvtxRangePop();
        if (slot < 0) return;
        ProfRing& r = extra_of(P)->ring[stage];
        cudaEventRecord(r.stop[slot], st);
        r.head = (r.head + 1) % ProfRing::kCap;
        r.count += 1;
    }
};

}  // namespace

void nuasm::plan_release(nuasm_plan_s* P) {
    if (!P) return;
    PlanExtra* X = extra_of(P);
    if (X) {
        for (auto& r : X->ring)
            if (r.created)
                for (int i = 0; i < ProfRing::kCap; ++i) {
                    cudaEventDestroy(r.start[i]);
                    cudaEventDestroy(r.stop[i]);
                }
        delete X;
    }
    void* ptrs[] = {P->d.tables, P->d.etab, P->d.etab2, P->d.rec, P->d.wpt, P->d.tile_off, P->d.tile_home,
                    P->d.tile_order, P->d.tile_skew, P->d.interp_items, P->d.spread_items, P->d.win,
                    P->d.bufA, P->d.bufB,
                    P->d.stage_in, P->d.stage_out};
    for (void* q : ptrs) xfree(q);
    if (P->d.h_err) xfree_host(P->d.h_err);
    else xfree(P->d.err);
    delete P;
}

namespace {

template <typename T> cudaError_t dalloc(nuasm_plan_s* P, T** out, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = xmalloc(&q, bytes);
    if (e == cudaSuccess) {
        *out = static_cast<T*>(q);
        P->device_bytes += int64_t(bytes);
    }
    return e;
}

// Upload the host tables in the plan's precision.
cudaError_t upload_tables(nuasm_plan_s* P, const HostTables& t, cudaStream_t st) {
    const int np = P->g.np;
    const size_t eb = elt_bytes(P);
    const size_t sb = P->f64 ? sizeof(double) : sizeof(float2);
    const size_t bytes = table_bytes(P->g, P->f64, true);
    const size_t tw_off = 6 * np * eb + np * sb;
    // F64 plans append the twiddles as float pairs (hi = the value rounded to
    // float, lo = the remainder rounded) for the double-float row passes
    const size_t df_bytes = P->f64 ? bytes - tw_off : 0;
    char* base = nullptr;
    cudaError_t e = dalloc(P, &base, bytes + df_bytes);
    if (e != cudaSuccess) return e;
    P->d.tables = base;
    P->d.t1x = base;
    P->d.t1y = base + np * eb;
    P->d.t2x = base + 2 * np * eb;
    P->d.t2y = base + 3 * np * eb;
    P->d.t3x = base + 4 * np * eb;
    P->d.t3y = base + 5 * np * eb;
    P->d.s = base + 6 * np * eb;
    P->d.tw = base + tw_off;
    P->d.tw_df = P->f64 ? base + bytes : nullptr;
    std::vector<char> host(bytes + df_bytes);
    pack_tables(t, P->g, P->f64, true, host.data());
    if (P->f64) {
        const double* tw = reinterpret_cast<const double*>(host.data() + tw_off);
        float* out = reinterpret_cast<float*>(host.data() + bytes);
        for (size_t i = 0; i < df_bytes / sizeof(double); ++i) {
            const float hi = float(tw[i]);
            out[2 * i] = hi;
            out[2 * i + 1] = float(tw[i] - double(hi));
        }
    }
    e = cudaMemcpyAsync(base, host.data(), bytes + df_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);   // host buffer goes out of scope
}

// Copy a host coordinate array to a temporary device buffer when needed.
cudaError_t device_copy(const double* src, int64_t m, double** dev_out, bool* owned, cudaStream_t st) {
    *owned = false;
    *dev_out = const_cast<double*>(src);
    if (!src || m == 0 || device_accessible(src)) return cudaSuccess;
    void* q = nullptr;
    cudaError_t e = xmalloc(&q, sizeof(double) * size_t(m));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(q, src, sizeof(double) * size_t(m), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { xfree(q); return e; }
    *dev_out = static_cast<double*>(q);
    *owned = true;
    return cudaSuccess;
}

// Bit 2 of a plan's host-mapped error word: a bounded device wait of an
// earlier execute gave up.  Reading it needs no synchronisation (the device
// writes the mapped word directly); it is reported once and cleared.
bool take_timeout(nuasm_plan_s* P) {
    if (!P->d.h_err) return false;
    volatile int* w = P->d.h_err;
    if (!(*w & 2)) return false;
    __atomic_fetch_and(P->d.h_err, ~2, __ATOMIC_SEQ_CST);
    return true;
}

nuasm_status check_plan_usable(nuasm_plan_s* P) {
    if (!P) return NUASM_EINVAL;
    // surface sticky asynchronous faults of earlier launches
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NUASM_ECUDA;
    }
    if (take_timeout(P)) return NUASM_ETIMEOUT;
    return NUASM_OK;
}

}  // namespace

// ---------------------------------------------------------------- device-pointer chains
// (per-stage event scopes are no-ops unless the plan's profiling is on)
cudaError_t nuasm::chain_type1(nuasm_plan_s* P, const void* c, void* u2, cudaStream_t st) {
    cudaError_t e;
    { StageScope sc(P, NUASM_STAGE_SPREAD, st); if ((e = launch_spread(P, c, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_COL_FWD_FOLD, st); if ((e = launch_col_fwd_fold(P, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_ROW_T1, st); if ((e = launch_row_t1(P, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_COL_INV, st); if ((e = launch_col_inv(P, u2, st)) != cudaSuccess) return e; }
    return cudaSuccess;
}

cudaError_t nuasm::chain_type2(nuasm_plan_s* P, const void* u1, void* v, cudaStream_t st) {
    cudaError_t e;
    { StageScope sc(P, NUASM_STAGE_COL_FWD, st); if ((e = launch_col_fwd(P, u1, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_ROW_T2, st); if ((e = launch_row_t2(P, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_COL_INV_FOLD, st); if ((e = launch_col_inv_fold(P, st)) != cudaSuccess) return e; }
    if (P->m > 0) {
        StageScope sc(P, NUASM_STAGE_INTERP, st);
        if ((e = launch_interp(P, v, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// type 3: spread the source plan's points, fused forward/H/inverse row pass,
// interpolate at the destination plan's points (same geometry, the source
// plan's workspace)
cudaError_t nuasm::chain_type3(nuasm_plan_s* P, const nuasm_plan_s* Q, const void* c, void* v, cudaStream_t st) {
    cudaError_t e;
    { StageScope sc(P, NUASM_STAGE_SPREAD, st); if ((e = launch_spread(P, c, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_COL_FWD_FOLD, st); if ((e = launch_col_fwd_fold(P, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_ROW_T3, st); if ((e = launch_row_t3(P, st)) != cudaSuccess) return e; }
    { StageScope sc(P, NUASM_STAGE_COL_INV_FOLD, st); if ((e = launch_col_inv_fold(P, st)) != cudaSuccess) return e; }
    if (Q->m > 0) {
        nuasm_plan_s view = *Q;          // destination records over the source plan's window
        view.d.win = P->d.win;
        view.prof = false;
        StageScope sc(P, NUASM_STAGE_INTERP, st);
        if ((e = launch_interp(&view, v, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

// ---------------------------------------------------------------- execute chains
nuasm_status exec_type1(nuasm_plan_s* P, const void* c, void* u2, cudaStream_t st) {
    nuasm_status s0 = check_plan_usable(P);
    if (s0 != NUASM_OK) return s0;
    if (!u2 || (P->m > 0 && !c)) return NUASM_EINVAL;
    const size_t eb = elt_bytes(P);
    const void* cin = c;
    if (P->m > 0 && !device_accessible(c)) {
        StageScope sc(P, NUASM_STAGE_H2D, st);
        NUASM_TRY(cudaMemcpyAsync(P->d.stage_in, c, eb * size_t(P->m), cudaMemcpyHostToDevice, st));
        cin = P->d.stage_in;
    }
    const bool out_dev = device_accessible(u2);
    void* uo = out_dev ? u2 : P->d.stage_out;
    NUASM_TRY(chain_type1(P, cin, uo, st));
    if (!out_dev) {
        StageScope sc(P, NUASM_STAGE_D2H, st);
        NUASM_TRY(cudaMemcpyAsync(u2, P->d.stage_out, eb * size_t(P->g.n) * P->g.n, cudaMemcpyDeviceToHost, st));
    }
    return NUASM_OK;
}

nuasm_status exec_type2(nuasm_plan_s* P, const void* u1, void* v, cudaStream_t st) {
    nuasm_status s0 = check_plan_usable(P);
    if (s0 != NUASM_OK) return s0;
    if (!u1 || (P->m > 0 && !v)) return NUASM_EINVAL;
    const size_t eb = elt_bytes(P);
    const void* uin = u1;
    if (!device_accessible(u1)) {
        StageScope sc(P, NUASM_STAGE_H2D, st);
        NUASM_TRY(cudaMemcpyAsync(P->d.stage_in, u1, eb * size_t(P->g.n) * P->g.n, cudaMemcpyHostToDevice, st));
        uin = P->d.stage_in;
    }
    const bool out_dev = P->m == 0 || device_accessible(v);
    void* vo = out_dev ? v : P->d.stage_out;
    NUASM_TRY(chain_type2(P, uin, vo, st));
    if (!out_dev) {
        StageScope sc(P, NUASM_STAGE_D2H, st);
        NUASM_TRY(cudaMemcpyAsync(v, P->d.stage_out, eb * size_t(P->m), cudaMemcpyDeviceToHost, st));
    }
    return NUASM_OK;
}

nuasm_status exec_type3(nuasm_plan_s* P, nuasm_plan_s* Q, const void* c, void* v, cudaStream_t st) {
    nuasm_status s0 = check_plan_usable(P);
    if (s0 != NUASM_OK) return s0;
    if (!Q || !same_problem(P->p, Q->p)) return NUASM_EINVAL;
    if ((P->m > 0 && !c) || (Q->m > 0 && !v)) return NUASM_EINVAL;
    const size_t eb = elt_bytes(P);
    const void* cin = c;
    if (P->m > 0 && !device_accessible(c)) {
        StageScope sc(P, NUASM_STAGE_H2D, st);
        NUASM_TRY(cudaMemcpyAsync(P->d.stage_in, c, eb * size_t(P->m), cudaMemcpyHostToDevice, st));
        cin = P->d.stage_in;
    }
    const bool out_dev = Q->m == 0 || device_accessible(v);
    void* vo = out_dev ? v : Q->d.stage_out;
    NUASM_TRY(chain_type3(P, Q, cin, vo, st));
    if (!out_dev) {
        StageScope sc(P, NUASM_STAGE_D2H, st);
        NUASM_TRY(cudaMemcpyAsync(v, Q->d.stage_out, eb * size_t(Q->m), cudaMemcpyDeviceToHost, st));
    }
    return NUASM_OK;
}

}  // namespace

extern "C" {

nuasm_status nuasm_plan(nuasm_plan_t* out, const nuasm_params_t* p, int64_t m, const double* x,
                        const double* y, const double* w, void* stream) {
    if (!out) return NUASM_EINVAL;
    *out = nullptr;
    return plan_create(out, p, m, x, y, w, static_cast<cudaStream_t>(stream), true);
}

}  // extern "C"

nuasm_status nuasm::plan_create(nuasm_plan_s** out, const nuasm_params_t* p, int64_t m, const double* x,
                                const double* y, const double* w, cudaStream_t st, bool workspace,
                                const LatticeSpec* lat) {
    *out = nullptr;
    if (!p) return NUASM_EINVAL;
    nuasm_params_t rp;
    nuasm_status s = validate(*p, m, &rp);
    if (s != NUASM_OK) return s;
    if (m > 0 && !lat && (!x || !y)) return NUASM_EINVAL;

    nuasm_plan_s* P = new (std::nothrow) nuasm_plan_s();
    if (!P) return NUASM_ENOMEM;
    PlanExtra* X = new (std::nothrow) PlanExtra();
    if (!X) { delete P; return NUASM_ENOMEM; }
    P->prof_state = X;
    P->p = rp;
    P->g = make_geometry(rp);
    P->m = m;
    P->f64 = rp.prec == NUASM_PREC_F64;
    P->has_w = w != nullptr;

    auto bail = [&](nuasm_status code) { plan_release(P); return code; };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return bail(NUASM_ECUDA); }

    HostTables ht{};
    build_tables(rp, P->g, &ht);
    P->rc = ht.rc;
    P->poly = ht.poly;
    if (P->f64) {
        fit_kernel_poly64(P->g, &P->poly64);
        split_kernel_poly64(P->poly64, &P->poly64df);
    }
    P->nonsep_mode = choose_nonsep_mode(rp, ht.rmax);
    cudaError_t e = upload_tables(P, ht, st);
    free_tables(&ht);
    if (e != cudaSuccess) return bail(cuda_status(e));

    const Geometry& g = P->g;
    const size_t eb = elt_bytes(P);
    if (workspace) {
        const size_t stage = std::max<size_t>(size_t(m), size_t(g.n) * g.n) * eb;
        if ((e = dalloc(P, &P->d.win, ws_win_elems(g) * eb)) != cudaSuccess) return bail(cuda_status(e));
        if ((e = dalloc(P, &P->d.bufA, ws_bufA_elems(g) * eb)) != cudaSuccess) return bail(cuda_status(e));
        if ((e = dalloc(P, &P->d.bufB, ws_bufB_elems(g) * eb)) != cudaSuccess) return bail(cuda_status(e));
        if ((e = dalloc(P, &P->d.stage_in, stage)) != cudaSuccess) return bail(cuda_status(e));
        if ((e = dalloc(P, &P->d.stage_out, stage)) != cudaSuccess) return bail(cuda_status(e));
        if (P->nonsep_mode != 0) {
            // the plan's transfer function is fixed: tabulate its non-separable factor once
            const size_t ne = etab_elems(g, &P->etab_pitch);
            if ((e = dalloc(P, &P->d.etab, ne * eb)) != cudaSuccess) return bail(cuda_status(e));
            if ((e = build_etab(P, st)) != cudaSuccess) return bail(cuda_status(e));
            if (NUASM_ETAB2 && !P->f64 && g.np <= 4096) {
                // type 2's row pass stages T2x E rows (merged row engines: N' <= 4096 in FP32)
                const size_t n2 = size_t(g.np / 2 + 1) * g.np;
                if ((e = dalloc(P, &P->d.etab2, n2 * eb)) != cudaSuccess) return bail(cuda_status(e));
                if ((e = build_etab2(P, st)) != cudaSuccess) return bail(cuda_status(e));
            }
        }
    }
    if ((e = dalloc(P, &P->d.tile_off, sizeof(int) * (g.ntiles + 1))) != cudaSuccess) return bail(cuda_status(e));
    if ((e = dalloc(P, &P->d.tile_home, sizeof(int) * g.ntiles)) != cudaSuccess) return bail(cuda_status(e));
    {
        // the error word is host-mapped: execute calls read it without synchronising
        void* h = nullptr;
        if ((e = xmalloc_host(&h, sizeof(int), cudaHostAllocMapped)) != cudaSuccess) return bail(cuda_status(e));
        P->d.h_err = static_cast<int*>(h);
        *P->d.h_err = 0;
        void* dp = nullptr;
        if ((e = cudaHostGetDevicePointer(&dp, h, 0)) != cudaSuccess) return bail(cuda_status(e));
        P->d.err = static_cast<int*>(dp);
        P->device_bytes += int64_t(sizeof(int));
    }

    if (lat) {
        s = run_binning_lattice(P, *lat, st);
        cudaStreamSynchronize(st);
        if (s != NUASM_OK) return bail(s);
        *out = P;
        return NUASM_OK;
    }
    double *dx = nullptr, *dy = nullptr, *dw = nullptr;
    bool ox = false, oy = false, ow = false;
    auto free_coords = [&]() {
        if (ox) xfree(dx);
        if (oy) xfree(dy);
        if (ow) xfree(dw);
    };
    if ((e = device_copy(x, m, &dx, &ox, st)) != cudaSuccess ||
        (e = device_copy(y, m, &dy, &oy, st)) != cudaSuccess ||
        (e = device_copy(w, m, &dw, &ow, st)) != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_coords();
        return bail(cuda_status(e));
    }
    s = run_binning(P, dx, dy, dw, st);
    cudaStreamSynchronize(st);
    free_coords();
    if (s != NUASM_OK) return bail(s);
    *out = P;
    return NUASM_OK;
}

namespace {

// one plan on the points with parameters q and the mean of three timed solves
// of `type` after an untimed one (CUDA events on st)
nuasm_status time_solve(const nuasm_params_t& q, int64_t m, const double* x, const double* y, int type,
                        cudaStream_t st, void* in, void* out, cudaEvent_t t0, cudaEvent_t t1, double* ms) {
    nuasm_plan_s* P = nullptr;
    const nuasm_status s = plan_create(&P, &q, m, x, y, nullptr, st, true);
    if (s != NUASM_OK) return s;
    cudaError_t e = cudaSuccess;
    float total = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first run untimed
        e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) e = type == 1 ? chain_type1(P, in, out, st) : chain_type2(P, in, out, st);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, t0, t1);
        if (rep > 0) total += t;
    }
    plan_release(P);
    if (e != cudaSuccess) return cuda_status(e);
    *ms = double(total) / 3.0;
    return NUASM_OK;
}

// The autotuner: tile sides (those the kernel width allows) and, with
// `chunks`, the interpolation chunk (type 2) or spreading split (type 1);
// the fastest parameters go to *best.
nuasm_status autotune_search(const nuasm_params_t* p, int64_t m, const double* x, const double* y, int type,
                             cudaStream_t st, bool chunks, nuasm_params_t* best, double* best_ms) {
    if (type != 1 && type != 2) return NUASM_EINVAL;
    nuasm_params_t rp;
    nuasm_status s = validate(*p, m, &rp);
    if (s != NUASM_OK) return s;
    if (m > 0 && (!x || !y || !device_accessible(x) || !device_accessible(y))) return NUASM_EINVAL;
    const size_t eb = rp.prec == NUASM_PREC_F64 ? 16 : 8;
    const size_t nn = size_t(rp.n) * rp.n;
    void* buf = nullptr;
    cudaError_t e = xmalloc(&buf, eb * (nn + size_t(m > 0 ? m : 1)));
    if (e != cudaSuccess) return cuda_status(e);
    char* in = static_cast<char*>(buf);
    char* out = in + eb * (type == 1 ? size_t(m) : nn);
    e = cudaMemsetAsync(buf, 0, eb * (nn + size_t(m > 0 ? m : 1)), st);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = xevent_create(&t0, cudaEventDefault);   // timing events
    if (e == cudaSuccess) e = xevent_create(&t1, cudaEventDefault);
    bool found = false;
    double found_ms = 0.0;
    s = NUASM_OK;
    const int type2_chunks[] = {0, 1024, 2048}, type1_chunks[] = {0, -1, 256};
    for (int cand : {16, 32, 64}) {
        if (e != cudaSuccess || s != NUASM_OK) break;
        for (int k = 0; k < (chunks ? 3 : 1); ++k) {
            nuasm_params_t q = *p;
            q.tile = cand;
            if (chunks) {
                if (type == 2) q.interp_chunk = type2_chunks[k];
                else q.spread_chunk = type1_chunks[k];
            }
            double t = 0.0;
            const nuasm_status r = time_solve(q, m, x, y, type, st, in, out, t0, t1, &t);
            if (r == NUASM_EUNSUPPORTED) break;   // a side below the kernel's reach: skip it
            if (r != NUASM_OK) {
                s = r;
                break;
            }
            if (!found || t < found_ms) {
                found = true;
                found_ms = t;
                *best = q;
            }
        }
    }
    if (t0) xevent_destroy(t0);
    if (t1) xevent_destroy(t1);
    cudaStreamSynchronize(st);
    xfree(buf);
    if (e != cudaSuccess) return cuda_status(e);
    if (s != NUASM_OK) return s;
    if (!found) return NUASM_EUNSUPPORTED;
    *best_ms = found_ms;
    return NUASM_OK;
}

}  // namespace

extern "C" {

nuasm_status nuasm_plan_lattice(nuasm_plan_t* out, const nuasm_params_t* p, int32_t nx, int32_t ny,
                                double pitch2, double x0, double y0, void* stream) {
    if (!out) return NUASM_EINVAL;
    *out = nullptr;
    if (!p || nx < 0 || ny < 0 || !std::isfinite(pitch2) || !(pitch2 > 0) || !std::isfinite(x0) ||
        !std::isfinite(y0))
        return NUASM_EINVAL;
    const int64_t m = int64_t(nx) * ny;
    if (m > (int64_t(1) << 29)) return NUASM_EUNSUPPORTED;
    nuasm_params_t rp;
    const nuasm_status s = validate(*p, m, &rp);
    if (s != NUASM_OK) return s;
    if (m == 0) return nuasm_plan(out, p, 0, nullptr, nullptr, nullptr, stream);
    const LatticeSpec lat{nx, ny, pitch2, x0, y0};
    return plan_create(out, p, m, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream), true, &lat);
}

nuasm_status nuasm1_execute(nuasm_plan_t plan, const void* c, void* u2, void* stream) {
    if (!plan) return NUASM_EINVAL;
    if (plan->p.kind != NUASM_KIND_ASM) return NUASM_EINVAL;
    return exec_type1(plan, c, u2, static_cast<cudaStream_t>(stream));
}

nuasm_status nuasm2_execute(nuasm_plan_t plan, const void* u1, void* v, void* stream) {
    if (!plan) return NUASM_EINVAL;
    if (plan->p.kind != NUASM_KIND_ASM) return NUASM_EINVAL;
    return exec_type2(plan, u1, v, static_cast<cudaStream_t>(stream));
}

nuasm_status nufresnel_execute(nuasm_plan_t plan, int32_t type, const void* in, void* out, void* stream) {
    if (!plan) return NUASM_EINVAL;
    if (plan->p.kind != NUASM_KIND_FRESNEL) return NUASM_EINVAL;
    if (type == 1) return exec_type1(plan, in, out, static_cast<cudaStream_t>(stream));
    if (type == 2) return exec_type2(plan, in, out, static_cast<cudaStream_t>(stream));
    return NUASM_EINVAL;
}

nuasm_status nuasm3_execute(nuasm_plan_t src, nuasm_plan_t dst, const void* c, void* v, void* stream) {
    if (!src || !dst) return NUASM_EINVAL;
    if (src->p.kind != NUASM_KIND_ASM) return NUASM_EINVAL;
    return exec_type3(src, dst, c, v, static_cast<cudaStream_t>(stream));
}

nuasm_status nufresnel3_execute(nuasm_plan_t src, nuasm_plan_t dst, const void* c, void* v, void* stream) {
    if (!src || !dst) return NUASM_EINVAL;
    if (src->p.kind != NUASM_KIND_FRESNEL) return NUASM_EINVAL;
    return exec_type3(src, dst, c, v, static_cast<cudaStream_t>(stream));
}

nuasm_status nuasm_autotune_tile(const nuasm_params_t* p, int64_t m, const double* x, const double* y, int32_t type,
                                 void* stream, int32_t* tile, double* ms) {
    if (!p || !tile) return NUASM_EINVAL;
    nuasm_params_t best;
    double t = 0.0;
    const nuasm_status s = autotune_search(p, m, x, y, type, static_cast<cudaStream_t>(stream), false, &best, &t);
    if (s != NUASM_OK) return s;
    *tile = best.tile;
    if (ms) *ms = t;
    return NUASM_OK;
}

nuasm_status nuasm_autotune(const nuasm_params_t* p, int64_t m, const double* x, const double* y, int32_t type,
                            void* stream, nuasm_params_t* best, double* ms) {
    if (!p || !best) return NUASM_EINVAL;
    double t = 0.0;
    const nuasm_status s = autotune_search(p, m, x, y, type, static_cast<cudaStream_t>(stream), true, best, &t);
    if (s == NUASM_OK && ms) *ms = t;
    return s;
}

nuasm_status nuasm_destroy(nuasm_plan_t plan) {
    if (!plan) return NUASM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    const bool timed_out = e == cudaSuccess && take_timeout(plan);
    plan_release(plan);
    if (timed_out) return NUASM_ETIMEOUT;
    return cuda_status(e);
}

const char* nuasm_strerror(nuasm_status s) {
    switch (s) {
        case NUASM_OK: return "success";
        case NUASM_EINVAL: return "invalid argument";
        case NUASM_ERANGE: return "point outside the window [-N pitch/2, N pitch/2)";
        case NUASM_ENOMEM: return "out of memory";
        case NUASM_ECUDA: return "CUDA error";
        case NUASM_ETIMEOUT: return "bounded device wait timed out";
        case NUASM_EUNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

nuasm_status nuasm_plan_info(nuasm_plan_t plan, nuasm_plan_info_t* info) {
    if (!plan || !info) return NUASM_EINVAL;
    const Geometry& g = plan->g;
    std::memset(info, 0, sizeof(*info));
    info->n = g.n;
    info->n_pad = g.np;
    info->grid = g.G;
    info->window = g.W;
    info->window_origin = g.Lo;
    info->kernel_width = g.w;
    info->kernel_beta = g.beta;
    info->tile = g.T;
    info->tiles = g.ntiles;
    info->band_lo_x = g.band[0];
    info->band_hi_x = g.band[1];
    info->band_lo_y = g.band[2];
    info->band_hi_y = g.band[3];
    info->points = plan->m;
    info->records = plan->nrec;
    info->device_bytes = plan->device_bytes;
    int pitch = 0;
    info->phase_table_bytes =
        (plan->d.etab ? int64_t(etab_elems(plan->g, &pitch) * (plan->f64 ? 16 : 8)) : 0) +
        (plan->d.etab2 ? int64_t(plan->g.np / 2 + 1) * plan->g.np * 8 : 0);
    info->bank_skew = plan->skew;
    info->spread_split_ctas = plan->d.spread_items ? plan->n_spread_items : 0;
    info->double_float = gridding_double_float(plan) ? 1 : 0;
    return NUASM_OK;
}

nuasm_status nuasm_band(const nuasm_params_t* p, int32_t out[4]) {
    if (!p || !out) return NUASM_EINVAL;
    nuasm_params_t rp;
    nuasm_status s = validate(*p, 0, &rp);
    if (s != NUASM_OK && s != NUASM_EUNSUPPORTED) return s;
    if (s == NUASM_EUNSUPPORTED) {
        rp = *p;
        if (rp.n_pad == 0) rp.n_pad = 2 * rp.n;
    }
    int b[4];
    band_range(rp, b);
    for (int i = 0; i < 4; ++i) out[i] = b[i];
    return NUASM_OK;
}

nuasm_status nuasm_kernel_shape(double tol, int32_t prec, int32_t kernel, int32_t* width, double* beta) {
    if (!width || !beta) return NUASM_EINVAL;
    if (prec != NUASM_PREC_F32_F64PHASE && prec != NUASM_PREC_F64) return NUASM_EINVAL;
    if (kernel != NUASM_KERNEL_ES && kernel != NUASM_KERNEL_GAUSSIAN) return NUASM_EINVAL;
    if (std::isnan(tol) || tol < 0 || tol > 0.1 || (tol > 0 && tol < 1e-15)) return NUASM_EINVAL;
    int w = 0;
    const bool ok = kernel_shape(tol, prec, kernel, &w, beta);
    *width = w;
    return ok ? NUASM_OK : NUASM_EUNSUPPORTED;
}

nuasm_status nuasm_profile_enable(nuasm_plan_t plan, int32_t enable) {
    if (!plan) return NUASM_EINVAL;
    plan->prof = enable != 0;
    return NUASM_OK;
}

nuasm_status nuasm_profile_read(nuasm_plan_t plan, double* ms, int64_t* launches) {
    if (!plan || !ms || !launches) return NUASM_EINVAL;
    PlanExtra* X = extra_of(plan);
    for (int s = 0; s < NUASM_STAGE_COUNT; ++s)
        while (X->ring[s].count > 0) ring_consume_oldest(plan, s);
    for (int s = 0; s < NUASM_STAGE_COUNT; ++s) {
        ms[s] = plan->prof_ms[s];
        launches[s] = plan->prof_n[s];
        plan->prof_ms[s] = 0.0;
        plan->prof_n[s] = 0;
    }
    return NUASM_OK;
}

const char* nuasm_stage_name(int32_t stage) {
    static const char* names[NUASM_STAGE_COUNT] = {"h2d",    "spread",       "col_fwd_fold", "row_t1",
                                                   "col_inv", "col_fwd",      "row_t2",       "col_inv_fold",
                                                   "interp", "d2h",          "row_t3"};
    if (stage < 0 || stage >= NUASM_STAGE_COUNT) return "unknown";
    return names[stage];
}

}  // extern "C"
