// nuasm2_solve_noalloc: a one-shot NU-ASM_2 solve that allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc or any allocating
// routine -- plug-ins whose host framework owns every byte of device memory
// through its own pool, and real-time loops that cannot afford an
// allocation's latency or its failure.  Such callers cannot build a plan with
// nuasm_plan (which allocates its tables, bins and workspace), so this entry
// point does the plan work and the solve in one call, with every intermediate
// in one file-scope device array.  The call copies its tables from host
// memory, reads the error word back and waits for its stream before it
// returns.
//
// The array (kScratchBytes) is part of the library image: every GPU that loads
// the library holds it until the process exits.  Its device address is looked
// up once per device with cudaGetSymbolAddress, with that device current, on
// the first call made on the device; make that first call before any stream
// capture begins.  All calls share the array and it keeps the last call's
// contents: counters and the error word are cleared at the start of every
// call, everything else is fully overwritten before it is read.  Calls whose
// work overlaps on the GPU (different streams, or another host thread) race
// on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "nuasm_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxN = 256;                           // N <= 256, so N' <= 512
constexpr int64_t kMaxPoints = 65536;
constexpr int kMaxDevices = 64;
constexpr int kMaxNp = 2 * kMaxN;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device).
cudaError_t scratch_on(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

nuasm_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

// bump carving of the scratch array, 256-byte aligned pieces
struct Carve {
    unsigned char* base;
    size_t used = 0;
    void* take(size_t bytes) {
        used = (used + 255) & ~size_t(255);
        void* p = base + used;
        used += bytes;
        return p;
    }
};

}  // namespace

extern "C" nuasm_status nuasm2_solve_noalloc(const nuasm_params_t* p, int64_t m, const double* x, const double* y,
                                             const void* u1, void* v, void* stream) {
    using namespace nuasm;
    if (!p) return NUASM_EINVAL;
    nuasm_params_t rp;
    nuasm_status s = validate(*p, m, &rp);
    if (s != NUASM_OK) return s;
    if (rp.kind != NUASM_KIND_ASM || rp.prec != NUASM_PREC_F32_F64PHASE) return NUASM_EINVAL;
    if (rp.n > kMaxN || rp.n_pad > kMaxNp || m > kMaxPoints) return NUASM_EUNSUPPORTED;
    if (!u1 || (m > 0 && (!x || !y || !v))) return NUASM_EINVAL;
    if (!on_device(u1) || (m > 0 && (!on_device(x) || !on_device(y) || !on_device(v)))) return NUASM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return NUASM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return NUASM_EUNSUPPORTED;
    unsigned char* base = nullptr;
    cudaError_t e = scratch_on(dev, &base);
    if (e != cudaSuccess) return status_of(e);

    // a plan record on the stack whose device pointers all point into the scratch array
    nuasm_plan_s P;
    P.p = rp;
    P.g = make_geometry(rp);
    P.m = m;
    P.f64 = false;
    const Geometry& g = P.g;
    const int np = g.np;
    Carve cv{base};
    int logl = 0;
    while ((1 << logl) < np) ++logl;
    const size_t ntw = size_t(g.G) + size_t(twp_entries(false, logl));   // full table, then pass twiddles
    float2* tables = static_cast<float2*>(cv.take(sizeof(float2) * (4 * size_t(np) + np + ntw)));
    P.d.t1x = tables;
    P.d.t1y = tables + np;
    P.d.t2x = tables + 2 * np;
    P.d.t2y = tables + 3 * np;
    P.d.s = tables + 4 * np;
    P.d.tw = tables + 5 * np;
    int* cnt = static_cast<int*>(cv.take(sizeof(int) * 4 * size_t(g.ntiles)));
    P.d.tile_off = static_cast<int*>(cv.take(sizeof(int) * (size_t(g.ntiles) + 1)));
    P.d.tile_home = static_cast<int*>(cv.take(sizeof(int) * size_t(g.ntiles)));
    P.d.err = static_cast<int*>(cv.take(sizeof(int)));
    const size_t recb = record_bytes(false) * 4 * size_t(m > 0 ? m : 1);
    P.d.rec = cv.take(recb);
    void* rec_tmp = cv.take(recb);
    P.d.bufB = cv.take(sizeof(float2) * size_t(np) * g.n);
    P.d.bufA = cv.take(sizeof(float2) * size_t(np) * g.Wp);
    P.d.win = cv.take(sizeof(float2) * size_t(g.W) * g.Wp);
    if (cv.used > kScratchBytes) return NUASM_EUNSUPPORTED;

    // type-2 tables (Eq. 4 separable part, deconvolution, twiddles), built on the stack
    constexpr int kMaxLog = 9;   // log2(kMaxNp)
    static_assert((1 << kMaxLog) == kMaxNp, "kMaxLog");
    float2 host[4 * kMaxNp + kMaxNp + 2 * kMaxNp + twp_entries(false, kMaxLog)];
    double twd[2 * 2 * kMaxNp];
    std::memset(host, 0, sizeof(host));
    KernelQuad qd;
    make_quad(g, &qd);
    double cre, cim;
    constant_factor(rp, &cre, &cim);
    for (int q = 0; q < np; ++q) {
        const int k = q < np / 2 ? q : q - np;
        const double ph = phihat_at(qd, double(k) / g.G);
        double hxr, hxi, hyr, hyi, re, im;
        asm_axis_factor(rp, np, k, 0, &hxr, &hxi);
        asm_axis_factor(rp, np, k, 1, &hyr, &hyi);
        table_entry(rp, g, q, 2, ph, hxr, hxi, &re, &im);
        host[2 * np + q] = make_float2(float(re), float(im));
        table_entry(rp, g, q, 2, ph, hyr * cre - hyi * cim, hyr * cim + hyi * cre, &re, &im);
        host[3 * np + q] = make_float2(float(re), float(im));
        const double f = double(k) / (double(np) * rp.pitch);
        const double sv = rp.lambda * rp.lambda * f * f;
        const float hi = float(sv);
        host[4 * np + q] = make_float2(hi, float(sv - double(hi)));
    }
    for (int i = 0; i < g.G; ++i) {
        twiddle(i, g.G, &twd[2 * i], &twd[2 * i + 1]);
        host[5 * np + i] = make_float2(float(twd[2 * i]), float(twd[2 * i + 1]));
    }
    pack_twp(twd, logl, false, host + 5 * np + g.G);
    P.rc = rp.z / (2.0 * rp.lambda);
    const double rmax = nonsep_rmax(rp, g);
    P.nonsep_mode = choose_nonsep_mode(rp, rmax);
    fit_kernel_poly(g, &P.poly);
    // pageable source: the copy is staged before the call returns, so the stack buffer may go
    e = cudaMemcpyAsync(tables, host, sizeof(float2) * (5 * size_t(np) + ntw), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return status_of(e);

    if ((e = bin_points_into(&P, x, y, cnt, rec_tmp, st)) != cudaSuccess) return status_of(e);
    if ((e = launch_col_fwd(&P, u1, st)) != cudaSuccess) return status_of(e);
    if ((e = launch_row_t2(&P, st)) != cudaSuccess) return status_of(e);
    if ((e = launch_col_inv_fold(&P, st)) != cudaSuccess) return status_of(e);
    if (m > 0 && (e = launch_interp(&P, v, st)) != cudaSuccess) return status_of(e);

    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, P.d.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return status_of(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return status_of(e);
    if (flag & 2) return NUASM_ETIMEOUT;   // a bounded wait of a column pass gave up
    return flag ? NUASM_ERANGE : NUASM_OK;
}
