// Internal plan representation and launcher prototypes (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nuasm.h"

namespace nuasm {

// Host-side geometry and tables derived from nuasm_params_t.
struct Geometry {
    int n, np, G;          // N, N', G = 2N'
    int logn, lognp;       // log2 N, log2 N'
    int w;                 // kernel width
    double beta;           // kernel shape parameter
    int kernel;            // nuasm_kernel
    int h;                 // window margin ceil(w/2)
    int W, Wp;             // window side, row pitch (elements)
    int Lo;                // window origin on the G grid
    int T, ntx, ntiles;    // tile side, tiles per axis, tile count
    int band[4];           // inclusive kept-mode ranges lo_x, hi_x, lo_y, hi_y
};

// Piecewise-polynomial form of the spreading kernel: tap i of a point with
// fractional offset f in [0, 1) has weight sum_k c[i][k] x^k, x = 2f - 1.
constexpr int kPolyMaxW = 26, kPolyMaxD = 16;   // taps: 16 for the ES kernel, 26 for the Gaussian
struct KernelPoly {
    float c[kPolyMaxW][kPolyMaxD];
    int deg;
};
#ifndef NUASM_POLY64_DEG
#define NUASM_POLY64_DEG 13   // measured: 15 and 14 give the same end-to-end errors, 4% more FP64 time
#endif
constexpr int kPoly64Deg = NUASM_POLY64_DEG;   // degree of the FP64 tap polynomials
static_assert(kPoly64Deg < kPolyMaxD, "FP64 tap degree");
// the same for FP64 gridding, always of degree kPoly64Deg: the fit error
// then sits near the kernel's own edge value (3.6e-14 at degree 15 for w = 13)
// and below the default FP64 tolerance (1e-12)
struct KernelPoly64 {
    double c[kPolyMaxW][kPolyMaxD];
    int deg;
};
// The FP64 coefficients as pairs of floats (x: the coefficient rounded to
// float, y: the rounded remainder), for FP64-mode gridding in double-float
// arithmetic.
struct KernelPolyDF {
    float2 c[kPolyMaxW][kPolyMaxD];
};

// Host tables in FP64 (complex as re/im pairs), natural N'-bin order.
struct HostTables {
    // per-axis separable factors for types 1, 2 and 3, length N' each
    double* t1x; double* t1y; double* t2x; double* t2y; double* t3x; double* t3y;   // 2*N' doubles each
    double* s;        // lambda^2 f_k^2 per bin (ASM), length N'
    double rc;        // z / (2 lambda)  (ASM non-separable phase scale)
    double rmax;      // largest |r| = |rc| q^2 over kept modes (0 when there is no such term)
    double* tw;       // exp(-2 pi i t / G), t in [0, G): 2*G doubles
    KernelPoly poly;  // FP32 Horner coefficients of the kernel taps
};

struct PlanDevice {
    void* tables = nullptr;     // one block holding every table below
    void* t1x = nullptr; void* t1y = nullptr; void* t2x = nullptr; void* t2y = nullptr;
    void* t3x = nullptr; void* t3y = nullptr;
    void* s = nullptr;          // float2 (hi, lo) per bin (F32) or double (F64)
    void* tw = nullptr;         // twiddles, G complex
    void* tw_df = nullptr;      // F64 plans: the twiddles as float pairs (re.hi, re.lo, im.hi, im.lo), for
                                // the double-float row passes
    void* etab = nullptr;       // ASM non-separable factor E(|kx|, |ky|): N'/2 + 1 rows of etab_pitch
                                // entries in the plan precision (null: evaluated per mode)
    void* etab2 = nullptr;      // type 2's T2x(kx) E(|kx|, |ky|): N'/2 + 1 rows of N' entries (FP32 plans
                                // with merged row engines; null: row_t2 uses etab and T2x)
    void* rec = nullptr;        // binned point records
    double* wpt = nullptr;      // optional per-point weights, in point order
    int* tile_off = nullptr;    // ntiles + 1 offsets into rec
    int* tile_home = nullptr;   // home-record count per tile
    int* tile_order = nullptr;  // launch order of the tiles (heaviest first); null = index order
    int8_t* tile_skew = nullptr;    // bank skew of each tile's layouts and record order; null: skew for all
    int4* interp_items = nullptr;   // interpolation work items (tile, first record, end record, 0),
                                    // heaviest first; null = one item per tile in tile_order
    int4* spread_items = nullptr;   // spreading work items (tile, first record, end record, chunked),
                                    // heaviest first, where a tile's records are split over CTAs;
                                    // null = one CTA per tile in tile_order
    void* win = nullptr;        // W x Wp fine-grid window
    void* bufA = nullptr;       // N' x Wp
    void* bufB = nullptr;       // N' x N
    void* stage_in = nullptr;   // host-pointer staging (max of M, N^2 complex)
    void* stage_out = nullptr;
    int* err = nullptr;         // device address of the error word
    int* h_err = nullptr;       // host view of the error word when it is host-mapped (plans made by
                                // plan_create); null when it lives in device memory (views, scratch)
};

}  // namespace nuasm

struct nuasm_plan_s {
    nuasm_params_t p;
    nuasm::Geometry g;
    int64_t m = 0;
    int64_t nrec = 0;
    bool has_w = false;
    bool f64 = false;
    double rc = 0.0;            // z / (2 lambda)
    int nonsep_mode = 0;        // ASM non-separable phase: 0 none, 1 plain, 2 double-float
    int etab_pitch = 0;         // entries per row of d.etab
    int skew = 0;               // bank skew of the gridding tile layouts and record order: the one most
                                // tiles use when d.tile_skew is set, else the one every tile uses
    int n_interp_items = 0;     // entries of d.interp_items
    int n_spread_items = 0;     // entries of d.spread_items
    nuasm::KernelPoly poly{};   // kernel taps as polynomials (F32 gridding)
    nuasm::KernelPoly64 poly64{};   // the same in FP64 (F64 gridding)
    nuasm::KernelPolyDF poly64df{};   // poly64 as float pairs (F64 gridding in double-float arithmetic)
    int64_t device_bytes = 0;
    nuasm::PlanDevice d;
    // profiling
    bool prof = false;
    void* prof_state = nullptr;   // per-stage CUDA event rings (capi.cu)
    double prof_ms[NUASM_STAGE_COUNT] = {};
    int64_t prof_n[NUASM_STAGE_COUNT] = {};
};

namespace nuasm {

// FP64 gridding in double-float arithmetic on the FP32 pipe (gridding.cu):
// FP64 plans at the kernel widths of the FP64 tolerances 1e-12 and 1e-10
// (ES: w = 13 and 11; Gaussian: w = 25 and 21, and 15 for 1e-7).
#ifndef NUASM_F64_DF
#define NUASM_F64_DF 1   // 0: FP64 gridding on the FP64 pipe throughout
#endif
inline bool gridding_double_float(const nuasm_plan_s* P) {
    if (!NUASM_F64_DF || !P->f64) return false;
    if (P->g.kernel == NUASM_KERNEL_ES) return P->g.w == 11 || P->g.w == 13;
    return P->g.w == 15 || P->g.w == 21 || P->g.w == 25;
}

// Gauss-Legendre quadrature of the kernel on [0, w/2] for its Fourier transform.
struct KernelQuad {
    static constexpr int kMax = 2 * kPolyMaxW + 48;
    int n;
    double t[kMax], f[kMax];   // nodes and weight x kernel value
};

// host math (hostmath.cpp); the per-mode helpers allocate nothing
void make_quad(const Geometry& g, KernelQuad* qd);
double phihat_at(const KernelQuad& qd, double nu);
void asm_axis_factor(const nuasm_params_t& p, int np, int k, int axis, double* re, double* im);
void table_entry(const nuasm_params_t& p, const Geometry& g, int q, int type, double phihat, double hs_re,
                 double hs_im, double* re, double* im);
void constant_factor(const nuasm_params_t& p, double* re, double* im);
void twiddle(int i, int G, double* re, double* im);
double nonsep_rmax(const nuasm_params_t& p, const Geometry& g);
void fit_kernel_poly(const Geometry& g, KernelPoly* kp);
void fit_kernel_poly64(const Geometry& g, KernelPoly64* kp);
void split_kernel_poly64(const KernelPoly64& kp, KernelPolyDF* out);
nuasm_status validate(const nuasm_params_t& p, int64_t m, nuasm_params_t* resolved);
bool kernel_shape(double tol, int prec, int kernel, int* w, double* beta);
double kernel_value(const Geometry& g, double t);
void band_range(const nuasm_params_t& p, int out[4]);
Geometry make_geometry(const nuasm_params_t& p);
// FP64 tables for the plan parameters; `phihat` (N' values of the kernel's
// Fourier transform at k/G, see phihat_table) may be passed in when cached,
// twiddles are left out (t->tw = nullptr) when with_twiddles is false.
void build_tables(const nuasm_params_t& p, const Geometry& g, HostTables* t, const double* phihat = nullptr,
                  bool with_twiddles = true);
void phihat_table(const Geometry& g, double* out);
void free_tables(HostTables* t);
size_t table_bytes(const Geometry& g, bool f64, bool with_twiddles);
void pack_tables(const HostTables& t, const Geometry& g, bool f64, bool with_twiddles, void* dst);

// Pass twiddles.  The full twiddle table tw[t] = exp(-2 pi i t / 2N'),
// t < 2N', is followed by the twiddle bases of every pass I >= 1 of the
// radix-8 and then the radix-16 Stockham schedule of an N'-point transform
// (fft_engine.cuh): for each butterfly group k < NS = 2^(I log2 E), the
// twp_per_k entries a butterfly of radix R = 2^lr loads, contiguous
// (FP64: w^k .. w^((R-1)k); FP32: w^k and w^4k, w^k and w^2k for R = 4, w^k
// for R = 2; w = exp(-2 pi i / (NS R))).  One group's entries are one load.
constexpr int twp_per_k(bool f64, int lr) { return (f64 || lr == 1) ? (1 << lr) - 1 : 2; }
constexpr int twp_sched_entries(bool f64, int le, int logl) {
    const int nfull = logl / le, rem = logl % le, npass = nfull + (rem ? 1 : 0);
    int n = 0;
    for (int i = 1; i < npass; ++i) n += (1 << (i * le)) * twp_per_k(f64, i < nfull ? le : rem);
    return n;
}
// entries before pass `pass` of the radix-2^le schedule (le = 3 or 4)
constexpr int twp_pass_offset(bool f64, int le, int logl, int pass) {
    const int nfull = logl / le, rem = logl % le;
    int off = le == 4 ? twp_sched_entries(f64, 3, logl) : 0;
    for (int i = 1; i < pass; ++i) off += (1 << (i * le)) * twp_per_k(f64, i < nfull ? le : rem);
    return off;
}
constexpr int twp_entries(bool f64, int logl) {
    return twp_sched_entries(f64, 3, logl) + twp_sched_entries(f64, 4, logl);
}
// Gather the pass twiddles (twp_entries complex values in the plan precision)
// from the full table `tw` (2^(logl+1) complex doubles, interleaved).
void pack_twp(const double* tw, int logl, bool f64, void* dst);
// ASM non-separable phase evaluation: 0 none, 1 plain, 2 double-float
int choose_nonsep_mode(const nuasm_params_t& p, double rmax);

// plan life cycle and device-pointer execute chains (capi.cu).  A plan made
// without workspace holds tables, twiddles and bins only; it is executed
// through a view that supplies the workspace (batch.cu, serve.cu).
// The points of a lattice plan: x0 + i pitch2, y0 + j pitch2, point j nx + i.
struct LatticeSpec {
    int nx, ny;
    double pitch2, x0, y0;
};
// x, y, w: the points' coordinates and weights; or, with `lat`, no coordinates
// (x, y, w null) and the lattice binned without a sort (run_binning_lattice)
nuasm_status plan_create(nuasm_plan_s** out, const nuasm_params_t* p, int64_t m, const double* x,
                         const double* y, const double* w, cudaStream_t st, bool workspace,
                         const LatticeSpec* lat = nullptr);
void plan_release(nuasm_plan_s* P);
bool same_problem(const nuasm_params_t& a, const nuasm_params_t& b);
bool device_accessible(const void* p);
cudaError_t chain_type1(nuasm_plan_s* P, const void* c, void* u2, cudaStream_t s);
cudaError_t chain_type2(nuasm_plan_s* P, const void* u1, void* v, cudaStream_t s);
cudaError_t chain_type3(nuasm_plan_s* P, const nuasm_plan_s* Q, const void* c, void* v, cudaStream_t s);
// workspace elements (complex) of a geometry: window W x Wp, bufA N' x Wp, bufB N' x N
inline size_t ws_win_elems(const Geometry& g) { return size_t(g.W) * g.Wp; }
inline size_t ws_bufA_elems(const Geometry& g) { return size_t(g.np) * g.Wp; }
inline size_t ws_bufB_elems(const Geometry& g) { return size_t(g.np) * g.n; }

// Resource acquisition (resources.cu): device, pool and pinned host
// allocations, streams, events and graph instantiations, with a count of the
// live ones and a test hook that fails the k-th acquisition
// (nuasm_debug_fail_alloc).  A failed acquisition returns
// cudaErrorMemoryAllocation and leaves the output null.
cudaError_t xmalloc(void** p, size_t bytes);
cudaError_t xmalloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t xmalloc_pool(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s);
cudaError_t xmalloc_host(void** p, size_t bytes, unsigned flags);
void xfree(void* p);
void xfree_async(void* p, cudaStream_t s);
void xfree_host(void* p);
cudaError_t xstream_create(cudaStream_t* s);
void xstream_destroy(cudaStream_t s);
cudaError_t xevent_create(cudaEvent_t* ev, unsigned flags = cudaEventDisableTiming);
void xevent_destroy(cudaEvent_t ev);
cudaError_t xgraph_instantiate(cudaGraphExec_t* exec, cudaGraph_t graph);
void xgraph_exec_destroy(cudaGraphExec_t exec);
cudaError_t xpool_create(cudaMemPool_t* pool, const cudaMemPoolProps* props);
cudaError_t xpool_destroy(cudaMemPool_t pool);

// launchers (gridding.cu / passes.cu); all asynchronous on `s`
// (the device error word P->d.err: bit 1 = point outside the window at plan
// time, bit 2 = a bounded device wait gave up)
nuasm_status run_binning(nuasm_plan_s* P, const double* x, const double* y, const double* w,
                         cudaStream_t s);
nuasm_status run_binning_lattice(nuasm_plan_s* P, const LatticeSpec& lat, cudaStream_t s);
cudaError_t bin_points_into(const nuasm_plan_s* P, const double* x, const double* y, int* cnt, void* rec_tmp,
                            cudaStream_t s);
size_t record_bytes(bool f64);
cudaError_t launch_spread(const nuasm_plan_s* P, const void* c, cudaStream_t s);
cudaError_t launch_interp(const nuasm_plan_s* P, void* v, cudaStream_t s);
cudaError_t launch_col_fwd_fold(const nuasm_plan_s* P, cudaStream_t s);
cudaError_t launch_row_t1(const nuasm_plan_s* P, cudaStream_t s);
cudaError_t launch_col_inv(const nuasm_plan_s* P, void* u2, cudaStream_t s);
cudaError_t launch_col_fwd(const nuasm_plan_s* P, const void* u1, cudaStream_t s);
cudaError_t launch_row_t2(const nuasm_plan_s* P, cudaStream_t s);
cudaError_t launch_row_t3(const nuasm_plan_s* P, cudaStream_t s);
// Fill P->d.etab (etab_elems entries, pitch P->etab_pitch) with the ASM non-separable factor.
size_t etab_elems(const Geometry& g, int* pitch);
cudaError_t build_etab(const nuasm_plan_s* P, cudaStream_t s);
// Fill P->d.etab2 ((N'/2 + 1) x N' entries) from d.etab and the type-2 Tx table.
cudaError_t build_etab2(const nuasm_plan_s* P, cudaStream_t s);
cudaError_t launch_col_inv_fold(const nuasm_plan_s* P, cudaStream_t s);

}  // namespace nuasm
