/*
 * nuasm.h -- C ABI of the GB300 non-uniform sampled diffraction library.
 *
 * Computes the non-uniform sampled angular spectrum method (NU-ASM) and its
 * Fresnel counterpart (NU-FRE) of Shimobaba et al., arXiv:1308.6644:
 *
 *   type 1 (NU-ASM_1, Eq. 6): non-uniform source samples -> uniform N x N plane
 *       u2(m) = (1/N'^2) sum_k F(k) H(k) exp(2 pi i k.m / N'),
 *       F(k)  = sum_j w_j c_j exp(-2 pi i f_k . x_j)           (NUFFT type 1, Eq. 7)
 *   type 2 (NU-ASM_2, Eq. 9): uniform N x N source -> non-uniform points
 *       v_j   = (1/N'^2) sum_k G(k) H(k) exp(2 pi i f_k . x_j)  (NUFFT type 2, Eq. 8)
 *       G(k)  = sum_m u1(m) exp(-2 pi i k.m / N')
 *
 * with N' = 2N (zero padding, Eq. 3 discussion), f_k = k / (N' pitch),
 * k in [-N'/2, N'/2)^2, m in [-N/2, N/2)^2, and H either the band-limited,
 * off-axis shifted ASM transfer function of Eq. 4 or the Fresnel transfer
 * function of Eq. 5 (the DFT of the sampled impulse response
 * exp(ikz)/(i lambda z) exp(i pi |m pitch + o|^2/(lambda z)), area element
 * pitch^2).
 *
 * Conventions shared by every call:
 *  - Coordinates are metres relative to the centre of the uniform plane; a
 *    point is valid iff x/pitch (IEEE division) lies in [-N/2, N/2) on both
 *    axes (the half-open window the paper states for x1 and x2).
 *  - Complex values are interleaved (re, im): float pairs under
 *    NUASM_PREC_F32_F64PHASE, double pairs under NUASM_PREC_F64.
 *  - Uniform planes are row-major [y][x], element (i_y, i_x) holding the
 *    sample at m = (i_x - N/2, i_y - N/2).
 *  - Array arguments of the execute calls may be device memory or host memory
 *    (pinned or pageable); host arrays are staged through plan-owned device
 *    buffers with cudaMemcpyAsync on the given stream.  Pageable host memory
 *    makes the call block the host until its copies are done.  Device arrays
 *    need only the alignment of their element type; 16-byte aligned ones let
 *    the N' >= 4096 column passes read and write them with TMA bulk copies
 *    (others take the same pass with per-thread loads and stores).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Execute calls
 *    are asynchronous on it, never allocate device memory and never
 *    synchronise the device; asynchronous CUDA faults surface as NUASM_ECUDA
 *    from a later call.
 *  - Errors are returned, never thrown or printed.  On any non-OK status no
 *    output has been written unless stated otherwise.
 *  - Device waits are bounded.  When one gives up (a copy that never
 *    arrived), the kernel sets a flag in the plan's host-mapped error word and
 *    that launch's output is incomplete; the plan's next execute call (or
 *    nuasm_batch_execute of a batch holding the plan, or nuasm_destroy)
 *    returns NUASM_ETIMEOUT without doing any work and clears the flag, so
 *    the call after it runs normally.  Reading the flag adds no
 *    synchronisation: a wait still running when the next call starts is
 *    reported by a later one.
 *  - A plan may be used by one stream at a time.
 */
#ifndef NUASM_H
#define NUASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nuasm_plan_s* nuasm_plan_t;   /* opaque; owned by the library */

typedef enum {
    NUASM_OK = 0,
    NUASM_EINVAL = 1,        /* invalid argument / parameter combination        */
    NUASM_ERANGE = 2,        /* a point lies outside [-N pitch/2, N pitch/2)    */
    NUASM_ENOMEM = 3,        /* device or host allocation failed                */
    NUASM_ECUDA = 4,         /* a CUDA call or an earlier asynchronous launch failed */
    NUASM_ETIMEOUT = 5,      /* a bounded device wait gave up                   */
    NUASM_EUNSUPPORTED = 6   /* valid but outside what this build implements    */
} nuasm_status;

typedef enum { NUASM_KIND_ASM = 0, NUASM_KIND_FRESNEL = 1 } nuasm_kind;

/* Spreading kernel (any kernel reaching the tolerance gives the same result to
 * within it; the exact result is the non-uniform DFT). */
typedef enum {
    NUASM_KERNEL_ES = 0,        /* exponential of semicircle, width ceil(log10(1/tol)) + 1 */
    NUASM_KERNEL_GAUSSIAN = 1   /* Gaussian (the Greengard-Lee gridding the paper uses),
                                   width ceil(ln(1/tol)/1.11) <= 26, so tol >= 3e-13 */
} nuasm_kernel;

typedef enum {
    NUASM_PREC_F32_F64PHASE = 0,  /* complex64 data; phases from FP64 tables and
                                     compensated (double-float) FP32 arithmetic */
    NUASM_PREC_F64 = 1            /* complex128 data; FP64 arithmetic, except that gridding at the
                                     kernel widths of the FP64 tolerances (see
                                     nuasm_plan_info_t.double_float) and the FFT passes of planes
                                     with N' >= 512 run in double-float arithmetic (pairs of FP32
                                     values, about 47 significant bits); results within 1e-10
                                     (rel-L2) of exact FP64 evaluation */
} nuasm_prec;

/* Problem definition (Eq. 4 / Eq. 5 parameters).  Plain old data. */
typedef struct {
    int32_t n;          /* N: side of the uniform plane, even (the paper's N' = 2N padding); this build
                           runs powers of two 16..4096 (F32) / 16..2048 (F64) and returns
                           NUASM_EUNSUPPORTED for other even sizes */
    int32_t n_pad;      /* N': 0 selects 2N (the paper's padding); else an even N' >= 2N, run when it
                           is a power of two (else NUASM_EUNSUPPORTED) */
    double  pitch;      /* pitch of the uniform plane in metres (Delta_2 for type 1, Delta_1 for type 2) */
    double  lambda;     /* wavelength, metres, > 0 */
    double  z;          /* propagation distance, metres; != 0 for Fresnel */
    double  ox, oy;     /* off-axis offset o of Eq. 4/5, metres: the destination
                           window is centred at o relative to the source window */
    int32_t band_auto;  /* ASM only.  1: Rect band derived from Nyquist sampling of
                           the transfer-function phase (keep f with
                           |o - z f / sqrt(1/lambda^2 - f^2)| <= N pitch per axis);
                           0: use c_m, c_n, w_m, w_n below */
    double  c_m, c_n;   /* Rect centre in mode-index units (x, y) when band_auto = 0 */
    double  w_m, w_n;   /* Rect full width in mode-index units: keep |k - c| <= w/2 */
    int32_t kind;       /* nuasm_kind */
    int32_t prec;       /* nuasm_prec */
    double  tol;        /* requested NUFFT relative tolerance; 0 selects 1e-6 (F32) or 1e-12 (F64) */
    int32_t kernel;     /* nuasm_kernel: spreading kernel of the NUFFT gridding */
    int32_t tile;       /* side of the gridding tiles (bins) in fine-grid cells: 16, 32 or 64;
                           0 = the library's rule (the largest side giving at least 608
                           tiles over the fine-grid window, else 16; at least w - 1 for
                           a kernel of w taps).  A side below w - 1 returns
                           NUASM_EUNSUPPORTED.  Results agree to rounding for every
                           choice; nuasm_autotune_tile measures which is fastest. */
    int32_t interp_chunk;  /* type-2 interpolation: 0 = one CTA per tile; N >= 64 = a tile with
                              more than N home records is split into chunks of at most N
                              (rounded up to a multiple of 32), one CTA each.  Results are the
                              same bit for bit; values 1..63 or < 0 return NUASM_EINVAL. */
    int32_t spread_chunk;  /* type-1 spreading, for the kernels that can split a tile (FP64, and
                              FP32 tiles of side <= 32): 0 = the library's rule (a tile with
                              more records than the larger of 128 (FP64) / 512 (FP32) and an
                              even share over two CTAs per SM is split into chunks of at most
                              that many, each adding into the window); -1 = never split;
                              N >= 32 = split above N records.  Results agree to rounding;
                              other values return NUASM_EINVAL.  nuasm_autotune measures the
                              fastest tile side and chunk sizes. */
} nuasm_params_t;

/* Geometry of a plan (read-only report). */
typedef struct {
    int32_t n, n_pad;          /* N, N' */
    int32_t grid;              /* oversampled NUFFT grid side G = 2 N' */
    int32_t window;            /* side W of the non-zero fine-grid window (2N + 2h) */
    int32_t window_origin;     /* first fine-grid index of the window */
    int32_t kernel_width;      /* spreading kernel width w (taps per axis) */
    double  kernel_beta;       /* exponential-of-semicircle shape parameter */
    int32_t tile;              /* tile side used for spreading / interpolation */
    int32_t tiles;             /* number of tiles */
    int32_t band_lo_x, band_hi_x, band_lo_y, band_hi_y;  /* kept modes, inclusive (ASM) */
    int64_t points;            /* M */
    int64_t records;           /* binned records (points plus tile-halo duplicates) */
    int64_t device_bytes;      /* device memory owned by the plan */
    int64_t phase_table_bytes; /* of which the tabulated non-separable ASM phase factor
                                  (Eq. 4) and its type-2 product with the per-column
                                  factor (0 when the plan evaluates it per mode) */
    int32_t bank_skew;         /* shared-memory bank skew of the gridding tiles (0 or 2; 0 .. 8
                                  in builds with a skew per tile, then the one most tiles
                                  use), chosen from the points' distribution */
    int32_t spread_split_ctas; /* CTAs of type-1 spreading over split dense tiles (0: one CTA
                                  per whole tile) */
    int32_t double_float;      /* 1: FP64 gridding runs in double-float arithmetic (pairs of
                                  FP32 values, about 47 significant bits) on the FP32 pipe --
                                  FP64 plans with the ES kernel at w = 11 or 13 or the
                                  Gaussian at w = 15, 21 or 25 */
} nuasm_plan_info_t;

/*
 * nuasm_plan -- build a plan for one plane geometry and one set of non-uniform
 * points (Eq. 4-9; coordinate normalisation as in the paper's Fig. 1
 * discussion).  Validates the parameters, derives the Rect band (Eq. 4), the
 * Fresnel transfer-function tables (Eq. 5), the NUFFT kernel and its
 * deconvolution, and sorts the points into fine-grid tiles on the device.
 *
 *  out      receives the plan (set to NULL on failure).
 *  p        parameters (host memory, copied).
 *  m        number of non-uniform points, >= 0.
 *  x, y     m coordinates in metres (device or host memory; read during the
 *           call only).  May be NULL when m == 0.
 *  w        optional per-point weights multiplying the type-1 source values
 *           (quadrature weights; NULL = 1 for every point, the paper's
 *           unweighted Eq. 7).  Device or host memory.
 *  stream   stream for the plan's device work; the call synchronises it
 *           before returning.
 *
 * Returns NUASM_EINVAL for bad parameters (N odd or < 2, N' odd or < 2N,
 * pitch/lambda <= 0, Fresnel with z == 0, m < 0, NULL coordinates with
 * m > 0, tol outside (0, 0.1]), NUASM_EUNSUPPORTED for valid problems this
 * build does not run (N or N' not a power of two, N < 16, N' above 8192
 * (F32) / 4096 (F64), a kernel needing more than 16 taps for the tolerance),
 * NUASM_ERANGE if any point is outside the window, NUASM_ENOMEM, NUASM_ECUDA.
 * A failure releases everything the call had acquired.  The plan allocates all the device memory
 * its execute calls will need.  For the ASM with z != 0 that includes a table
 * of the transfer function's non-separable phase factor over |kx|, |ky| in
 * [0, N'/2] (about N'^2/4 complex values in the plan precision, computed in
 * FP64 during the call), which the execute calls read instead of evaluating a
 * square root and a sine/cosine per mode; FP32 plans with N' <= 4096 add the
 * same factor times type 2's per-column table (about N'^2/2 complex64).
 */
nuasm_status nuasm_plan(nuasm_plan_t* out, const nuasm_params_t* p, int64_t m,
                        const double* x, const double* y, const double* w, void* stream);

/*
 * nuasm_plan_lattice -- a plan whose points form a uniform nx x ny lattice,
 *     x = x0 + i * pitch2,  y = y0 + j * pitch2,  point index j * nx + i,
 * binned on the device without a sort and without coordinate arrays (a
 * tile's points are a product of one index range per axis).  With it, type 2 evaluates
 * the destination plane at pitch2 and type 1 propagates a source plane
 * sampled at pitch2 onto the uniform plane at p->pitch: the scaled ASM /
 * scaled Fresnel the paper's introduction discusses (different but uniform
 * pitches on the two planes), as the lattice special case of NU-ASM.
 * nx, ny >= 0 (nx * ny <= 2^29), pitch2 > 0; every lattice point must lie
 * in the window (else NUASM_ERANGE).  Other arguments and errors as
 * nuasm_plan (no weights).
 */
nuasm_status nuasm_plan_lattice(nuasm_plan_t* out, const nuasm_params_t* p, int32_t nx, int32_t ny,
                                double pitch2, double x0, double y0, void* stream);

/*
 * nuasm1_execute -- NU-ASM_1 (Eq. 6): non-uniform source -> uniform plane.
 *  c   m complex source values in the order the plan's points were given.
 *  u2  N*N complex output plane.
 * Plan kind must be NUASM_KIND_ASM (else NUASM_EINVAL).
 */
nuasm_status nuasm1_execute(nuasm_plan_t plan, const void* c, void* u2, void* stream);

/*
 * nuasm2_execute -- NU-ASM_2 (Eq. 9): uniform plane -> non-uniform points.
 *  u1  N*N complex source plane.
 *  v   m complex outputs, in the order of the plan's points.
 * Plan kind must be NUASM_KIND_ASM (else NUASM_EINVAL).
 */
nuasm_status nuasm2_execute(nuasm_plan_t plan, const void* u1, void* v, void* stream);

/*
 * nufresnel_execute -- NU-FRE_1 / NU-FRE_2: Eq. 6 / Eq. 9 with the Fresnel
 * transfer function of Eq. 5.  type = 1: `in` holds m source values and
 * `out` the N*N plane; type = 2: `in` holds the N*N plane and `out` the m
 * point values.  Plan kind must be NUASM_KIND_FRESNEL and type 1 or 2.
 */
nuasm_status nufresnel_execute(nuasm_plan_t plan, int32_t type, const void* in, void* out,
                               void* stream);

/*
 * nuasm3_execute -- NU-ASM_3: non-uniform source -> non-uniform destination,
 * obtained by combining NU-ASM_1 and NU-ASM_2 through the spectrum (Eq. 6-9):
 *     v_j = (1/N'^2) sum_k [sum_i w_i c_i exp(-2 pi i f_k . x_i)] H(k) exp(2 pi i f_k . y_j).
 *  src  plan whose points x_i (and optional weights w_i) are the source samples;
 *       its workspace is used.
 *  dst  plan whose points y_j are the destination samples (read only).
 *  c    src->m complex source values;  v  dst->m complex outputs.
 * Both plans must have been built with identical parameters (else
 * NUASM_EINVAL) and kind NUASM_KIND_ASM.
 */
nuasm_status nuasm3_execute(nuasm_plan_t src, nuasm_plan_t dst, const void* c, void* v, void* stream);

/* nufresnel3_execute -- NU-FRE_3: as nuasm3_execute with the Fresnel transfer
 * function of Eq. 5 (both plans of kind NUASM_KIND_FRESNEL). */
nuasm_status nufresnel3_execute(nuasm_plan_t src, nuasm_plan_t dst, const void* c, void* v, void* stream);

/*
 * nuasm_rs_direct -- Rayleigh-Sommerfeld diffraction (Eq. 10) as a direct
 * O(m1 m2) sum: the rigorous reference the paper measures NU-ASM and NU-FRE
 * against (its experiments and Fig. 4).
 *     u2(x2) = (1/2 pi) sum_j a_j c_j (z/r)(1 - i k r) exp(i k r) / r^2,
 *     r = sqrt(|x2 + o - x1_j|^2 + z^2),  k = 2 pi / lambda.
 *  p        uses lambda, z (> 0), ox, oy and prec only (no plan is built).
 *  x1, y1   m1 source coordinates (metres), device memory.
 *  c        m1 complex source values (complex64 for NUASM_PREC_F32_F64PHASE,
 *           complex128 for NUASM_PREC_F64), device memory.
 *  area     m1 area elements a_j (square metres), device memory.
 *  x2, y2   m2 destination coordinates relative to the destination window
 *           centre o, device memory.
 *  out      m2 complex outputs, device memory.
 * Asynchronous on `stream`; NUASM_EINVAL for bad parameters or host pointers.
 * FP32 evaluates the phase as 2 pi (frac(z/lambda) + (r - z)/lambda) with
 * r - z = rho^2/(r + z); FP64 evaluates every term in double precision.
 */
nuasm_status nuasm_rs_direct(const nuasm_params_t* p, int64_t m1, const double* x1, const double* y1,
                             const void* c, const double* area, int64_t m2, const double* x2, const double* y2,
                             void* out, void* stream);

/*
 * nuasm_autotune_tile -- time one solve of `type` (1 or 2) on the given
 * points for each tile side (16, 32, 64) and return the fastest in *tile
 * (and its time in *ms, may be NULL).  The paper has no counterpart.  p->tile
 * is ignored; x, y (device, m entries) as for nuasm_plan.  Builds and
 * destroys temporary plans and zero-filled input/output arrays; synchronises
 * `stream`.  Errors as nuasm_plan.
 */
nuasm_status nuasm_autotune_tile(const nuasm_params_t* p, int64_t m, const double* x, const double* y, int32_t type,
                                 void* stream, int32_t* tile, double* ms);

/*
 * nuasm_autotune -- the project's autotuner over the gridding knobs that only
 * change speed (the paper has no counterpart): for each tile side (16, 32,
 * 64 that the kernel width allows) and, for type 2, interpolation chunks
 * (interp_chunk 0, 1024, 2048) or, for type 1, spreading splits
 * (spread_chunk 0, -1, 256), it builds a plan on the given points, times one
 * solve of `type` (1 or 2) with CUDA events (after one untimed solve; three
 * timed) and writes the fastest parameters to *best (a copy of *p with tile,
 * interp_chunk and spread_chunk set) and their time to *ms (may be NULL).
 * The spreading width is not searched: it is the smallest that meets p->tol
 * for p->kernel.  x, y (device, m entries) as for nuasm_plan.  Builds and
 * destroys temporary plans and zero-filled arrays; synchronises `stream`.
 * Errors as nuasm_plan; best NULL or type not 1/2: NUASM_EINVAL.
 */
nuasm_status nuasm_autotune(const nuasm_params_t* p, int64_t m, const double* x, const double* y, int32_t type,
                            void* stream, nuasm_params_t* best, double* ms);

/*
 * nuasm_debug_plan_wait -- the same diagnostic aimed at a plan (the paper has
 * no counterpart): runs the bounded wait on an mbarrier nothing completes,
 * with `plan`'s error word as the flag it sets when it gives up after
 * `spins` try-waits (1 .. 2^24), exactly as a column pass whose copy never
 * arrived would.  Synchronises `stream` and returns NUASM_OK; the plan's
 * next execute call then returns NUASM_ETIMEOUT.  NUASM_EINVAL for a NULL
 * plan or a bad count.
 */
nuasm_status nuasm_debug_plan_wait(nuasm_plan_t plan, int32_t spins, void* stream);

/*
 * nuasm_debug_fail_alloc -- test hook for the clean-up paths (the paper has
 * no counterpart).  k > 0: the k-th resource acquisition of the library from
 * now on -- a device, pool or pinned host allocation, a stream, an event or a
 * graph instantiation, in any call and any thread -- fails as if the device
 * were out of memory (the call that made it returns NUASM_ENOMEM, a server
 * request that made it completes with that status); the hook then disarms.
 * k = 0 disarms it.  NUASM_EINVAL for k < 0.  Host only.
 */
nuasm_status nuasm_debug_fail_alloc(int64_t k);

/*
 * nuasm_debug_live_resources -- number of the library's resource
 * acquisitions (as counted by nuasm_debug_fail_alloc) not yet released, in
 * *count.  After a failed call it is back where it was before the call.
 * Host only.
 */
nuasm_status nuasm_debug_live_resources(int64_t* count);

/*
 * nuasm_debug_bounded_wait -- diagnostic for the failure path of the bounded
 * device waits (the paper has no counterpart).  Runs one CTA that waits, with
 * the loop the TMA column passes use, on an mbarrier nothing completes,
 * giving up after `spins` try-waits (1 .. 2^24).  Returns NUASM_ETIMEOUT when
 * the wait gave up (always, unless the device fails), after which the device
 * context stays usable; NUASM_EINVAL for a bad count.  Synchronises `stream`.
 */
nuasm_status nuasm_debug_bounded_wait(int32_t spins, void* stream);

/*
 * nuasm_debug_bounds -- bounds records of the debug library (the paper has no
 * counterpart; a stand-in for a memory checker).  The library built with
 * NUASM_DEBUG_BOUNDS=1 (libnuasm_debug.so) checks the shared- and
 * global-memory indices and TMA coordinates its kernels compute against the
 * extents of the buffers they address, skips any access that would fall
 * outside and counts it.  After a device synchronisation, *hits receives the
 * number of skipped accesses since the last reset (0 when every access was in
 * range) and, when it is non-zero, *site / *index / *limit the check site
 * code, the index and the extent of the first one (any of the three may be
 * NULL).  reset != 0 clears the records.  hits NULL: NUASM_EINVAL.  The normal
 * library has no checks: it sets *hits = -1 and returns NUASM_EUNSUPPORTED.
 */
nuasm_status nuasm_debug_bounds(int64_t* hits, int32_t* site, int64_t* index, int64_t* limit, int32_t reset);

/* Release every resource of the plan (synchronises the plan's device work). NULL is a no-op. */
nuasm_status nuasm_destroy(nuasm_plan_t plan);

/* Static English description of a status code. */
const char* nuasm_strerror(nuasm_status s);

/* Copy the plan's geometry into *info (host only, no device work). */
nuasm_status nuasm_plan_info(nuasm_plan_t plan, nuasm_plan_info_t* info);

/*
 * nuasm_band -- host-only evaluation of the Rect band of Eq. 4 for the given
 * parameters, as inclusive mode-index ranges [lo, hi] per axis (out[0..3] =
 * lo_x, hi_x, lo_y, hi_y, clamped to [-N'/2, N'/2 - 1]; an empty band has
 * lo > hi).  Fresnel parameters give the full range.  No device work.
 */
nuasm_status nuasm_band(const nuasm_params_t* p, int32_t out[4]);

/*
 * nuasm_kernel_shape -- host-only: the spreading kernel width w and shape
 * parameter beta the library uses for a requested tolerance (0 = the
 * precision's default), precision and kernel (nuasm_kernel): exp(beta
 * (sqrt(1 - (2t/w)^2) - 1)) for the exponential of semicircle, exp(-beta t^2)
 * for the Gaussian, t in fine-grid cells, |t| <= w/2.  NUASM_EUNSUPPORTED
 * when the kernel needs more taps than this build runs for the tolerance (16
 * for the exponential of semicircle, which reaches 1e-15 within them; 26 for
 * the Gaussian).  No device work.
 */
nuasm_status nuasm_kernel_shape(double tol, int32_t prec, int32_t kernel, int32_t* width, double* beta);

/*
 * Per-stage timing (instrumentation for benchmarks).  When enabled, execute
 * calls record CUDA events around each stage on their stream; nuasm_profile_read
 * synchronises on the last recorded event and returns the summed elapsed
 * milliseconds and launch counts per stage since the last reset (arrays of
 * NUASM_STAGE_COUNT entries), then resets.  Stage names come from
 * nuasm_stage_name.  Disabled by default; enabling adds event records only.
 */
enum {
    NUASM_STAGE_H2D = 0, NUASM_STAGE_SPREAD, NUASM_STAGE_COL_FWD_FOLD, NUASM_STAGE_ROW_T1,
    NUASM_STAGE_COL_INV, NUASM_STAGE_COL_FWD, NUASM_STAGE_ROW_T2, NUASM_STAGE_COL_INV_FOLD,
    NUASM_STAGE_INTERP, NUASM_STAGE_D2H, NUASM_STAGE_ROW_T3, NUASM_STAGE_COUNT
};
nuasm_status nuasm_profile_enable(nuasm_plan_t plan, int32_t enable);
nuasm_status nuasm_profile_read(nuasm_plan_t plan, double* ms, int64_t* launches);
const char* nuasm_stage_name(int32_t stage);

/*
 * nuasm2_solve_noalloc -- NU-ASM_2 (the same result as nuasm_plan followed by
 * nuasm2_execute) in one call that allocates nothing.  The paper has no
 * counterpart: this exists for callers that must not call cudaMalloc or any
 * allocating routine -- plug-ins whose host framework owns all device
 * memory, real-time loops that cannot take an allocation's latency or
 * failure.  Those callers cannot build a plan, so the plan work and the
 * solve happen here, with every intermediate in one 16 MiB file-scope device
 * array that every GPU loading the library holds until the process exits.
 * The call copies its tables from host memory, reads its error word back and
 * synchronises its stream before returning.
 *
 *  p         parameters; kind must be NUASM_KIND_ASM and prec
 *            NUASM_PREC_F32_F64PHASE (else NUASM_EINVAL).
 *  m         number of destination points, 0 <= m <= 65536.
 *  x, y      m coordinates in metres, device memory.
 *  u1        N*N complex64 source plane, device memory.
 *  v         m complex64 outputs in point order, device memory.
 *  stream    stream for the work; the call waits for it to finish before
 *            returning (it reads back the out-of-window flag).
 *
 * Limits: N <= 256 and N' <= 512 and m <= 65536, else NUASM_EUNSUPPORTED;
 * host pointers give NUASM_EINVAL; a point outside the window gives
 * NUASM_ERANGE and a bounded device wait that gave up NUASM_ETIMEOUT.  The device address of the array is looked
 * up on the first call made on each device; make that first call before any
 * stream capture begins.  Every call reuses the same array (counters are
 * cleared at the start of each call); calls whose device work overlaps --
 * other streams, other host threads -- race on it and must be serialised by
 * the caller.
 */
nuasm_status nuasm2_solve_noalloc(const nuasm_params_t* p, int64_t m, const double* x, const double* y,
                                  const void* u1, void* v, void* stream);

/*
 * Batches -- many planes (depth layers, colour channels, mixed N and point
 * counts) solved together.  The paper solves one plane per call; a batch is
 * a fixed list of solves on existing plans that nuasm_batch_create records
 * once into a CUDA graph, distributing the planes over `lanes` internal
 * streams so that planes too small to fill the GPU run side by side, and
 * that nuasm_batch_execute replays with a single graph launch.
 *
 * Items that name the same `plan` share its workspace: they are placed on
 * one lane and run in list order.  Other planes are assigned to lanes
 * longest-first by an estimate of their HBM bytes and kernel taps.
 * The plans and every `in`/`out` array are caller-owned device memory that
 * must stay valid, at the same addresses, for the life of the batch (their
 * addresses are baked into the graph); the contents of `in` are read anew on
 * every execute.
 */
typedef struct nuasm_batch_s* nuasm_batch_t;

typedef struct {
    nuasm_plan_t plan;   /* the plane's plan (type 3: the source plan) */
    nuasm_plan_t dst;    /* type 3: destination plan built with identical parameters; else NULL */
    int32_t type;        /* 1 (Eq. 6), 2 (Eq. 9) or 3 (both planes non-uniform); the
                            transfer function (Eq. 4 or Eq. 5) is the plan's kind */
    const void* in;      /* device: type 1/3 m source values, type 2 the N*N plane */
    void* out;           /* device: type 1 the N*N plane, type 2 m values, type 3 dst->m values */
} nuasm_batch_item_t;

/*
 * nuasm_batch_create -- validate `count` items (1..65536) and record them.
 * lanes: 1..64 concurrent streams (0 = 8).  NUASM_EINVAL for a NULL plan, a
 * type that is not 1-3, host pointers, or type-3 plans whose parameters
 * differ; NUASM_ECUDA when capture or instantiation fails.  No device work
 * is run by this call.
 */
nuasm_status nuasm_batch_create(nuasm_batch_t* out, const nuasm_batch_item_t* items, int32_t count, int32_t lanes);

/* Run every item once: one graph launch on `stream`, asynchronous; the work
 * is ordered after earlier work on `stream` and later work waits for all of it. */
nuasm_status nuasm_batch_execute(nuasm_batch_t batch, void* stream);

/* lanes actually used and kernel launches per execute (host only). */
nuasm_status nuasm_batch_info(nuasm_batch_t batch, int32_t* lanes, int64_t* kernels);

/* Release the graph and the batch's streams (synchronises the device). NULL is a no-op. */
nuasm_status nuasm_batch_destroy(nuasm_batch_t batch);

/*
 * Serving -- a request loop with continuous batching.  The paper times
 * single solves and has no counterpart.  A server runs `slots` worker
 * threads, each with its own CUDA stream.  Submitted requests wait in one
 * FIFO queue; the head is admitted as soon as a slot is free and its device
 * memory fits in the budget, and then runs on that slot's stream while the
 * other slots run theirs, so requests arriving while others are on the GPU
 * overlap with them on the device (copies of one with kernels of another).
 *
 * Resident point sets: a request names its points by a non-zero `points_id`.
 * The first request with a given (points_id, n, n_pad, pitch, prec, tol,
 * kernel) bins its points (reading x, y); later requests with the same key
 * reuse the resident bins and do not read x, y.  Wavelength, distance,
 * offset, band and kind may differ between requests on one point set: the
 * FP64 transfer-function tables (Eq. 4 / Eq. 5) are built per request, while
 * the kernel's Fourier transform and the FFT twiddles stay with the bins.
 * Resident sets not in use are evicted least recently used when the budget
 * needs room; points_id = 0 bins the points for that request only.
 *
 * Memory: resident sets plus, per admitted request, its workspace (the
 * fine-grid window and two pass buffers), tables and input/output copies,
 * taken from a stream-ordered pool owned by the server and returned when the
 * request completes.  The budget bounds their sum.
 */
typedef struct nuasm_server_s* nuasm_server_t;

typedef struct {
    int32_t slots;        /* requests on the device at once, 1..32 (0 = 4) */
    int32_t device;       /* CUDA device ordinal */
    int64_t hbm_budget;   /* bytes for resident sets + admitted requests (0 = 150e9) */
} nuasm_server_config_t;

typedef struct {
    nuasm_params_t p;     /* as for nuasm_plan */
    int32_t type;         /* 1 (Eq. 6) or 2 (Eq. 9); the transfer function is p.kind */
    uint64_t points_id;   /* key of the point set; 0 = not kept */
    int64_t m;            /* number of points */
    const double* x;      /* m coordinates in metres (host or device), read only when the set is binned */
    const double* y;
    const void* in;       /* type 1: m values, type 2: the N*N plane (complex64, or complex128 for
                             NUASM_PREC_F64); host or device memory */
    void* out;            /* type 1: the N*N plane, type 2: m values; host or device memory */
} nuasm_request_t;

typedef struct {
    int32_t status;          /* nuasm_status of the request */
    int32_t reused_points;   /* 1 when resident bins were used */
    double latency_ms;       /* submit -> result complete in `out` */
    double queue_ms;         /* submit -> admitted to a slot */
} nuasm_request_result_t;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t points;          /* sum of m over completed requests */
    double p50_ms, p99_ms;   /* latency percentiles over completed requests */
    double wall_s;           /* first submit -> last completion */
    int64_t resident_sets, resident_bytes, bins_built, bins_reused, evictions;
    int64_t peak_bytes;      /* largest budget use */
} nuasm_server_stats_t;

/* Start the workers on `device`.  NUASM_EINVAL for a bad configuration. */
nuasm_status nuasm_server_create(nuasm_server_t* out, const nuasm_server_config_t* cfg);

/*
 * Queue a request; *ticket identifies it for nuasm_server_wait.  The
 * descriptor is copied, the arrays are not: x, y, in and out must stay valid
 * until the request's wait returns.  NUASM_EINVAL for invalid parameters,
 * type or pointers; NUASM_ENOMEM when the request alone exceeds the budget.
 * Errors found while it runs (NUASM_ERANGE for points outside the window,
 * NUASM_ECUDA, ...) are returned in its result.
 */
nuasm_status nuasm_server_submit(nuasm_server_t server, const nuasm_request_t* req, int64_t* ticket);

/*
 * Wait up to timeout_s seconds (< 0: no limit) for a request; on completion
 * fills *res and forgets the ticket (a second wait gives NUASM_EINVAL).
 * NUASM_ETIMEOUT when it is still running (the ticket stays valid).
 */
nuasm_status nuasm_server_wait(nuasm_server_t server, int64_t ticket, double timeout_s,
                               nuasm_request_result_t* res);

/* Counters and latency percentiles since creation or the last reset (reset != 0 clears them
 * after reading; resident-set figures are not reset). */
nuasm_status nuasm_server_stats(nuasm_server_t server, nuasm_server_stats_t* st, int32_t reset);

/* Finish every queued request, stop the workers and release all device memory. */
nuasm_status nuasm_server_destroy(nuasm_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* NUASM_H */
