// NUFFT gridding: point binning (plan time), type-1 spreading and type-2
// interpolation on the oversampled fine grid (Eq. 7 / Eq. 8, the gridding
// step of Greengard and Lee's NUFFT that the paper uses).
//
// Coordinate normalisation (the paper's x' = 2 pi (o' + x)/N, read as a map of
// the window onto the central half of the padded period): a point x (metres)
// becomes xi = x / pitch in [-N/2, N/2), then g = 2 (xi + N'/2) on the fine
// grid of G = 2N' cells per period.  Relative to the window origin Lo =
// N' - N - h (h = ceil(w/2)) this is g_w = 2 xi + N + h, and the w taps of the
// kernel sit at l0 + i, i in [0, w), l0 = ceil(g_w - w/2), with offsets
// t_i = i + f - w/2, f = l0 - (g_w - w/2) in [0, 1).  The split into the
// integer cell and the fraction f is done in FP64 once per plan.
//
// The kernel is the exponential of semicircle
//   phi(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1)),  |t| <= w/2,
// or the truncated Gaussian; each tap phi(i + f - w/2) is evaluated from a
// polynomial in f fitted at plan time (the fit error sits below the kernel's
// own truncation error in both precisions).
//
// Tiles: the W x W window is cut into T x T tiles.  Each point is binned to the
// tile that holds its first tap l0 (its home tile) and duplicated into the +x,
// +y and +x+y neighbours its taps reach.  Spreading is output-stationary: one
// CTA owns one tile, accumulates every record of its bin into shared memory
// (shared-memory atomics, or for small tiles one private copy per warp with
// plain read-modify-writes; no global atomics) clipping taps to the tile, and
// writes the tile once.  Interpolation loads the tile plus a (w-1) halo into
// shared memory and evaluates its home records only.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"
#include "nuasm_internal.h"

namespace nuasm {

// Binned point records.  cell = l0y << 16 | l0x (window coordinates of the first tap).
struct RecF { uint32_t cell; float fx, fy; int32_t j; };
struct RecD { uint32_t cell; int32_t j; double fx, fy; };

template <typename S> struct RecOf;
template <> struct RecOf<float> { using type = RecF; };
template <> struct RecOf<double> { using type = RecD; };

namespace {

struct BinArgs {
    int n, W, T, ntx, w, h;
    double pitch;
    int64_t m;
    int64_t cap = 0;   // record slots (extent for the debug library's checks)
};

struct PointSplit { int l0x, l0y; double fx, fy; bool ok; };

__device__ __forceinline__ PointSplit split_point(double x, double y, const BinArgs& a) {
    PointSplit s;
    const double xi = x / a.pitch, yi = y / a.pitch;
    const double half = 0.5 * a.n;
    s.ok = xi >= -half && xi < half && yi >= -half && yi < half;
    const double gx = 2.0 * xi + double(a.n + a.h) - 0.5 * a.w;
    const double gy = 2.0 * yi + double(a.n + a.h) - 0.5 * a.w;
    const double cx = ceil(gx), cy = ceil(gy);
    s.l0x = int(cx);
    s.l0y = int(cy);
    s.fx = cx - gx;
    s.fy = cy - gy;
    if (!s.ok) { s.l0x = 0; s.l0y = 0; s.fx = 0; s.fy = 0; }
    return s;
}

// up to four tiles per point: home, +x, +y, +x+y
__device__ __forceinline__ int point_tiles(const PointSplit& s, const BinArgs& a, int tiles[4]) {
    const int tx = s.l0x / a.T, ty = s.l0y / a.T;
    const bool dx = (s.l0x - tx * a.T) + a.w - 1 >= a.T;
    const bool dy = (s.l0y - ty * a.T) + a.w - 1 >= a.T;
    int k = 0;
    tiles[k++] = ty * a.ntx + tx;
    if (dx) tiles[k++] = ty * a.ntx + tx + 1;
    if (dy) tiles[k++] = (ty + 1) * a.ntx + tx;
    if (dx && dy) tiles[k++] = (ty + 1) * a.ntx + tx + 1;
    return k;
}

__global__ void bin_count_kernel(const double* __restrict__ x, const double* __restrict__ y, BinArgs a,
                                 int* __restrict__ home_cnt, int* __restrict__ dup_cnt, int* __restrict__ err) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.m; i += int64_t(gridDim.x) * blockDim.x) {
        PointSplit s = split_point(x[i], y[i], a);
        if (!s.ok) { atomicOr(err, 1); continue; }
        int t[4];
        const int k = point_tiles(s, a, t);
        atomicAdd(&home_cnt[t[0]], 1);
        for (int q = 1; q < k; ++q) atomicAdd(&dup_cnt[t[q]], 1);
    }
}

// exclusive scan of home_cnt + dup_cnt into off[0..ntiles], single CTA of 1024 threads
__global__ void bin_scan_kernel(const int* __restrict__ home_cnt, const int* __restrict__ dup_cnt,
                                int ntiles, int* __restrict__ off, int* __restrict__ home) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, P = blockDim.x;
    const int chunk = (ntiles + P - 1) / P;
    const int b = t * chunk, e = min(ntiles, b + chunk);
    long long acc = 0;
    for (int i = b; i < e; ++i) acc += home_cnt[i] + dup_cnt[i];
    part[t] = acc;
    __syncthreads();
    for (int d = 1; d < P; d <<= 1) {
        long long v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - acc;
    for (int i = b; i < e; ++i) {
        off[i] = int(run);
        home[i] = home_cnt[i];
        run += home_cnt[i] + dup_cnt[i];
    }
    if (t == P - 1) off[ntiles] = int(part[P - 1]);
}

template <typename Rec, typename S>
__global__ void bin_scatter_kernel(const double* __restrict__ x, const double* __restrict__ y, BinArgs a,
                                   const int* __restrict__ off, const int* __restrict__ home_cnt,
                                   int* __restrict__ cur_home, int* __restrict__ cur_dup, Rec* __restrict__ rec) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.m; i += int64_t(gridDim.x) * blockDim.x) {
        PointSplit s = split_point(x[i], y[i], a);
        if (!s.ok) continue;
        int t[4];
        const int k = point_tiles(s, a, t);
        Rec r;
        r.cell = (uint32_t(s.l0y) << 16) | uint32_t(s.l0x);
        r.fx = S(s.fx);
        r.fy = S(s.fy);
        r.j = int32_t(i);
        for (int q = 0; q < k; ++q) {
            int pos;
            if (q == 0) pos = off[t[0]] + atomicAdd(&cur_home[t[0]], 1);
            else pos = off[t[q]] + home_cnt[t[q]] + atomicAdd(&cur_dup[t[q]], 1);
            if (NUASM_IN_RANGE(pos, a.cap, dbg::kBinRec)) rec[pos] = r;
        }
    }
}

// Shared-memory tile rows are laid out `skew` words (32-bit planes), 8-byte or
// 16-byte elements apart modulo the 32 banks: a tap at tile cell (x, y) sits in
// bank class (skew y + x) mod 32 (mod 16 for 8-byte, mod 8 for 16-byte
// elements), and the records are ordered by that class of their first tap.
// With skew 0 the class is the column alone, which repeats whenever points sit
// on a lattice coarser than the fine grid (every 4th column at the 16 um edge
// of the graded NU-ASM_2 plane); skew 2 mixes in the row.  The plan takes
// skew 2 only where it balances the classes clearly better (class_balance),
// since on unstructured clusters skew 0 measured faster at equal balance.
// A warp's 32 records can only have distinct classes while the tile's classes
// are balanced, and in sparse tiles their counts are uneven (Poisson).  With
// NUASM_TILE_SKEW each tile takes instead the even skew (0 .. 8) that
// minimises the largest class count of its home records (tile_skew_kernel;
// 0 unless another is strictly better).  A CPU model of the bank pattern
// gives 18% fewer shared-memory wavefronts for the spreading atomics on the
// 4M clustered points, but measured: spreading 283 -> 296 us there, the
// interpolation 29.2 -> 28.7 us (NU-ASM_2 benchmark) and 95.3 -> 94.2 us
// (4M clustered points); off by default.
#ifndef NUASM_TILE_SKEW
#define NUASM_TILE_SKEW 0   // 1: a bank skew per tile
#endif
constexpr int kNumSkews = 5, kMaxSkew = 8;
__host__ __device__ constexpr int skew_candidate(int i) { return 2 * i; }   // 0, 2, 4, 6, 8
__host__ __device__ constexpr int plane_stride(int T, int skew) { return T + skew; }   // T = 32, 64: = skew mod 32
__host__ __device__ constexpr int halo_pitch(int th, int skew) { return th + (((skew - th) % 16) + 16) % 16; }

// Per tile: the candidate skew whose largest class count over the tile's home
// records is smallest (ties keep the smaller skew); hist[i] counts the tiles
// that chose candidate i.
template <typename Rec>
__global__ void tile_skew_kernel(const Rec* __restrict__ rec, const int* __restrict__ off,
                                 const int* __restrict__ home, int T, int ntx, int8_t* __restrict__ tskew,
                                 unsigned long long* __restrict__ hist) {
    __shared__ int cnt[kNumSkews][32];
    __shared__ int best[kNumSkews];
    const int tile = blockIdx.x;
    const int x0 = (tile - (tile / ntx) * ntx) * T, y0 = (tile / ntx) * T;
    for (int i = threadIdx.x; i < kNumSkews * 32; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    for (int i = off[tile] + threadIdx.x; i < off[tile] + home[tile]; i += blockDim.x) {
        const uint32_t cell = rec[i].cell;
        const int lx = int(cell & 0xffffu) - x0, ly = int(cell >> 16) - y0;
#pragma unroll
        for (int k = 0; k < kNumSkews; ++k) atomicAdd(&cnt[k][(skew_candidate(k) * ly + lx) & 31], 1);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < kNumSkews) {
        int m = cnt[warp][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) best[warp] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int bi = 0;
        for (int k = 1; k < kNumSkews; ++k)
            if (best[k] < best[bi]) bi = k;
        tskew[tile] = int8_t(skew_candidate(bi));
        atomicAdd(&hist[bi], 1ull);
    }
}

// Sum over tiles of the largest bank-class count of the tile's home records
// (the ones interpolation visits and most of what spreading visits), for skew
// 0 (sums[0]) and skew 2 (sums[1]): the record slots a perfectly balanced warp
// schedule would need, up to a factor 32.
template <typename Rec>
__global__ void class_balance_kernel(const Rec* __restrict__ rec, const int* __restrict__ off,
                                     const int* __restrict__ home, int T, int ntx,
                                     unsigned long long* __restrict__ sums) {
    __shared__ int cnt[2][32];
    const int tile = blockIdx.x;
    const int x0 = (tile - (tile / ntx) * ntx) * T, y0 = (tile / ntx) * T;
    if (threadIdx.x < 64) (&cnt[0][0])[threadIdx.x] = 0;
    __syncthreads();
    for (int i = off[tile] + threadIdx.x; i < off[tile] + home[tile]; i += blockDim.x) {
        const uint32_t cell = rec[i].cell;
        const int lx = int(cell & 0xffffu) - x0, ly = int(cell >> 16) - y0;
        atomicAdd(&cnt[0][lx & 31], 1);
        atomicAdd(&cnt[1][(2 * ly + lx) & 31], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int m0 = cnt[0][threadIdx.x], m1 = cnt[1][threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
            m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        }
        if (threadIdx.x == 0) {
            atomicAdd(&sums[0], (unsigned long long)m0);
            atomicAdd(&sums[1], (unsigned long long)m1);
        }
    }
}

// Order each tile's records so that consecutive records have distinct bank
// classes (skew ly + lx) mod 32 of their first tap (round-robin over the
// 32 classes, home records and halo duplicates separately).  A warp then
// gathers (type 2) or accumulates (type 1) its w x w taps at distinct banks
// for every tap offset, as far as the tile's classes are balanced.  One CTA
// per tile, reading the unordered copy `src` and writing `dst`; the order
// within a class is arbitrary (results do not depend on record order in
// type 2; type 1 sums in shared memory whatever the order).
template <typename Rec>
__global__ void order_tile_kernel(const Rec* __restrict__ src, Rec* __restrict__ dst, const int* __restrict__ off,
                                  const int* __restrict__ home, int T, int ntx, int skew,
                                  const int8_t* __restrict__ tskew) {
    __shared__ int cnt[2][32], cur[2][32];
    const int tile = blockIdx.x;
    if (tskew) skew = tskew[tile];
    const int x0 = (tile - (tile / ntx) * ntx) * T, y0 = (tile / ntx) * T;
    auto bank_class = [&](uint32_t cell) {
        return (skew * (int(cell >> 16) - y0) + (int(cell & 0xffffu) - x0)) & 31;
    };
    const int b = off[tile], e = off[tile + 1], eh = b + home[tile];
    if (threadIdx.x < 64) {
        (&cnt[0][0])[threadIdx.x] = 0;
        (&cur[0][0])[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int i = b + threadIdx.x; i < e; i += blockDim.x)
        atomicAdd(&cnt[i >= eh][bank_class(src[i].cell)], 1);
    __syncthreads();
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        const Rec r = src[i];
        const int seg = i >= eh;
        const int c = bank_class(r.cell);
        const int rank = atomicAdd(&cur[seg][c], 1);
        int pos = 0;   // records of lower rank, then same rank and lower class
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int n = cnt[seg][k];
            pos += min(n, rank) + ((k < c && n > rank) ? 1 : 0);
        }
        dst[(seg ? eh : b) + pos] = r;
    }
}

// --------------------------------------------------------------- kernel values
// Tap weights of one axis as polynomials in x = 2f - 1 (Horner's rule; the
// coefficients beyond the fitted degree and the taps beyond w are zero, so
// the loops unroll fully): degree w + 1 in FP32, kPoly64Deg in FP64.
template <int WMAX> __device__ __forceinline__ void tap_weights(float f, const KernelPoly& kp, float* out) {
    constexpr int DMAX = WMAX + 2 < kPolyMaxD ? WMAX + 2 : kPolyMaxD;
    const float x = fmaf(2.f, f, -1.f);
#pragma unroll
    for (int i = 0; i < WMAX; ++i) {
        float acc = kp.c[i][DMAX - 1];
#pragma unroll
        for (int k = DMAX - 2; k >= 0; --k) acc = fmaf(acc, x, kp.c[i][k]);
        out[i] = acc;
    }
}
template <int WMAX> __device__ __forceinline__ void tap_weights(double f, const KernelPoly64& kp, double* out) {
    const double x = fma(2.0, f, -1.0);
#pragma unroll
    for (int i = 0; i < WMAX; ++i) {
        double acc = kp.c[i][kPoly64Deg];
#pragma unroll
        for (int k = kPoly64Deg - 1; k >= 0; --k) acc = fma(acc, x, kp.c[i][k]);
        out[i] = acc;
    }
}

template <typename S> struct PolyOf;
template <> struct PolyOf<float> { using type = KernelPoly; };
template <> struct PolyOf<double> { using type = KernelPoly64; };

template <typename S> struct VecOf;
template <> struct VecOf<float> { using type = float2; };
template <> struct VecOf<double> { using type = double2; };

struct GridArgs {
    int W, Wp, T, ntx, w;
    long long m, nrec;     // points and record slots (extents for the debug library's checks)
    int skew;   // bank skew of the tile layouts (plane_stride, halo_pitch) when tskew is null
    const int8_t* tskew;   // per-tile skews, or null
    int max_skew;          // largest skew any tile uses (sizes the shared memory)
    __device__ int skew_of(int tile) const { return tskew ? int(tskew[tile]) : skew; }
};

// --------------------------------------------------------------- spreading (type 1)
// EXACT: the kernel width is WMAX itself (compile-time loops); else w <= WMAX at run time.
// Three accumulation schemes, picked by precision and tile side in spread_impl:
// warp-private copies (small tiles), batched int32 sums (FP32, T = 64) and,
// here, shared-memory atomicAdd in the plan's precision (FP64 large tiles; on
// sm_103a a float or double shared-memory atomicAdd is a compare-and-swap
// loop -- 9.4 instructions and 2 wavefronts per float add, against one native
// operation for a 32-bit integer).  Also measured and not kept: one int32
// word per value at a single quantum per 8-row band for all of a tile's
// records (1.6x faster than float but 1.1e-5 end to end where thousands of
// random-phase points crowd a few cells -- the batched scheme fixes this by a
// quantum per batch), two words (value and remainder; slower than float), and
// one 64-bit compare-and-swap per (re, im) pair (3.9x slower than two float
// adds).
#ifndef NUASM_SPREAD_MINB
#define NUASM_SPREAD_MINB 1
#endif
#ifndef NUASM_SPREAD_FIXED
#define NUASM_SPREAD_FIXED 1       // FP32 tiles beyond the private-copy sizes: batched integer accumulation
#endif
#ifndef NUASM_SPREAD_FIXED_RPB
#define NUASM_SPREAD_FIXED_RPB 2   // records per thread per batch (4: 4% faster, 1.6x the error of dense cancelling sums)
#endif
#ifndef NUASM_SPREAD_PRIVATE
#define NUASM_SPREAD_PRIVATE 1   // per-warp private tiles where they fit (T <= 32 F32, <= 16 F64)
#endif
template <typename S, int WMAX, bool EXACT>
__global__ void __launch_bounds__(256, sizeof(S) == 4 ? NUASM_SPREAD_MINB : 1) spread_kernel(const typename RecOf<S>::type* __restrict__ rec,
                                                     const int* __restrict__ off, const double* __restrict__ wpt,
                                                     const int* __restrict__ order,
                                                     const typename VecOf<S>::type* __restrict__ c,
                                                     typename VecOf<S>::type* __restrict__ win, GridArgs a,
                                                     const typename PolyOf<S>::type kp,
                                                     const int4* __restrict__ items) {
    using V = typename VecOf<S>::type;
    extern __shared__ unsigned char smem_raw[];
    int tile, b, e, chunked = 0;
    if (items) {   // a chunk of a tile's records (several CTAs add into the tile)
        const int4 it = items[blockIdx.x];
        tile = it.x;
        b = it.y;
        e = it.z;
        chunked = it.w;
    } else {       // a whole tile, heaviest tiles first
        tile = order ? order[blockIdx.x] : blockIdx.x;
        b = off[tile];
        e = off[tile + 1];
    }
    const int T = a.T, w = EXACT ? WMAX : a.w, TS = plane_stride(T, a.skew_of(tile)), TT = T * TS;
    S* sre = reinterpret_cast<S*>(smem_raw);
    S* sim = sre + TT;
    pdl_allow_next();
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    for (int i = threadIdx.x; i < TT; i += blockDim.x) { sre[i] = S(0); sim[i] = S(0); }
    __syncthreads();
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        if (!NUASM_IN_RANGE(i, a.nrec, dbg::kSpreadRec)) continue;
        const auto r = rec[i];
        if (!NUASM_IN_RANGE(r.j, a.m, dbg::kSpreadValue)) continue;
        const int lx = int(r.cell & 0xffffu) - x0, ly = int(r.cell >> 16) - y0;
        V val = c[r.j];
        if (wpt) { const S wt = S(wpt[r.j]); val.x *= wt; val.y *= wt; }
        S wx[WMAX], wy[WMAX];
        tap_weights<WMAX>(S(r.fx), kp, wx);
        tap_weights<WMAX>(S(r.fy), kp, wy);
        const int ya = max(0, -ly), yb = min(w, T - ly);
        const int xa = max(0, -lx), xb = min(w, T - lx);
#pragma unroll(WMAX <= 16 ? WMAX : 1)
        for (int qy = 0; qy < WMAX; ++qy) {
            if (qy < ya || qy >= yb) continue;
            const S vr = val.x * wy[qy], vi = val.y * wy[qy];
            S* rowr = sre + (ly + qy) * TS + lx;
            S* rowi = sim + (ly + qy) * TS + lx;
#pragma unroll
            for (int qx = 0; qx < WMAX; ++qx) {
                if (qx < xa || qx >= xb) continue;
                if (!NUASM_IN_RANGE((ly + qy) * TS + lx + qx, TT, dbg::kSpreadPlane)) continue;
                atomicAdd(rowr + qx, vr * wx[qx]);
                atomicAdd(rowi + qx, vi * wx[qx]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int yy = i / T, xx = i - yy * T;
        const int gy = y0 + yy, gx = x0 + xx;
        if (gy < a.W && gx < a.W && NUASM_IN_RANGE(gy * (long long)a.Wp + gx, (long long)a.W * a.Wp, dbg::kSpreadWindow)) {
            V v;
            v.x = sre[yy * TS + xx];
            v.y = sim[yy * TS + xx];
            V* p = &win[size_t(gy) * a.Wp + gx];
            if (chunked) {   // the window was cleared; the tile's chunks add into it
                atomicAdd(&p->x, v.x);
                atomicAdd(&p->y, v.y);
            } else {
                *p = v;
            }
        }
    }
}

// Spreading for large FP32 tiles with integer accumulation in batches.  On
// sm_103a a shared-memory float atomicAdd is a compare-and-swap loop while a
// 32-bit integer atomicAdd is native.  The CTA takes its records in batches of
// RPB x 256; per batch it sums S = sum(|re| + |im|) of the batch's values
// (weights included) and adds every tap contribution v wx wy / q, q = S 2^-30,
// rounded to an integer, into int32 planes: a batch's sum at one cell is at
// most S / q = 2^30 in magnitude because the kernel is at most 1.  The planes
// are then folded into FP32 totals (tot += q acc) and cleared.  A contribution
// is thus rounded to within max(q/2, its own FP32 rounding), q being a 2^-30
// share of one batch's magnitude, where a float atomic rounds to the running
// cell value.  A batch whose S is zero is skipped; one whose S is not a normal
// finite number (infinities, NaNs, or values so small that q would underflow)
// adds to the totals with float atomics, so non-finite inputs propagate as in
// the float path.  The last batch of a tile folds its planes straight into
// the window write (no fold into the totals, no clearing), and folds work
// on pairs of cells (8-byte shared accesses).
//
// Measured and not kept: planes extended by a (w - 1)-cell margin so that no
// tap needs clipping (the 49 taps become straight-line atomics; 31% of the
// kernel's instructions were the clipping branches): 295 -> 309 us on the 4M
// clustered points, since the halo duplicates then add all their taps and the
// larger planes leave two CTAs per SM instead of three.  The shared-memory
// atomics take about two wavefronts each on that workload; a CPU model of the
// bank pattern gives the same 1.8x: the round-robin record order cannot give
// 32 distinct bank classes per warp once a tile's classes run unevenly
// (Poisson counts in the sparse background tiles).  Also measured and not
// kept: ordering each tile's home records as those whose taps all lie in the
// tile, then the others, so that whole warps spread without clipping (283 ->
// 265 us there), since the second segment's bank classes crowd into the
// tile's last columns and the interpolation over the same records slowed by
// more (94.8 -> 109.5 us).  And: the FP32 totals kept in the tile's own
// window cells (read and written through L2 by the folds) instead of shared
// memory, which leaves 32 KB per CTA and room for five CTAs per SM: 279 ->
// 288 us (304 us at four CTAs, 320 us at six), so more resident tiles do not
// make the shared atomics go faster.
#ifndef NUASM_SPREAD_FIXED_MINB
#define NUASM_SPREAD_FIXED_MINB 3   // CTAs per SM the register budget is set for
#endif
constexpr int kFixedThreads = 256;
template <int WMAX, bool EXACT, int RPB>
__global__ void __launch_bounds__(kFixedThreads, NUASM_SPREAD_FIXED_MINB) spread_fixed_kernel(const RecF* __restrict__ rec,
                                                                      const int* __restrict__ off,
                                                                      const double* __restrict__ wpt,
                                                                      const int* __restrict__ order,
                                                                      const float2* __restrict__ c,
                                                                      float2* __restrict__ win, GridArgs a,
                                                                      const KernelPoly kp) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ float red[kFixedThreads / 32];
    __shared__ float batch_sum;
    const int tile = order ? order[blockIdx.x] : blockIdx.x;   // heaviest tiles first
    const int T = a.T, w = EXACT ? WMAX : a.w, TS = plane_stride(T, a.skew_of(tile)), TT = T * TS;
    int* are = reinterpret_cast<int*>(smem_raw);
    int* aim = are + TT;
    float* tre = reinterpret_cast<float*>(aim + TT);
    float* tim = tre + TT;
    pdl_allow_next();
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    for (int i = threadIdx.x; i < TT; i += kFixedThreads) {
        are[i] = 0;
        aim[i] = 0;
        tre[i] = 0.f;
        tim[i] = 0.f;
    }
    const int b = off[tile], e = off[tile + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = T / 2;   // cells are folded and written in pairs
    for (int i0 = b; i0 < e; i0 += RPB * kFixedThreads) {
        RecF r[RPB];
        float2 val[RPB];
        float part = 0.f;
#pragma unroll
        for (int k = 0; k < RPB; ++k) {
            const int i = i0 + threadIdx.x + k * kFixedThreads;
            val[k] = make_float2(0.f, 0.f);
            r[k].cell = 0;
            if (i < e && NUASM_IN_RANGE(i, a.nrec, dbg::kSpreadRec)) {
                r[k] = rec[i];
                if (!NUASM_IN_RANGE(r[k].j, a.m, dbg::kSpreadValue)) r[k].j = 0;
                val[k] = c[r[k].j];
                if (wpt) {
                    const float wt = float(wpt[r[k].j]);
                    val[k].x *= wt;
                    val[k].y *= wt;
                }
                part += fabsf(val[k].x) + fabsf(val[k].y);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();   // also orders the clearing above and the previous batch's fold
        if (threadIdx.x == 0) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < kFixedThreads / 32; ++k) t += red[k];
            batch_sum = t;
        }
        __syncthreads();
        const float S = batch_sum;
        if (S == 0.f) continue;   // every value of the batch is zero (uniform)
        const bool fixed = S >= 1e-30f && S <= 3.0e38f;
        const float q = ldexpf(S, -30), inv = fixed ? 1.f / q : 1.f;
        // The batch's mode is uniform across the CTA: one copy of the tap loops
        // per mode, so that the integer atomics of clipped taps are predicated
        // instead of branching around the float path's compare-and-swap loops.
        auto add_taps = [&](auto fixed_mode) {
            constexpr bool FX = decltype(fixed_mode)::value;
            auto add = [&](int cell, float vr, float vi) {
                if (!NUASM_IN_RANGE(cell, TT, dbg::kSpreadPlane)) return;
                if constexpr (FX) {
                    atomicAdd(&are[cell], __float2int_rn(vr));
                    atomicAdd(&aim[cell], __float2int_rn(vi));
                } else {
                    atomicAdd(&tre[cell], vr);
                    atomicAdd(&tim[cell], vi);
                }
            };
#pragma unroll
            for (int k = 0; k < RPB; ++k) {
                const int i = i0 + threadIdx.x + k * kFixedThreads;
                if (i >= e) continue;
                const int lx = int(r[k].cell & 0xffffu) - x0, ly = int(r[k].cell >> 16) - y0;
                float wx[WMAX], wy[WMAX];
                tap_weights<WMAX>(r[k].fx, kp, wx);
                tap_weights<WMAX>(r[k].fy, kp, wy);
                const float sr = val[k].x * inv, si = val[k].y * inv;
                const int ya = max(0, -ly), yb = min(w, T - ly);
                const int xa = max(0, -lx), xb = min(w, T - lx);
#pragma unroll(WMAX <= 16 ? WMAX : 1)
                for (int qy = 0; qy < WMAX; ++qy) {
                    if (qy < ya || qy >= yb) continue;
                    const float vr = sr * wy[qy], vi = si * wy[qy];
                    const int rowi = (ly + qy) * TS + lx;
#pragma unroll
                    for (int qx = 0; qx < WMAX; ++qx) {
                        if (qx < xa || qx >= xb) continue;
                        add(rowi + qx, vr * wx[qx], vi * wx[qx]);
                    }
                }
            }
        };
        if (fixed) add_taps(std::true_type{});
        else add_taps(std::false_type{});
        if (fixed) {
            __syncthreads();
            if (i0 + RPB * kFixedThreads >= e) {
                // last batch: fold into the window write
                for (int i = threadIdx.x; i < T * half; i += kFixedThreads) {
                    const int yy = i / half, xx = 2 * (i - yy * half), j = yy * TS + xx;
                    const int2 rr = *reinterpret_cast<const int2*>(&are[j]);
                    const int2 mm = *reinterpret_cast<const int2*>(&aim[j]);
                    const float2 tr = *reinterpret_cast<const float2*>(&tre[j]);
                    const float2 ti = *reinterpret_cast<const float2*>(&tim[j]);
                    const int gy = y0 + yy, gx = x0 + xx;
                    if (gy < a.W && gx < a.W &&   // W, x0 and xx are even: both cells or neither
                        NUASM_IN_RANGE(gy * (long long)a.Wp + gx + 1, (long long)a.W * a.Wp, dbg::kSpreadWindow))
                        *reinterpret_cast<float4*>(&win[size_t(gy) * a.Wp + gx]) =
                            make_float4(fmaf(float(rr.x), q, tr.x), fmaf(float(mm.x), q, ti.x),
                                        fmaf(float(rr.y), q, tr.y), fmaf(float(mm.y), q, ti.y));
                }
                return;
            }
            for (int i = threadIdx.x; i < T * half; i += kFixedThreads) {
                const int yy = i / half, xx = 2 * (i - yy * half), j = yy * TS + xx;
                int2* pr = reinterpret_cast<int2*>(&are[j]);
                int2* pm = reinterpret_cast<int2*>(&aim[j]);
                float2* pa = reinterpret_cast<float2*>(&tre[j]);
                float2* pb = reinterpret_cast<float2*>(&tim[j]);
                const int2 rr = *pr, mm = *pm;
                const float2 tr = *pa, ti = *pb;
                *pa = make_float2(fmaf(float(rr.x), q, tr.x), fmaf(float(rr.y), q, tr.y));
                *pb = make_float2(fmaf(float(mm.x), q, ti.x), fmaf(float(mm.y), q, ti.y));
                *pr = make_int2(0, 0);
                *pm = make_int2(0, 0);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * half; i += kFixedThreads) {
        const int yy = i / half, xx = 2 * (i - yy * half), j = yy * TS + xx;
        const float2 tr = *reinterpret_cast<const float2*>(&tre[j]);
        const float2 ti = *reinterpret_cast<const float2*>(&tim[j]);
        const int gy = y0 + yy, gx = x0 + xx;
        if (gy < a.W && gx < a.W &&
            NUASM_IN_RANGE(gy * (long long)a.Wp + gx + 1, (long long)a.W * a.Wp, dbg::kSpreadWindow))
            *reinterpret_cast<float4*>(&win[size_t(gy) * a.Wp + gx]) = make_float4(tr.x, ti.x, tr.y, ti.y);
    }
}

// Spreading into per-warp private copies of the tile, without atomics.  Each
// warp takes 32 consecutive records and adds their taps into its own T x T
// copy with plain loads and stores, one tap offset (qy, qx) at a time for all
// lanes, with a __syncwarp between offsets so that every store of one offset
// is seen by the loads of the next.  Within one offset two lanes touch the
// same cell only if their records share the first-tap cell; such a batch
// (found with __match_any_sync) adds with atomics instead.  The copies are
// summed at the end.  Shared memory: 8 warps x T^2 complex, so T <= 32 (F32)
// or T <= 16 (F64).
template <typename S, int WMAX, bool EXACT>
__global__ void __launch_bounds__(256, 2) spread_private_kernel(const typename RecOf<S>::type* __restrict__ rec,
                                                             const int* __restrict__ off,
                                                             const double* __restrict__ wpt,
                                                             const int* __restrict__ order,
                                                             const typename VecOf<S>::type* __restrict__ c,
                                                             typename VecOf<S>::type* __restrict__ win, GridArgs a,
                                                             const typename PolyOf<S>::type kp,
                                                             const int4* __restrict__ items) {
    using V = typename VecOf<S>::type;
    using Rec = typename RecOf<S>::type;
    extern __shared__ unsigned char smem_raw[];
    V* copies = reinterpret_cast<V*>(smem_raw);
    int tile, b, e, chunked = 0;
    if (items) {   // a chunk of a tile's records (several CTAs add into the tile)
        const int4 it = items[blockIdx.x];
        tile = it.x;
        b = it.y;
        e = it.z;
        chunked = it.w;
    } else {       // a whole tile, heaviest tiles first
        tile = order ? order[blockIdx.x] : blockIdx.x;
        b = off[tile];
        e = off[tile + 1];
    }
    const int T = a.T, w = EXACT ? WMAX : a.w, TS = plane_stride(T, a.skew_of(tile)), TT = T * TS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V* mine = copies + warp * TT;
    pdl_allow_next();
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    const V zero = CTraits<V>::zero();
    for (int i = threadIdx.x; i < 8 * TT; i += blockDim.x) copies[i] = zero;
    __syncthreads();
    for (int i0 = b + warp * 32; i0 < e; i0 += 256) {
        const int i = i0 + lane;
        const bool live = i < e && NUASM_IN_RANGE(i, a.nrec, dbg::kSpreadRec) &&
                          NUASM_IN_RANGE(rec[i].j, a.m, dbg::kSpreadValue);
        Rec r{};
        if (live) r = rec[i];
        // lanes whose records share a first-tap cell would add to one cell in the same step
        const uint32_t key = live ? r.cell : 0xffffffffu - uint32_t(lane);
        const bool clash = __any_sync(0xffffffffu, __popc(__match_any_sync(0xffffffffu, key)) > 1);
        const int lx = live ? int(r.cell & 0xffffu) - x0 : 0, ly = live ? int(r.cell >> 16) - y0 : 0;
        V val = zero;
        if (live) {
            val = c[r.j];
            if (wpt) { const S wt = S(wpt[r.j]); val.x *= wt; val.y *= wt; }
        }
        S wx[WMAX], wy[WMAX];
        tap_weights<WMAX>(S(r.fx), kp, wx);
        tap_weights<WMAX>(S(r.fy), kp, wy);
        const int ya = max(0, -ly), yb = min(w, T - ly);
        const int xa = max(0, -lx), xb = min(w, T - lx);
#pragma unroll(WMAX <= 16 ? WMAX : 1)
        for (int qy = 0; qy < WMAX; ++qy) {
            if (qy >= w) continue;   // warp-uniform
            const bool rowok = live && qy >= ya && qy < yb;
            const S vr = val.x * wy[qy], vi = val.y * wy[qy];
            V* row = mine + (ly + qy) * TS + lx;
#pragma unroll
            for (int qx = 0; qx < WMAX; ++qx) {
                if (qx >= w) continue;   // warp-uniform
                const bool ok = rowok && qx >= xa && qx < xb &&
                                (!rowok || NUASM_IN_RANGE((ly + qy) * TS + lx + qx, TT, dbg::kSpreadPlane));
                if (!clash) {
                    if (ok) {
                        V g = row[qx];
                        g.x += vr * wx[qx];
                        g.y += vi * wx[qx];
                        row[qx] = g;
                    }
                    __syncwarp();
                } else if (ok) {
                    atomicAdd(&row[qx].x, vr * wx[qx]);
                    atomicAdd(&row[qx].y, vi * wx[qx]);
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int yy = i / T, xx = i - yy * T;
        const int gy = y0 + yy, gx = x0 + xx;
        if (gy < a.W && gx < a.W && NUASM_IN_RANGE(gy * (long long)a.Wp + gx, (long long)a.W * a.Wp, dbg::kSpreadWindow)) {
            const int si = yy * TS + xx;
            V v = copies[si];
#pragma unroll
            for (int k = 1; k < 8; ++k) {
                const V u = copies[k * TT + si];
                v.x += u.x;
                v.y += u.y;
            }
            V* p = &win[size_t(gy) * a.Wp + gx];
            if (chunked) {   // the window was cleared; the tile's chunks add into it
                atomicAdd(&p->x, v.x);
                atomicAdd(&p->y, v.y);
            } else {
                *p = v;
            }
        }
    }
}

// --------------------------------------------------------------- interpolation (type 2)
// The tile plus its (w-1) halo is staged with a row stride = skew mod 16
// elements (halo_pitch), matching the record order's bank classes.
// The first kInterpPrefetch records of every thread are loaded before the
// staging loads so that their latency overlaps the tile's; FP32 tiles are
// staged two complex values (16 B) per cp.async copy, straight into shared
// memory (measured against loads through registers: NU-ASM_2 interpolation
// 32.0 -> 30.2 us, 4M clustered points 106.8 -> 96.6 us).
constexpr int kInterpThreads = 256, kInterpPrefetch = 4;
#ifndef NUASM_F64_EXACT13
#define NUASM_F64_EXACT13 1
#endif
#ifndef NUASM_INTERP_CPASYNC
#define NUASM_INTERP_CPASYNC 1   // FP32 tiles staged with cp.async (no register round trip)
#endif
#ifndef NUASM_INTERP_MINB
#define NUASM_INTERP_MINB 4   // CTAs per SM the register budget is sized for (64 registers)
#endif

template <typename S, int WMAX, bool EXACT, typename Rec, typename V>
__device__ __forceinline__ void interp_point(const Rec& r, const V* __restrict__ tl, int THP, int x0, int y0, int w,
                                             const typename PolyOf<S>::type& kp, V* __restrict__ v,
                                             [[maybe_unused]] int tl_n, [[maybe_unused]] long long m) {
    const int lx = int(r.cell & 0xffffu) - x0, ly = int(r.cell >> 16) - y0;
    S wx[WMAX], wy[WMAX];
    tap_weights<WMAX>(S(r.fx), kp, wx);
    tap_weights<WMAX>(S(r.fy), kp, wy);
    S ar = S(0), ai = S(0);
#pragma unroll(WMAX <= 16 ? WMAX : 1)
    for (int qy = 0; qy < WMAX; ++qy) {
        if (qy >= w) continue;
        const V* row = tl + (ly + qy) * THP + lx;
        S rr = S(0), ri = S(0);
#pragma unroll
        for (int qx = 0; qx < WMAX; ++qx) {
            if (qx >= w) continue;
            if (!NUASM_IN_RANGE((ly + qy) * THP + lx + qx, tl_n, dbg::kInterpTile)) continue;
            const V g = row[qx];
            rr = fma(g.x, wx[qx], rr);
            ri = fma(g.y, wx[qx], ri);
        }
        ar = fma(rr, wy[qy], ar);
        ai = fma(ri, wy[qy], ai);
    }
    V out;
    out.x = ar;
    out.y = ai;
    if (NUASM_IN_RANGE(r.j, m, dbg::kInterpOut)) v[r.j] = out;
}

template <typename S, int WMAX, bool EXACT>
__global__ void __launch_bounds__(kInterpThreads, sizeof(S) == 4 ? NUASM_INTERP_MINB : 2) interp_kernel(const typename RecOf<S>::type* __restrict__ rec,
                                                                const int* __restrict__ off,
                                                                const int* __restrict__ home,
                                                                const int* __restrict__ order,
                                                                const int4* __restrict__ items,
                                                                const typename VecOf<S>::type* __restrict__ win,
                                                                typename VecOf<S>::type* __restrict__ v, GridArgs a,
                                                                const typename PolyOf<S>::type kp) {
    using V = typename VecOf<S>::type;
    using Rec = typename RecOf<S>::type;
    extern __shared__ unsigned char smem_raw[];
    V* tl = reinterpret_cast<V*>(smem_raw);
    const int T = a.T, w = EXACT ? WMAX : a.w, TH = T + w - 1;
    int tile, b, e;
    if (items) {   // a chunk of a tile's home records
        const int4 it = items[blockIdx.x];
        tile = it.x;
        b = it.y;
        e = it.z;
    } else {       // a whole tile, heaviest tiles first
        tile = order ? order[blockIdx.x] : blockIdx.x;
        b = off[tile];
        e = b + home[tile];
    }
    const int THP = halo_pitch(TH, a.skew_of(tile));
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    pdl_allow_next();
    Rec pre[kInterpPrefetch];
#pragma unroll
    for (int k = 0; k < kInterpPrefetch; ++k) {
        const int i = b + threadIdx.x + k * kInterpThreads;
        if (i < e && NUASM_IN_RANGE(i, a.nrec, dbg::kInterpRec)) pre[k] = rec[i];
    }
    pdl_wait();   // the window comes from the previous kernel; the records are the plan's
    if constexpr (sizeof(V) == 8) {
        // pairs of complex64: x0 and the row pitch are even, so every pair is
        // 16-byte aligned, and W is even, so a pair never straddles the window edge
        const int HP = THP / 2;
        float4* tl4 = reinterpret_cast<float4*>(tl);
        for (int i = threadIdx.x; i < TH * HP; i += kInterpThreads) {
            const int yy = i / HP, u = i - yy * HP;
            const int gy = y0 + yy, gx = x0 + 2 * u;
#if NUASM_INTERP_CPASYNC
            if (2 * u < TH && gy < a.W && gx < a.W) cp_async16(&tl4[i], &win[size_t(gy) * a.Wp + gx]);
            else tl4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#else
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (2 * u < TH && gy < a.W && gx < a.W)
                val = *reinterpret_cast<const float4*>(&win[size_t(gy) * a.Wp + gx]);
            tl4[i] = val;
#endif
        }
#if NUASM_INTERP_CPASYNC
        cp_async_commit();
        cp_async_wait_all();
#endif
    } else {
        for (int i = threadIdx.x; i < TH * THP; i += kInterpThreads) {
            const int yy = i / THP, xx = i - yy * THP;
            const int gy = y0 + yy, gx = x0 + xx;
            V val;
            val.x = S(0);
            val.y = S(0);
            if (xx < TH && gy < a.W && gx < a.W) val = win[size_t(gy) * a.Wp + gx];
            tl[i] = val;
        }
    }
    __syncthreads();
    // a ring of kInterpPrefetch records in flight: each slot is refilled with
    // the record kInterpPrefetch strides ahead before its point is computed
    constexpr int AHEAD = kInterpPrefetch * kInterpThreads;
    for (int base = b + threadIdx.x; base < e; base += AHEAD) {
#pragma unroll
        for (int k = 0; k < kInterpPrefetch; ++k) {
            const int i = base + k * kInterpThreads;
            if (i < e) {
                const Rec r = pre[k];
                if (i + AHEAD < e && NUASM_IN_RANGE(i + AHEAD, a.nrec, dbg::kInterpRec)) pre[k] = rec[i + AHEAD];
                interp_point<S, WMAX, EXACT>(r, tl, THP, x0, y0, w, kp, v, TH * THP, a.m);
            }
        }
    }
}

// ---------------------------------------------------------------- FP64 mode in double-float arithmetic
// FP64-mode gridding with the ES kernel at its exact widths (see
// gridding_double_float) runs on the FP32 pipe, whose rate is 64 times that
// of the FP64 pipe here: window values and tap weights are unevaluated sums
// hi + lo of two floats (47 significant bits), products go through FMA-based
// error-free transforms, and FP64 arithmetic is left to once per point or
// per staged cell.

// x 2^-s as hi + lo (dfr_split: integer operations on the bits, relative
// error below 2^-46; subnormals rescaled exactly first).  The caller picks s
// so that the result is below 2 in magnitude.
__device__ __forceinline__ df df_split(double x, int s) {
    const dfr r = dfr_split(x, s);
    return {r.hi, r.lo};
}

// exponent k of a double with 2^k <= |x| < 2^(k+1) (-1023 for zeros and
// subnormals, 1024 for infinities and NaNs)
__device__ __forceinline__ int dexp(double x) {
    return (int(static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff) - 1023;
}

// a b + c; the sum is kept as hi + lo without renormalisation (lo collects
// the rounding errors of the products and of the hi sums exactly or to 2^-24
// of its own size)
__device__ __forceinline__ df df_fma(df a, df b, df c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const df t = df_two_sum(p, c.hi);
    return {t.hi, t.lo + (e + c.lo)};
}

// Tap weights of one axis in double-float: Horner's rule on the FP64
// polynomials, the degrees from kDfTail up in FP32 (the coefficients' hi
// parts; their sum is below 3.1e-7 for the ES kernel at w = 11 and 13 and
// 1.1e-7 for the Gaussian at w = 15, 21 and 25, so this adds below 2e-14 to
// a weight) and the rest in double-float.
constexpr int kDfTail = 9;
static_assert(kPoly64Deg >= kDfTail, "FP64 tap degree");
// c: the kPoly64Deg + 1 coefficients of one tap (parameter or shared memory)
__device__ __forceinline__ df tap_weight_df(const float2* c, df x) {
    float t = c[kPoly64Deg].x;
#pragma unroll
    for (int k = kPoly64Deg - 1; k >= kDfTail; --k) t = fmaf(t, x.hi, c[k].x);
    df acc = {t, 0.f};
#pragma unroll
    for (int k = kDfTail - 1; k >= 0; --k) acc = df_fma(acc, x, df{c[k].x, c[k].y});
    return df_two_sum(acc.hi, acc.lo);
}
constexpr int kDfCoef = kPoly64Deg + 1;

// x weights from the parameter copy of the coefficients (unrolled), y
// weights one row at a time from the CTA's shared copy cs (rolled row loop)
template <int WMAX>
__device__ __forceinline__ void interp_point_df(const RecD& r, const float4* __restrict__ tl, int THP, int x0, int y0,
                                                const KernelPolyDF& kp, const float2* cs, double scale,
                                                double2* __restrict__ v, [[maybe_unused]] int tl_n,
                                                [[maybe_unused]] long long m) {
    const int lx = int(r.cell & 0xffffu) - x0, ly = int(r.cell >> 16) - y0;
    df wx[WMAX];
    const df xv = df_split(fma(2.0, r.fx, -1.0), 0), yv = df_split(fma(2.0, r.fy, -1.0), 0);
#pragma unroll
    for (int q = 0; q < WMAX; ++q) wx[q] = tap_weight_df(kp.c[q], xv);
    df ar = {0.f, 0.f}, ai = {0.f, 0.f};
#pragma unroll 1
    for (int qy = 0; qy < WMAX; ++qy) {
        const df wyq = tap_weight_df(cs + qy * kDfCoef, yv);
        const float4* row = tl + (ly + qy) * THP + lx;
        df rr = {0.f, 0.f}, ri = {0.f, 0.f};
#pragma unroll
        for (int qx = 0; qx < WMAX; ++qx) {
            if (!NUASM_IN_RANGE((ly + qy) * THP + lx + qx, tl_n, dbg::kInterpTile)) continue;
            const float4 g = row[qx];
            rr = df_fma(df{g.x, g.y}, wx[qx], rr);
            ri = df_fma(df{g.z, g.w}, wx[qx], ri);
        }
        ar = df_fma(df_two_sum(rr.hi, rr.lo), wyq, ar);
        ai = df_fma(df_two_sum(ri.hi, ri.lo), wyq, ai);
    }
    const double2 out = make_double2((double(ar.hi) + double(ar.lo)) * scale, (double(ai.hi) + double(ai.lo)) * scale);
    if (NUASM_IN_RANGE(r.j, m, dbg::kInterpOut)) v[r.j] = out;
}

// FP64-mode spreading in double-float arithmetic with exact integer sums,
// one CTA per whole tile or per chunk of a split tile.  Records go in
// batches of kDfBatch; a batch's values are scaled by 2^-E, S = sum(|re| +
// |im|) < 2^E over the batch (weights included), so every scaled tap
// contribution p = v wy wx is at most 1 and a batch adds at most 1 at any
// cell.  p is split into n_h 2^-30 + n_l 2^-52 + (|error| <= 2^-53 + 2^-55)
// with |n_l| <= 2^21 + 32, and n_h, n_l go to two int32 planes per component with
// shared-memory integer atomics: a batch's sums stay below 2^31 at every
// cell and are exact.  After each batch the planes become the integer V =
// n_h 2^22 + n_l (units 2^(E-52)); a tile with one batch writes V 2^(E-52)
// as FP64, one with several adds V into int64 totals held in its own window
// cells at the unit 2^(Et-62), Et from the tile's whole sum (a first pass
// over its records), and converts them to FP64 at the end; a chunk adds each
// batch's V 2^(E-52) into the cleared window with FP64 atomics.  A batch whose
// sum is not finite makes the tile's cells NaN (so do the FFTs of any
// window with such a cell).
constexpr int kDfBatch = 512;
#ifndef NUASM_DF_SPLIT
#define NUASM_DF_SPLIT 1   // 0: split tiles keep the FP64 spreading kernels
#endif
#ifndef NUASM_DF_SPREAD_MINB
// CTAs per SM the register budget of spread_df_kernel is set for (4M
// clustered FP64 points: 3.04 ms at 2, 2.85 ms at 3)
#define NUASM_DF_SPREAD_MINB 3
#endif
// a b without renormalisation (the low part is the product's exact error
// plus the cross terms)
__device__ __forceinline__ df df_prod(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return {p, e};
}
// n_h, n_l of p (|p| < 1) by round-to-nearest additions of "magic" constants
// on the FP32 pipe instead of conversion instructions (whose pipe runs at a
// quarter of the FP32 rate): t = p.hi 2^30 is rounded to a multiple of 256 by
// adding 3 2^30 (the sum lies in [2^31, 2^32), whose float spacing is 256),
// the exact remainder plus p.lo 2^30 (|.| <= 192) to an integer by adding
// 1.5 2^23 (spacing 1), and what is left (|.| <= 1/2 + 2^-17), times 2^22,
// likewise; a sum's bits minus the constant's bits are the rounded value in
// units of the spacing.
__device__ __forceinline__ void df_quant_add(df p, int cell, int* ph, int* pl) {
    constexpr float M1 = 3221225472.f, M2 = 12582912.f;   // 3 2^30, 1.5 2^23
    const float t = p.hi * 1073741824.f;                    // 2^30: exact; |t| < 2^30
    const float tl = p.lo * 1073741824.f;                   // |tl| < 2^6
    const float s1 = t + M1;
    const float r1 = t - (s1 - M1);                         // exact, |r1| <= 128
    const float s2 = (r1 + tl) + M2;
    const float d = (r1 - (s2 - M2)) + tl;                  // r1 - (s2 - M2) exact; |d| <= 1/2 + 2^-17
    const float s3 = fmaf(d, 4194304.f, M2);                // d 2^22 rounded (|d 2^22| <= 2^21 + 32)
    const int nh = ((__float_as_int(s1) - __float_as_int(M1)) << 8) + (__float_as_int(s2) - __float_as_int(M2));
    const int nl = __float_as_int(s3) - __float_as_int(M2);
    atomicAdd(&ph[cell], nh);
    atomicAdd(&pl[cell], nl);
}
// 2^k as a double for k in [-1022, 1023]
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double(static_cast<long long>(k + 1023) << 52); }
// V 2^k for an integer |V| < 2^62 (two exact power-of-two factors when k is below the normal range)
__device__ __forceinline__ double scaled_int(long long V, int k) {
    const double v = double(V);
    return k >= -1022 ? v * pow2d(k) : (v * pow2d(k + 512)) * pow2d(-512);
}

template <int WMAX>
__global__ void __launch_bounds__(256, WMAX <= 13 ? NUASM_DF_SPREAD_MINB : 2) spread_df_kernel(const RecD* __restrict__ rec, const int* __restrict__ off,
                                                          const double* __restrict__ wpt,
                                                          const int* __restrict__ order,
                                                          const double2* __restrict__ c, double2* __restrict__ win,
                                                          GridArgs a, const KernelPolyDF kp,
                                                          const int4* __restrict__ items) {
    constexpr int NT = 256, RPB = kDfBatch / NT;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float2 cs[WMAX * kDfCoef];
    __shared__ double red[NT / 32];
    __shared__ double bsum;
    int tile, b, e;
    bool chunked = false;
    if (items) {   // a chunk of a tile's records: several CTAs add into the tile (window cleared)
        const int4 it = items[blockIdx.x];
        tile = it.x;
        b = it.y;
        e = it.z;
        chunked = it.w != 0;
    } else {       // a whole tile, heaviest tiles first
        tile = order ? order[blockIdx.x] : blockIdx.x;
        b = off[tile];
        e = off[tile + 1];
    }
    const int T = a.T, TS = plane_stride(T, a.skew_of(tile)), TT = T * TS;
    int* rh = reinterpret_cast<int*>(smem_raw);
    int* rl = rh + TT;
    int* ih = rl + TT;
    int* il = ih + TT;
    pdl_allow_next();
    for (int i = threadIdx.x; i < WMAX * kDfCoef; i += NT) cs[i] = kp.c[i / kDfCoef][i % kDfCoef];
    for (int i = threadIdx.x; i < TT; i += NT) {
        rh[i] = 0;
        rl[i] = 0;
        ih[i] = 0;
        il[i] = 0;
    }
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool multi = !chunked && e - b > kDfBatch;   // int64 totals in the tile's own cells
    // block sum of one double per thread
    auto block_sum = [&](double part) -> double {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < NT / 32; ++k) t += red[k];
            bsum = t;
        }
        __syncthreads();
        return bsum;
    };
    auto value_of = [&](int i) -> double2 {
        const RecD r = rec[i];
        const int j = NUASM_IN_RANGE(r.j, a.m, dbg::kSpreadValue) ? r.j : 0;
        double2 v = c[j];
        if (wpt) {
            const double wt = wpt[j];
            v.x *= wt;
            v.y *= wt;
        }
        return v;
    };
    pdl_wait();   // c may come from the previous kernel
    int Et = 0;   // the tile's unit exponent for int64 totals (several batches)
    if (multi) {
        double part = 0.0;
        for (int i = b + threadIdx.x; i < e; i += NT) {
            if (!NUASM_IN_RANGE(i, a.nrec, dbg::kSpreadRec)) continue;
            const double2 v = value_of(i);
            part += fabs(v.x) + fabs(v.y);
        }
        const double St = block_sum(part);
        Et = dexp(St) + 2;   // St < 2^(Et - 1): the totals stay below 2^61 units
    }
    bool started = false, nonfinite = false;
    for (int i0 = b; i0 < e; i0 += kDfBatch) {
        RecD r[RPB];
        double2 val[RPB];
        double part = 0.0;
#pragma unroll
        for (int k = 0; k < RPB; ++k) {
            const int i = i0 + threadIdx.x + k * NT;
            val[k] = make_double2(0.0, 0.0);
            r[k].cell = 0;
            if (i < e && NUASM_IN_RANGE(i, a.nrec, dbg::kSpreadRec)) {
                r[k] = rec[i];
                val[k] = value_of(i);
                part += fabs(val[k].x) + fabs(val[k].y);
            }
        }
        __syncthreads();   // the previous batch's fold is done before the sum reuses red
        const double S = block_sum(part);
        if (S == 0.0) continue;
        if (!(S <= 1.7976931348623157e308)) {   // infinity or NaN among the values
            nonfinite = true;
            break;
        }
        const int Eb = dexp(S) + 1;   // S < 2^Eb
#pragma unroll
        for (int k = 0; k < RPB; ++k) {
            const int i = i0 + threadIdx.x + k * NT;
            if (i >= e) continue;
            const int lx = int(r[k].cell & 0xffffu) - x0, ly = int(r[k].cell >> 16) - y0;
            const df vr = df_split(val[k].x, Eb), vi = df_split(val[k].y, Eb);
            const df xv = df_split(fma(2.0, r[k].fx, -1.0), 0), yv = df_split(fma(2.0, r[k].fy, -1.0), 0);
            df wx[WMAX];
#pragma unroll
            for (int q = 0; q < WMAX; ++q) wx[q] = tap_weight_df(kp.c[q], xv);
            const int ya = max(0, -ly), yb = min(WMAX, T - ly);
            const int xa = max(0, -lx), xb = min(WMAX, T - lx);
#pragma unroll 1
            for (int qy = ya; qy < yb; ++qy) {
                const df wyq = tap_weight_df(cs + qy * kDfCoef, yv);
                const df pr = df_mul(vr, wyq), pi = df_mul(vi, wyq);
                const int rowi = (ly + qy) * TS + lx;
#pragma unroll
                for (int qx = 0; qx < WMAX; ++qx) {
                    if (qx < xa || qx >= xb) continue;
                    const int cell = rowi + qx;
                    if (!NUASM_IN_RANGE(cell, TT, dbg::kSpreadPlane)) continue;
                    df_quant_add(df_prod(pr, wx[qx]), cell, rh, rl);
                    df_quant_add(df_prod(pi, wx[qx]), cell, ih, il);
                }
            }
        }
        __syncthreads();
        // fold: V = n_h 2^22 + n_l per component, then clear the planes
        const int sh = Eb - Et + 10;   // units 2^(Eb - 52) to units 2^(Et - 62)
        for (int i = threadIdx.x; i < T * T; i += NT) {
            const int yy = i / T, xx = i - yy * T, j = yy * TS + xx;
            const long long Vr = (static_cast<long long>(rh[j]) << 22) + rl[j];
            const long long Vi = (static_cast<long long>(ih[j]) << 22) + il[j];
            rh[j] = 0;
            rl[j] = 0;
            ih[j] = 0;
            il[j] = 0;
            const int gy = y0 + yy, gx = x0 + xx;
            if (gy >= a.W || gx >= a.W ||
                !NUASM_IN_RANGE(gy * (long long)a.Wp + gx, (long long)a.W * a.Wp, dbg::kSpreadWindow))
                continue;
            double2* p = &win[size_t(gy) * a.Wp + gx];
            if (chunked) {   // FP64 atomic adds of this batch's exact sums
                if (Vr) atomicAdd(&p->x, scaled_int(Vr, Eb - 52));
                if (Vi) atomicAdd(&p->y, scaled_int(Vi, Eb - 52));
            } else if (!multi) {
                *p = make_double2(scaled_int(Vr, Eb - 52), scaled_int(Vi, Eb - 52));
            } else {
                long long* q = reinterpret_cast<long long*>(p);
                auto to_tot = [&](long long V) -> long long {
                    return sh >= 0 ? V * (1LL << min(sh, 62)) : (V + (1LL << (min(-sh, 62) - 1))) >> min(-sh, 62);
                };
                const long long tr = to_tot(Vr), ti = to_tot(Vi);
                if (started) {
                    q[0] += tr;
                    q[1] += ti;
                } else {
                    q[0] = tr;
                    q[1] = ti;
                }
            }
        }
        started = true;
    }
    __syncthreads();
    // cells the batches did not write: NaN (non-finite values), FP64 from the
    // int64 totals, or zero (a chunk leaves the cleared window to the others)
    if (nonfinite || multi || (!started && !chunked)) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        for (int i = threadIdx.x; i < T * T; i += NT) {
            const int yy = i / T, xx = i - yy * T;
            const int gy = y0 + yy, gx = x0 + xx;
            if (gy >= a.W || gx >= a.W ||
                !NUASM_IN_RANGE(gy * (long long)a.Wp + gx, (long long)a.W * a.Wp, dbg::kSpreadWindow))
                continue;
            double2* p = &win[size_t(gy) * a.Wp + gx];
            if (nonfinite) {
                *p = make_double2(nan, nan);
            } else if (started) {   // several batches
                const longlong2 t = *reinterpret_cast<const longlong2*>(p);
                *p = make_double2(scaled_int(t.x, Et - 62), scaled_int(t.y, Et - 62));
            } else {
                *p = make_double2(0.0, 0.0);
            }
        }
    }
}

// FP64-mode interpolation in double-float arithmetic: the interp_kernel
// schedule (one CTA per tile or chunk, a ring of prefetched records); the
// tile is staged in FP64, scaled by 2^-s, s the largest exponent among its
// values (so no value leaves the float range), and split in place into
// (re.hi, re.lo, im.hi, im.lo) cells of the same 16 bytes.
template <int WMAX>
__global__ void __launch_bounds__(kInterpThreads, 2) interp_df_kernel(const RecD* __restrict__ rec,
                                                                      const int* __restrict__ off,
                                                                      const int* __restrict__ home,
                                                                      const int* __restrict__ order,
                                                                      const int4* __restrict__ items,
                                                                      const double2* __restrict__ win,
                                                                      double2* __restrict__ v, GridArgs a,
                                                                      const KernelPolyDF kp) {
    extern __shared__ unsigned char smem_raw[];
    double2* tld = reinterpret_cast<double2*>(smem_raw);
    float4* tl = reinterpret_cast<float4*>(smem_raw);
    __shared__ int emax;
    __shared__ float2 cs[WMAX * kDfCoef];
    for (int i = threadIdx.x; i < WMAX * kDfCoef; i += kInterpThreads) cs[i] = kp.c[i / kDfCoef][i % kDfCoef];
    const int T = a.T, TH = T + WMAX - 1;
    int tile, b, e;
    if (items) {
        const int4 it = items[blockIdx.x];
        tile = it.x;
        b = it.y;
        e = it.z;
    } else {
        tile = order ? order[blockIdx.x] : blockIdx.x;
        b = off[tile];
        e = b + home[tile];
    }
    const int THP = halo_pitch(TH, a.skew_of(tile));
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    const int x0 = tx * T, y0 = ty * T;
    pdl_allow_next();
    RecD pre[kInterpPrefetch];
#pragma unroll
    for (int k = 0; k < kInterpPrefetch; ++k) {
        const int i = b + threadIdx.x + k * kInterpThreads;
        if (i < e && NUASM_IN_RANGE(i, a.nrec, dbg::kInterpRec)) pre[k] = rec[i];
    }
    if (threadIdx.x == 0) emax = -1023;
    pdl_wait();   // the window comes from the previous kernel
    __syncthreads();
    int em = -1023;
    for (int i = threadIdx.x; i < TH * THP; i += kInterpThreads) {
        const int yy = i / THP, xx = i - yy * THP;
        const int gy = y0 + yy, gx = x0 + xx;
        double2 val = make_double2(0.0, 0.0);
        if (xx < TH && gy < a.W && gx < a.W) val = win[size_t(gy) * a.Wp + gx];
        tld[i] = val;
        em = max(em, max(dexp(val.x), dexp(val.y)));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if ((threadIdx.x & 31) == 0) atomicMax(&emax, em);
    __syncthreads();
    const int sc = min(max(emax, -1022), 1023);
    for (int i = threadIdx.x; i < TH * THP; i += kInterpThreads) {   // each thread splits the cells it staged
        const double2 val = tld[i];
        const df re = df_split(val.x, sc), im = df_split(val.y, sc);
        tl[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const double scale = __longlong_as_double(static_cast<long long>(sc + 1023) << 52);   // 2^sc
    constexpr int AHEAD = kInterpPrefetch * kInterpThreads;
    for (int base = b + threadIdx.x; base < e; base += AHEAD) {
#pragma unroll
        for (int k = 0; k < kInterpPrefetch; ++k) {
            const int i = base + k * kInterpThreads;
            if (i < e) {
                const RecD r = pre[k];
                if (i + AHEAD < e && NUASM_IN_RANGE(i + AHEAD, a.nrec, dbg::kInterpRec)) pre[k] = rec[i + AHEAD];
                interp_point_df<WMAX>(r, tl, THP, x0, y0, kp, cs, scale, v, TH * THP, a.m);
            }
        }
    }
}

// whether the plan's spreading runs spread_private_kernel or spread_kernel,
// which take work items (spread_fixed_kernel keeps one CTA per tile)
bool spread_by_items(const nuasm_plan_s* P) {
    if (NUASM_SPREAD_PRIVATE && P->g.T <= (P->f64 ? 16 : 32)) return true;
    return P->f64 || !NUASM_SPREAD_FIXED;
}

GridArgs grid_args(const nuasm_plan_s* P) {
    GridArgs a;
    a.W = P->g.W;
    a.Wp = P->g.Wp;
    a.T = P->g.T;
    a.ntx = P->g.ntx;
    a.w = P->g.w;
    a.skew = P->skew;
    a.tskew = P->d.tile_skew;
    a.max_skew = P->d.tile_skew ? kMaxSkew : P->skew;
    a.m = P->m;
    a.nrec = P->nrec > 0 ? P->nrec : 4 * P->m;   // unknown on the host (no-allocation path): the capacity
    return a;
}

template <typename K> cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// the tap polynomials of the plan's precision
template <typename S> typename PolyOf<S>::type taps_arg(const nuasm_plan_s* P) {
    if constexpr (sizeof(S) == 8) return P->poly64;
    else return P->poly;
}

template <typename S, int WMAX, bool EXACT>
cudaError_t spread_impl(const nuasm_plan_s* P, const void* c, cudaStream_t st) {
    using V = typename VecOf<S>::type;
    GridArgs a = grid_args(P);
    // chunked tiles add into a cleared window
    const int4* items = P->d.spread_items;
    const int grid = items ? P->n_spread_items : P->g.ntiles;
    auto clear = [&]() -> cudaError_t {
        return items ? cudaMemsetAsync(P->d.win, 0, ws_win_elems(P->g) * sizeof(V), st) : cudaSuccess;
    };
    {
        cudaError_t e = clear();
        if (e != cudaSuccess) return e;
    }
    if (NUASM_SPREAD_PRIVATE && a.T <= (sizeof(S) == 4 ? 32 : 16)) {
        const size_t sm = size_t(8) * a.T * plane_stride(a.T, a.max_skew) * sizeof(V);
        cudaError_t e = set_smem(spread_private_kernel<S, WMAX, EXACT>, sm);
        if (e != cudaSuccess) return e;
        spread_private_kernel<S, WMAX, EXACT><<<grid, 256, sm, st>>>(
            static_cast<const typename RecOf<S>::type*>(P->d.rec), P->d.tile_off, P->d.wpt, P->d.tile_order,
            static_cast<const V*>(c), static_cast<V*>(P->d.win), a, taps_arg<S>(P), items);
        return cudaGetLastError();
    }
    if constexpr (sizeof(S) == 4) {
        if (NUASM_SPREAD_FIXED) {
            constexpr int RPB = NUASM_SPREAD_FIXED_RPB;
            const size_t sm = size_t(4) * a.T * plane_stride(a.T, a.max_skew) * sizeof(float);
            cudaError_t e = set_smem(spread_fixed_kernel<WMAX, EXACT, RPB>, sm);
            if (e != cudaSuccess) return e;
            spread_fixed_kernel<WMAX, EXACT, RPB><<<P->g.ntiles, kFixedThreads, sm, st>>>(
                static_cast<const RecF*>(P->d.rec), P->d.tile_off, P->d.wpt, P->d.tile_order,
                static_cast<const float2*>(c), static_cast<float2*>(P->d.win), a, taps_arg<S>(P));
            return cudaGetLastError();
        }
    }
    const size_t sm = size_t(2) * a.T * plane_stride(a.T, a.max_skew) * sizeof(S);
    cudaError_t e = set_smem(spread_kernel<S, WMAX, EXACT>, sm);
    if (e != cudaSuccess) return e;
    spread_kernel<S, WMAX, EXACT><<<grid, 256, sm, st>>>(
        static_cast<const typename RecOf<S>::type*>(P->d.rec), P->d.tile_off, P->d.wpt, P->d.tile_order,
        static_cast<const V*>(c), static_cast<V*>(P->d.win), a, taps_arg<S>(P), items);
    return cudaGetLastError();
}

template <typename S, int WMAX, bool EXACT>
cudaError_t interp_impl(const nuasm_plan_s* P, void* v, cudaStream_t st) {
    using V = typename VecOf<S>::type;
    GridArgs a = grid_args(P);
    int THP = 0;   // the largest staged row pitch over the skews in use
    for (int k = 0; k <= a.max_skew; k += 2) THP = std::max(THP, halo_pitch(a.T + a.w - 1, k));
    if (!a.tskew) THP = halo_pitch(a.T + a.w - 1, a.skew);
    const int TH = a.T + a.w - 1;
    const size_t sm = size_t(TH) * THP * sizeof(V);
    cudaError_t e = set_smem(interp_kernel<S, WMAX, EXACT>, sm);
    if (e != cudaSuccess) return e;
    const int grid = P->d.interp_items ? P->n_interp_items : P->g.ntiles;
    e = launch_chained(interp_kernel<S, WMAX, EXACT>, dim3(grid), dim3(kInterpThreads), sm, st,
                       static_cast<const typename RecOf<S>::type*>(P->d.rec), P->d.tile_off, P->d.tile_home,
                       P->d.tile_order, static_cast<const int4*>(P->d.interp_items), static_cast<const V*>(P->d.win),
                       static_cast<V*>(v), a, taps_arg<S>(P));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int WMAX> cudaError_t spread_df_impl(const nuasm_plan_s* P, const void* c, cudaStream_t st) {
    GridArgs a = grid_args(P);
    const int4* items = P->d.spread_items;   // chunks of split tiles add into a cleared window
    cudaError_t e = items ? cudaMemsetAsync(P->d.win, 0, ws_win_elems(P->g) * sizeof(double2), st) : cudaSuccess;
    if (e != cudaSuccess) return e;
    const size_t sm = size_t(4) * a.T * plane_stride(a.T, a.max_skew) * sizeof(int);
    if ((e = set_smem(spread_df_kernel<WMAX>, sm)) != cudaSuccess) return e;
    const int grid = items ? P->n_spread_items : P->g.ntiles;
    spread_df_kernel<WMAX><<<grid, 256, sm, st>>>(static_cast<const RecD*>(P->d.rec), P->d.tile_off, P->d.wpt,
                                                  P->d.tile_order, static_cast<const double2*>(c),
                                                  static_cast<double2*>(P->d.win), a, P->poly64df, items);
    return cudaGetLastError();
}

template <int WMAX> cudaError_t interp_df_impl(const nuasm_plan_s* P, void* v, cudaStream_t st) {
    GridArgs a = grid_args(P);
    const int TH = a.T + WMAX - 1;
    int THP = 0;   // the largest staged row pitch over the skews in use
    for (int k = 0; k <= a.max_skew; k += 2) THP = std::max(THP, halo_pitch(TH, k));
    if (!a.tskew) THP = halo_pitch(TH, a.skew);
    const size_t sm = size_t(TH) * THP * sizeof(double2);
    cudaError_t e = set_smem(interp_df_kernel<WMAX>, sm);
    if (e != cudaSuccess) return e;
    const int grid = P->d.interp_items ? P->n_interp_items : P->g.ntiles;
    e = launch_chained(interp_df_kernel<WMAX>, dim3(grid), dim3(kInterpThreads), sm, st,
                       static_cast<const RecD*>(P->d.rec), P->d.tile_off, P->d.tile_home, P->d.tile_order,
                       static_cast<const int4*>(P->d.interp_items), static_cast<const double2*>(P->d.win),
                       static_cast<double2*>(v), a, P->poly64df);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename S_, int W_, bool X_> struct GTag {
    using S = S_;
    static constexpr int W = W_;
    static constexpr bool X = X_;
};

// width dispatch: exact instantiations for the common FP32 widths
template <bool SPREAD> cudaError_t gridding(const nuasm_plan_s* P, const void* in, void* out, cudaStream_t st) {
    auto run = [&](auto tag) -> cudaError_t {
        using Tg = decltype(tag);
        if constexpr (SPREAD) return spread_impl<typename Tg::S, Tg::W, Tg::X>(P, in, st);
        else return interp_impl<typename Tg::S, Tg::W, Tg::X>(P, out, st);
    };
    if (P->f64) {
        // double-float gridding at the kernel widths of the FP64 tolerances
        // (gridding_double_float); split tiles too unless NUASM_DF_SPLIT is 0
        if (gridding_double_float(P)) {
            auto df_run = [&](auto wtag) -> cudaError_t {
                constexpr int WD = decltype(wtag)::value;
                if constexpr (SPREAD) return spread_df_impl<WD>(P, in, st);
                else return interp_df_impl<WD>(P, out, st);
            };
            if (!SPREAD || NUASM_DF_SPLIT || !P->d.spread_items) {
                switch (P->g.w) {
                    case 11: return df_run(std::integral_constant<int, 11>{});
                    case 13: return df_run(std::integral_constant<int, 13>{});
                    case 15: return df_run(std::integral_constant<int, 15>{});
                    case 21: return df_run(std::integral_constant<int, 21>{});
                    default: return df_run(std::integral_constant<int, 25>{});
                }
            }
        }
        // the FP64 default tolerance (1e-12) gives w = 13 and a tolerance of
        // 1e-10 w = 11: exact instantiations
#if NUASM_F64_EXACT13
        if (P->g.w == 13) return run(GTag<double, 13, true>{});
        if (P->g.w == 11) return run(GTag<double, 11, true>{});
#endif
        if (P->g.w <= 8) return run(GTag<double, 8, false>{});
        return P->g.w <= 16 ? run(GTag<double, 16, false>{}) : run(GTag<double, kPolyMaxW, false>{});
    }
    switch (P->g.w) {
        case 4: return run(GTag<float, 4, true>{});
        case 5: return run(GTag<float, 5, true>{});
        case 6: return run(GTag<float, 6, true>{});
        case 7: return run(GTag<float, 7, true>{});
        case 8: return run(GTag<float, 8, true>{});
        default: return P->g.w <= 16 ? run(GTag<float, 16, false>{}) : run(GTag<float, kPolyMaxW, false>{});
    }
}

}  // namespace

static nuasm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return NUASM_OK;
    return e == cudaErrorMemoryAllocation ? NUASM_ENOMEM : NUASM_ECUDA;
}

// Tiles in decreasing record count (ties by index): the launch order of the
// one-CTA-per-tile kernels, so the heaviest tiles start first and the last
// wave holds the lightest.
//
// Interpolation items: a tile with more than the plan's interp_chunk home
// records (NUASM_INTERP_CHUNK where the plan leaves it 0) is split into
// chunks of at most that many, each its own CTA (which stages the same tile),
// so that the densest tiles do not hold the last wave; items are launched
// heaviest first.  0 keeps one item per tile.
#ifndef NUASM_INTERP_CHUNK
#define NUASM_INTERP_CHUNK 0
#endif
// smallest spreading chunk (records) of a split tile, by precision
#ifndef NUASM_SPREAD_CHUNK64
#define NUASM_SPREAD_CHUNK64 128
#endif
#ifndef NUASM_SPREAD_CHUNK32
#define NUASM_SPREAD_CHUNK32 512
#endif
constexpr int64_t kSpreadChunk64 = NUASM_SPREAD_CHUNK64, kSpreadChunk32 = NUASM_SPREAD_CHUNK32;
cudaError_t make_tile_order(nuasm_plan_s* P, cudaStream_t st) {
    const int nt = P->g.ntiles;
    std::vector<int> off(size_t(nt) + 1), home(nt), order(nt);
    cudaError_t e = cudaMemcpyAsync(off.data(), P->d.tile_off, sizeof(int) * (size_t(nt) + 1),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(home.data(), P->d.tile_home, sizeof(int) * size_t(nt), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    if ((e = xmalloc(reinterpret_cast<void**>(&P->d.tile_order), sizeof(int) * size_t(nt))) != cudaSuccess) return e;
    P->device_bytes += int64_t(sizeof(int)) * nt;
    e = cudaMemcpyAsync(P->d.tile_order, order.data(), sizeof(int) * size_t(nt), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return e;   // host vectors go out of scope
    if (spread_by_items(P) && P->nrec > 0 && P->p.spread_chunk >= 0) {
        // Spreading items: a tile whose records would keep one SM busy well past
        // the rest (more than K, K the larger of a per-precision floor and the
        // records of an even share over two CTAs per SM) is split into chunks of
        // at most K records, each its own CTA adding into the window; no split,
        // no items.
        const int64_t floor_k = P->f64 ? kSpreadChunk64 : kSpreadChunk32;
        const int64_t k = P->p.spread_chunk > 0 ? int64_t(P->p.spread_chunk)
                                                : std::max<int64_t>(floor_k, (P->nrec + 2 * 152 - 1) / (2 * 152));
        bool split = false;
        for (int t = 0; t < nt && !split; ++t) split = off[t + 1] - off[t] > k;
        if (split) {
            std::vector<int4> items;
            items.reserve(size_t(nt) + size_t(P->nrec / k) + 1);
            for (int t : order) {
                const int b = off[t], e2 = off[t + 1], n = e2 - b;
                if (n <= k) {
                    items.push_back(make_int4(t, b, e2, 0));
                    continue;
                }
                const int pieces = int((n + k - 1) / k), step = (n + pieces - 1) / pieces;
                for (int s0 = b; s0 < e2; s0 += step) items.push_back(make_int4(t, s0, std::min(e2, s0 + step), 1));
            }
            std::stable_sort(items.begin(), items.end(),
                             [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
            if ((e = xmalloc(reinterpret_cast<void**>(&P->d.spread_items), sizeof(int4) * items.size())) !=
                cudaSuccess)
                return e;
            P->device_bytes += int64_t(sizeof(int4) * items.size());
            P->n_spread_items = int(items.size());
            e = cudaMemcpyAsync(P->d.spread_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                st);
            if (e != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        }
    }
    const int ich = P->p.interp_chunk > 0 ? P->p.interp_chunk : NUASM_INTERP_CHUNK;
    if (ich > 0) {
        const int ch = ich;
        std::vector<int4> items;
        items.reserve(size_t(nt) + size_t(P->m / ch) + 1);
        for (int t = 0; t < nt; ++t) {
            const int b = off[t], e2 = off[t] + home[t];
            if (b == e2) continue;   // no home records: nothing to interpolate
            // chunks start on a multiple of 32 records from the tile start: the record order's
            // bank classes repeat every 32 records, so each warp keeps its distinct classes
            const int pieces = (e2 - b + ch - 1) / ch, step = (((e2 - b + pieces - 1) / pieces) + 31) & ~31;
            for (int s = b; s < e2; s += step) items.push_back(make_int4(t, s, std::min(e2, s + step), 0));
        }
        std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
        if (items.empty()) return cudaSuccess;
        if ((e = xmalloc(reinterpret_cast<void**>(&P->d.interp_items), sizeof(int4) * items.size())) != cudaSuccess)
            return e;
        P->device_bytes += int64_t(sizeof(int4) * items.size());
        P->n_interp_items = int(items.size());
        e = cudaMemcpyAsync(P->d.interp_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(st);
    }
    return cudaSuccess;
}

// --------------------------------------------------------------- lattice plans
// A lattice x0 + i p2, y0 + j p2 (point j nx + i) bins without a sort: a
// point's first-tap cell and fraction depend on its column i (x) and row j
// (y) alone and do not decrease along them, so the points a tile holds, halo
// duplicates included, are a product of one contiguous index range per axis:
// for tile k of an axis, [a, b) the indices whose first tap lies in it (home)
// and [c, a) the preceding ones whose taps reach into it.  Records are
// written in tile order, home records first, then ordered by bank class like
// any other plan's.
__global__ void lattice_axis_kernel(int n, double v0, double p2, BinArgs a, int* __restrict__ l0,
                                    double* __restrict__ frac, int* __restrict__ err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = v0 + double(i) * p2;
        const PointSplit s = split_point(v, v, a);   // the x part of a point at (v, v)
        if (!s.ok) atomicOr(err, 1);
        l0[i] = s.l0x;
        frac[i] = s.fx;
    }
}

// one CTA per tile; rx / ry: (c, a, b) of each tile index per axis
template <typename Rec, typename S>
__global__ void lattice_records_kernel(const int* __restrict__ l0x, const double* __restrict__ fx,
                                       const int* __restrict__ l0y, const double* __restrict__ fy,
                                       const int4* __restrict__ rx, const int4* __restrict__ ry,
                                       const int* __restrict__ off, int ntx, int nx, long long cap,
                                       Rec* __restrict__ rec) {
    const int t = blockIdx.x, ky = t / ntx, kx = t - ky * ntx;
    const int4 X = rx[kx], Y = ry[ky];
    const int hw = X.z - X.y, ew = X.y - X.x, aw = X.z - X.x;   // home, extension and all widths in x
    const int home = hw * (Y.z - Y.y), all = aw * (Y.z - Y.x);
    const int d1 = ew * (Y.z - Y.x);   // duplicates with i in [c, a), any row of the tile
    const int b0 = off[t];
    for (int r = threadIdx.x; r < all; r += blockDim.x) {
        int i, j;
        if (r < home) {
            i = X.y + r % hw;
            j = Y.y + r / hw;
        } else if (r - home < d1) {
            const int q = r - home;
            i = X.x + q % ew;
            j = Y.x + q / ew;
        } else {   // i in [a, b), rows [c, a) of y
            const int q = r - home - d1;
            i = X.y + q % hw;
            j = Y.x + q / hw;
        }
        Rec o;
        o.cell = (uint32_t(l0y[j]) << 16) | uint32_t(l0x[i]);
        o.fx = S(fx[i]);
        o.fy = S(fy[j]);
        o.j = int32_t(j * nx + i);
        if (NUASM_IN_RANGE(b0 + r, cap, dbg::kBinRec)) rec[b0 + r] = o;
    }
}

// Per-plan bank skew (or per-tile skews) and the round-robin record order of
// every tile (order_tile_kernel), for records already placed in P->d.rec
// in tile order with the offsets and home counts set.
cudaError_t order_records(nuasm_plan_s* P, cudaStream_t st) {
    const Geometry& g = P->g;
    const int nt = g.ntiles;
    const int total = int(P->nrec);
    const size_t rsz = P->f64 ? sizeof(RecD) : sizeof(RecF);
    cudaError_t e;
    if (NUASM_TILE_SKEW) {
        // per-tile bank skew: the candidate that balances the tile's record classes best
        unsigned long long* hist = nullptr;
        unsigned long long hh[kNumSkews] = {};
        if ((e = xmalloc(reinterpret_cast<void**>(&P->d.tile_skew), size_t(nt))) != cudaSuccess) return e;
        P->device_bytes += nt;
        if ((e = xmalloc_async(reinterpret_cast<void**>(&hist), sizeof(hh), st)) != cudaSuccess) return e;
        e = cudaMemsetAsync(hist, 0, sizeof(hh), st);
        if (e == cudaSuccess) {
            if (P->f64)
                tile_skew_kernel<RecD><<<nt, 256, 0, st>>>(static_cast<const RecD*>(P->d.rec), P->d.tile_off,
                                                           P->d.tile_home, g.T, g.ntx, P->d.tile_skew, hist);
            else
                tile_skew_kernel<RecF><<<nt, 256, 0, st>>>(static_cast<const RecF*>(P->d.rec), P->d.tile_off,
                                                           P->d.tile_home, g.T, g.ntx, P->d.tile_skew, hist);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        xfree_async(hist, st);
        if (e != cudaSuccess) return e;
        int most = 0;
        for (int k = 1; k < kNumSkews; ++k)
            if (hh[k] > hh[most]) most = k;
        P->skew = skew_candidate(most);
    } else {
        // one bank skew for every tile: 2 where it balances the record classes at least 5% better
        unsigned long long* sums = nullptr;
        unsigned long long hs[2] = {0, 0};
        if ((e = xmalloc_async(reinterpret_cast<void**>(&sums), sizeof(hs), st)) != cudaSuccess) return e;
        e = cudaMemsetAsync(sums, 0, sizeof(hs), st);
        if (e == cudaSuccess) {
            if (P->f64)
                class_balance_kernel<RecD><<<nt, 256, 0, st>>>(static_cast<const RecD*>(P->d.rec),
                                                               P->d.tile_off, P->d.tile_home, g.T, g.ntx, sums);
            else
                class_balance_kernel<RecF><<<nt, 256, 0, st>>>(static_cast<const RecF*>(P->d.rec),
                                                               P->d.tile_off, P->d.tile_home, g.T, g.ntx, sums);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        xfree_async(sums, st);
        if (e != cudaSuccess) return e;
        P->skew = double(hs[1]) < 0.95 * double(hs[0]) ? 2 : 0;
    }
    void* tmp = nullptr;
    if ((e = xmalloc_async(&tmp, rsz * size_t(total), st)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(tmp, P->d.rec, rsz * size_t(total), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        if (P->f64)
            order_tile_kernel<RecD><<<nt, 256, 0, st>>>(static_cast<const RecD*>(tmp), static_cast<RecD*>(P->d.rec),
                                                        P->d.tile_off, P->d.tile_home, g.T, g.ntx, P->skew,
                                                P->d.tile_skew);
        else
            order_tile_kernel<RecF><<<nt, 256, 0, st>>>(static_cast<const RecF*>(tmp), static_cast<RecF*>(P->d.rec),
                                                        P->d.tile_off, P->d.tile_home, g.T, g.ntx, P->skew,
                                                P->d.tile_skew);
        e = cudaGetLastError();
    }
    xfree_async(tmp, st);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

nuasm_status run_binning(nuasm_plan_s* P, const double* x, const double* y, const double* w, cudaStream_t st) {
    const Geometry& g = P->g;
    BinArgs a{g.n, g.W, g.T, g.ntx, g.w, g.h, P->p.pitch, P->m};
    const int nt = g.ntiles;
    int* cnt = nullptr;   // home_cnt, dup_cnt, cur_home, cur_dup
    cudaError_t e = xmalloc_async(reinterpret_cast<void**>(&cnt), sizeof(int) * 4 * size_t(nt), st);
    if (e != cudaSuccess) return cuda_status(e);
    int* home_cnt = cnt;
    int* dup_cnt = cnt + nt;
    int* cur_home = cnt + 2 * nt;
    int* cur_dup = cnt + 3 * nt;
    auto fail = [&](cudaError_t err) {
        xfree_async(cnt, st);
        cudaStreamSynchronize(st);
        return cuda_status(err);
    };
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * 4 * size_t(nt), st)) != cudaSuccess) return fail(e);
    if (P->d.h_err) *P->d.h_err = 0;   // host-mapped: no device work has touched it yet
    else if ((e = cudaMemsetAsync(P->d.err, 0, sizeof(int), st)) != cudaSuccess) return fail(e);
    const int blocks = int(std::min<int64_t>((P->m + 255) / 256, 152 * 16));
    if (P->m > 0) {
        bin_count_kernel<<<blocks, 256, 0, st>>>(x, y, a, home_cnt, dup_cnt, P->d.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    }
    bin_scan_kernel<<<1, 1024, 0, st>>>(home_cnt, dup_cnt, nt, P->d.tile_off, P->d.tile_home);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    int total = 0, errw = 0;
    if ((e = cudaMemcpyAsync(&total, P->d.tile_off + nt, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
    if (!P->d.h_err &&
        (e = cudaMemcpyAsync(&errw, P->d.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    if (P->d.h_err) errw = *static_cast<volatile int*>(P->d.h_err);
    if (errw) {
        fail(cudaSuccess);
        return NUASM_ERANGE;
    }
    P->nrec = total;
    a.cap = total;
    if ((e = make_tile_order(P, st)) != cudaSuccess) return fail(e);
    const size_t rsz = P->f64 ? sizeof(RecD) : sizeof(RecF);
    if ((e = xmalloc(&P->d.rec, rsz * size_t(total > 0 ? total : 1))) != cudaSuccess) return fail(e);
    P->device_bytes += int64_t(rsz) * (total > 0 ? total : 1);
    if (w && P->m > 0) {
        if ((e = xmalloc(reinterpret_cast<void**>(&P->d.wpt), sizeof(double) * size_t(P->m))) != cudaSuccess)
            return fail(e);
        P->device_bytes += int64_t(sizeof(double)) * P->m;
        e = cudaMemcpyAsync(P->d.wpt, w, sizeof(double) * size_t(P->m), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail(e);
    }
    if (P->m > 0) {
        if (P->f64)
            bin_scatter_kernel<RecD, double><<<blocks, 256, 0, st>>>(x, y, a, P->d.tile_off, home_cnt, cur_home,
                                                                     cur_dup, static_cast<RecD*>(P->d.rec));
        else
            bin_scatter_kernel<RecF, float><<<blocks, 256, 0, st>>>(x, y, a, P->d.tile_off, home_cnt, cur_home,
                                                                    cur_dup, static_cast<RecF*>(P->d.rec));
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    }
    if (P->m > 0 && total > 0 && (e = order_records(P, st)) != cudaSuccess) return fail(e);
    xfree_async(cnt, st);
    return cuda_status(cudaStreamSynchronize(st));
}

nuasm_status run_binning_lattice(nuasm_plan_s* P, const LatticeSpec& lat, cudaStream_t st) {
    const Geometry& g = P->g;
    const BinArgs a{g.n, g.W, g.T, g.ntx, g.w, g.h, P->p.pitch, P->m};
    const int nt = g.ntiles, ntx = g.ntx, nx = lat.nx, ny = lat.ny;
    // scratch: l0x, l0y (int), fx, fy (double), rx, ry (int4)
    const size_t bi = sizeof(int) * (size_t(nx) + ny), bd = sizeof(double) * (size_t(nx) + ny),
                 br = sizeof(int4) * 2 * size_t(ntx);
    char* scratch = nullptr;
    cudaError_t e = xmalloc_async(reinterpret_cast<void**>(&scratch), bd + br + bi, st);
    if (e != cudaSuccess) return cuda_status(e);
    double* dfx = reinterpret_cast<double*>(scratch);
    double* dfy = dfx + nx;
    int4* drx = reinterpret_cast<int4*>(scratch + bd);
    int4* dry = drx + ntx;
    int* dl0x = reinterpret_cast<int*>(scratch + bd + br);
    int* dl0y = dl0x + nx;
    auto fail = [&](cudaError_t err) {
        cudaStreamSynchronize(st);   // host vectors below may still be read by copies
        xfree_async(scratch, st);
        cudaStreamSynchronize(st);
        return cuda_status(err);
    };
    if (P->d.h_err) *P->d.h_err = 0;   // host-mapped: no device work has touched it yet
    else if ((e = cudaMemsetAsync(P->d.err, 0, sizeof(int), st)) != cudaSuccess) return fail(e);
    lattice_axis_kernel<<<std::max(1, std::min((nx + 255) / 256, 152 * 4)), 256, 0, st>>>(nx, lat.x0, lat.pitch2, a,
                                                                                         dl0x, dfx, P->d.err);
    lattice_axis_kernel<<<std::max(1, std::min((ny + 255) / 256, 152 * 4)), 256, 0, st>>>(ny, lat.y0, lat.pitch2, a,
                                                                                         dl0y, dfy, P->d.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    std::vector<int> l0x(nx), l0y(ny);
    int errw = 0;
    if ((e = cudaMemcpyAsync(l0x.data(), dl0x, sizeof(int) * size_t(nx), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(l0y.data(), dl0y, sizeof(int) * size_t(ny), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(e);
    if (!P->d.h_err &&
        (e = cudaMemcpyAsync(&errw, P->d.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    if (P->d.h_err) errw = *static_cast<volatile int*>(P->d.h_err);
    if (errw) {
        fail(cudaSuccess);
        return NUASM_ERANGE;
    }
    // per axis and tile index k: c = first index whose taps reach tile k (l0 >= kT - (w - 1)),
    // a = first home index (l0 >= kT), b = first index of the next tile (l0 >= (k + 1)T)
    auto ranges = [&](const std::vector<int>& l0) {
        std::vector<int4> r(ntx);
        for (int k = 0; k < ntx; ++k) {
            auto first = [&](long long v) {
                return int(std::lower_bound(l0.begin(), l0.end(), v) - l0.begin());
            };
            const int ak = first(int64_t(k) * g.T), bk = first(int64_t(k + 1) * g.T);
            const int ck = k == 0 ? ak : first(int64_t(k) * g.T - (g.w - 1));
            r[k] = make_int4(ck, ak, bk, 0);
        }
        return r;
    };
    const std::vector<int4> rx = ranges(l0x), ry = ranges(l0y);
    std::vector<int> off(size_t(nt) + 1), home(nt);
    int64_t total = 0;
    for (int ky = 0; ky < ntx; ++ky)
        for (int kx = 0; kx < ntx; ++kx) {
            const int t = ky * ntx + kx;
            off[t] = int(total);
            home[t] = (rx[kx].z - rx[kx].y) * (ry[ky].z - ry[ky].y);
            total += int64_t(rx[kx].z - rx[kx].x) * (ry[ky].z - ry[ky].x);
            if (total > INT32_MAX) {
                fail(cudaSuccess);
                return NUASM_EUNSUPPORTED;
            }
        }
    off[nt] = int(total);
    if ((e = cudaMemcpyAsync(drx, rx.data(), sizeof(int4) * size_t(ntx), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dry, ry.data(), sizeof(int4) * size_t(ntx), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->d.tile_off, off.data(), sizeof(int) * (size_t(nt) + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->d.tile_home, home.data(), sizeof(int) * size_t(nt), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return fail(e);
    P->nrec = total;
    if ((e = make_tile_order(P, st)) != cudaSuccess) return fail(e);
    const size_t rsz = P->f64 ? sizeof(RecD) : sizeof(RecF);
    if ((e = xmalloc(&P->d.rec, rsz * size_t(total > 0 ? total : 1))) != cudaSuccess) return fail(e);
    P->device_bytes += int64_t(rsz) * (total > 0 ? total : 1);
    if (total > 0) {
        if (P->f64)
            lattice_records_kernel<RecD, double><<<nt, 256, 0, st>>>(dl0x, dfx, dl0y, dfy, drx, dry, P->d.tile_off,
                                                                    ntx, nx, total, static_cast<RecD*>(P->d.rec));
        else
            lattice_records_kernel<RecF, float><<<nt, 256, 0, st>>>(dl0x, dfx, dl0y, dfy, drx, dry, P->d.tile_off,
                                                                   ntx, nx, total, static_cast<RecF*>(P->d.rec));
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
        if ((e = order_records(P, st)) != cudaSuccess) return fail(e);
    }
    xfree_async(scratch, st);
    return cuda_status(cudaStreamSynchronize(st));
}

// Binning into caller-provided device storage, with no allocation and no host
// read-back: `cnt` holds 4 * ntiles ints of scratch, `rec_tmp` and P->d.rec
// hold at least 4 * m records each (a point lands in at most four tiles), and
// P->d.tile_off, P->d.tile_home and P->d.err are set by the caller.  The
// out-of-window flag is left in P->d.err for the caller to read.
cudaError_t bin_points_into(const nuasm_plan_s* P, const double* x, const double* y, int* cnt, void* rec_tmp,
                            cudaStream_t st) {
    const Geometry& g = P->g;
    const BinArgs a{g.n, g.W, g.T, g.ntx, g.w, g.h, P->p.pitch, P->m, 4 * P->m};
    const int nt = g.ntiles;
    int* home_cnt = cnt;
    int* dup_cnt = cnt + nt;
    int* cur_home = cnt + 2 * nt;
    int* cur_dup = cnt + 3 * nt;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * 4 * size_t(nt), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(P->d.err, 0, sizeof(int), st)) != cudaSuccess) return e;
    const int blocks = int(std::min<int64_t>((P->m + 255) / 256, 152 * 16));
    if (P->m > 0) {
        bin_count_kernel<<<blocks, 256, 0, st>>>(x, y, a, home_cnt, dup_cnt, P->d.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    bin_scan_kernel<<<1, 1024, 0, st>>>(home_cnt, dup_cnt, nt, P->d.tile_off, P->d.tile_home);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (P->m == 0) return cudaSuccess;
    if (P->f64) {
        bin_scatter_kernel<RecD, double><<<blocks, 256, 0, st>>>(x, y, a, P->d.tile_off, home_cnt, cur_home,
                                                                 cur_dup, static_cast<RecD*>(rec_tmp));
        order_tile_kernel<RecD><<<nt, 256, 0, st>>>(static_cast<const RecD*>(rec_tmp), static_cast<RecD*>(P->d.rec),
                                                    P->d.tile_off, P->d.tile_home, g.T, g.ntx, P->skew,
                                                    P->d.tile_skew);
    } else {
        bin_scatter_kernel<RecF, float><<<blocks, 256, 0, st>>>(x, y, a, P->d.tile_off, home_cnt, cur_home,
                                                                cur_dup, static_cast<RecF*>(rec_tmp));
        order_tile_kernel<RecF><<<nt, 256, 0, st>>>(static_cast<const RecF*>(rec_tmp), static_cast<RecF*>(P->d.rec),
                                                    P->d.tile_off, P->d.tile_home, g.T, g.ntx, P->skew,
                                                    P->d.tile_skew);
    }
    return cudaGetLastError();
}

size_t record_bytes(bool f64) { return f64 ? sizeof(RecD) : sizeof(RecF); }

cudaError_t launch_spread(const nuasm_plan_s* P, const void* c, cudaStream_t st) {
    return gridding<true>(P, c, nullptr, st);
}

cudaError_t launch_interp(const nuasm_plan_s* P, void* v, cudaStream_t st) {
    return gridding<false>(P, nullptr, v, st);
}

}  // namespace nuasm
