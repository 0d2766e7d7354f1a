// Block-level Stockham FFT engine with a compile-time radix schedule.
//
// One CTA transforms 2^LOGC independent sequences of length L = 2^LOGL with E
// elements per thread held in registers (blockDim.x == L * 2^LOGC / E).  Each
// pass applies radix-R butterflies in the self-sorting Stockham form
// (decimation in time, natural order in and out): butterfly j reads elements
// j + r L/R, multiplies input r by exp(DIR 2 pi i (j mod Ns) r / (Ns R)),
// applies the length-R DFT and writes (j div Ns) Ns R + (j mod Ns) + r Ns,
// Ns being the product of the earlier radices.  The schedule is LOGL / log2(E)
// passes of radix E followed by one smaller-radix pass for the remainder.
//
// The first pass reads through a load functor (global memory, another shared
// buffer, or values computed on the fly: zero padding, folds, pre-twiddles)
// and the last pass writes through a store functor (pruned, scattered or fused
// epilogues), so neither the padded input nor the full output touches shared
// memory.  Intermediate passes exchange through one padded shared buffer used
// in place: all threads load, the block synchronises, then all threads store.
//
// Layouts: ROWMAJOR = true stores sequence c contiguously (index c L + p;
// consecutive threads take consecutive j).  ROWMAJOR = false interleaves the
// sequences (index p C + c; consecutive threads take consecutive c), which
// makes C adjacent columns of a row-major array coalesced.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"
#include "nuasm_internal.h"

namespace nuasm {

// ---------------------------------------------------------------- DFTs in registers
template <int R, int DIR, typename V> struct Dft;

template <int DIR, typename V> struct Dft<1, DIR, V> {
    __device__ __forceinline__ static void run(V*) {}
};

template <int DIR, typename V> struct Dft<2, DIR, V> {
    __device__ __forceinline__ static void run(V* v) {
        V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR, typename V> struct Dft<4, DIR, V> {
    __device__ __forceinline__ static void run(V* v) {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), t3 = mul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

// multiply by exp(DIR 2 pi i e / 8) for e = 1 and e = 3
template <int DIR, typename V> __device__ __forceinline__ V w8_1(V a) {
    using S = typename CTraits<V>::real;
    const S r = S(0.70710678118654752440);
    return DIR < 0 ? CTraits<V>::make((a.x + a.y) * r, (a.y - a.x) * r)
                   : CTraits<V>::make((a.x - a.y) * r, (a.x + a.y) * r);
}
template <int DIR, typename V> __device__ __forceinline__ V w8_3(V a) { return mul_i<DIR>(w8_1<DIR>(a)); }

template <int DIR, typename V> struct Dft<8, DIR, V> {
    __device__ __forceinline__ static void run(V* v) {
        V e[4] = {v[0], v[2], v[4], v[6]};
        V o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR, V>::run(e);
        Dft<4, DIR, V>::run(o);
        o[1] = w8_1<DIR>(o[1]);
        o[2] = mul_i<DIR>(o[2]);
        o[3] = w8_3<DIR>(o[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// multiply by exp(DIR 2 pi i e / 16) for the exponents a 4 x 4 split needs
template <int DIR, int EXP, typename V> __device__ __forceinline__ V w16(V a) {
    using S = typename CTraits<V>::real;
    const S c1 = S(0.92387953251128675613), s1 = S(0.38268343236508977173);
    if (EXP == 0) return a;
    if (EXP == 2) return w8_1<DIR>(a);
    if (EXP == 4) return mul_i<DIR>(a);
    if (EXP == 6) return w8_3<DIR>(a);
    if (EXP == 1) return cmul(a, CTraits<V>::make(c1, DIR * s1));
    if (EXP == 3) return cmul(a, CTraits<V>::make(s1, DIR * c1));
    return cmul(a, CTraits<V>::make(-c1, -DIR * s1));   // EXP == 9
}

template <int DIR, typename V> struct Dft<16, DIR, V> {
    template <int N1> __device__ __forceinline__ static void col(const V* v, V* a) {
        V t[4] = {v[N1], v[N1 + 4], v[N1 + 8], v[N1 + 12]};
        Dft<4, DIR, V>::run(t);
        a[N1] = t[0];
        a[4 + N1] = w16<DIR, N1>(t[1]);
        a[8 + N1] = w16<DIR, 2 * N1>(t[2]);
        a[12 + N1] = w16<DIR, 3 * N1>(t[3]);
    }
    __device__ __forceinline__ static void run(V* v) {
        // 16 = 4 x 4: DFT4 over n2 for each n1, twiddle w16^(n1 k2), DFT4 over n1
        V a[16];
        col<0>(v, a);
        col<1>(v, a);
        col<2>(v, a);
        col<3>(v, a);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            V t[4] = {a[4 * k2], a[4 * k2 + 1], a[4 * k2 + 2], a[4 * k2 + 3]};
            Dft<4, DIR, V>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = t[k1];
        }
    }
};

template <int R> struct Log2 { static constexpr int v = R <= 1 ? 0 : 1 + Log2<R / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

// exp(DIR i pi k / 16) for k in [0, 16): constants once k is known at compile time
template <int DIR, typename V> __device__ __forceinline__ V cis_pi16(int k) {
    using S = typename CTraits<V>::real;
    // cos(pi k / 16), k = 0 .. 8
    constexpr S c[9] = {S(1.0),
                        S(0.98078528040323044912618223613424),
                        S(0.92387953251128675612818318939679),
                        S(0.83146961230254523707878837761791),
                        S(0.70710678118654752440084436210485),
                        S(0.55557023301960222474283081394853),
                        S(0.38268343236508977172845998403040),
                        S(0.19509032201612826784828486847702),
                        S(0.0)};
    const S re = k <= 8 ? c[k] : -c[16 - k];
    const S im = k <= 8 ? c[8 - k] : c[k - 8];
    return CTraits<V>::make(re, DIR > 0 ? im : -im);
}

// exp(DIR i pi q / L) for q in [0, L), for the load functor of the first pass of
// an engine of radix E, whose radix R0 is E (or L if smaller): there
// q = j + r L/R0 with j < L/R0 the same for
// every input of a butterfly and r a compile-time constant of the unrolled
// loop, so the factor is tw[j] (or its conjugate; tw[t] = exp(-i pi t / L))
// times the constant exp(DIR i pi r / R0): one table load per butterfly
// instead of one per input (FP32; on the FP64 pipe the extra complex product
// costs more than the loads it saves, so FP64 reads tw[q] itself).
template <typename V, int DIR, int LOGL, int E>
__device__ __forceinline__ V half_bin(const V* __restrict__ tw, int q) {
    if constexpr (sizeof(V) == 16) {
        const V t = ldgv(&tw[q]);
        return DIR < 0 ? t : cconj(t);
    } else {
        // the first pass has radix E, or 2^LOGL when the whole transform is shorter
        constexpr int R0 = LOGL >= Log2<E>::v ? E : (1 << LOGL);
        static_assert(R0 >= 2 && R0 <= 16, "first-pass radix");
        constexpr int LOGLDR = LOGL - Log2<R0>::v;
        const int j = q & ((1 << LOGLDR) - 1), r = q >> LOGLDR;
        const V t = ldgv(&tw[j]);
        return cmul(DIR < 0 ? t : cconj(t), cis_pi16<DIR, V>(r * (16 / R0)));
    }
}

// ---------------------------------------------------------------- twiddle powers
// w[r] = exp(-2 pi i k r / (Ns R)) for r in [1, R).  FP64 reads every power;
// FP32 reads w^1 and w^4 (w^1 and w^2 for R = 4) and forms the others by
// complex products (at most four roundings, about 2.4e-7 relative), which
// trades table loads for FMA-pipe work.  The reads come from the pass's own
// compact table (the pass twiddles that follow the full 2L-entry table; the
// layout is given with twp_pass_offset): one butterfly group's bases are
// adjacent, so FP32 reads them with one 16-byte load and a pass's table is a
// few KB of L1.  The table reads are split from the products (twiddle_base /
// twiddle_powers) so a pass can issue them before its barrier.
template <typename V, int R> struct TwBase {
    static constexpr int N = (sizeof(V) == 16 || R == 2) ? R - 1 : 2;
    V t[N > 0 ? N : 1];
};

// offset of a pass's table from the start of the full table
template <typename V, int LE, int LOGL, int PASS> struct TwpOffset {
    static_assert(LE == 3 || LE == 4, "pass twiddles exist for the radix-8 and radix-16 schedules");
    static constexpr int v = (2 << LOGL) + twp_pass_offset(sizeof(V) == 16, LE, LOGL, PASS);
};

template <typename V, int R>
__device__ __forceinline__ void twiddle_base(const V* __restrict__ tp, int k, TwBase<V, R>& b) {
    constexpr int N = TwBase<V, R>::N;
    if constexpr (sizeof(V) == 8 && N == 2) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(tp) + k);
        b.t[0] = CTraits<V>::make(q.x, q.y);
        b.t[1] = CTraits<V>::make(q.z, q.w);
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r) b.t[r] = ldgv(&tp[k * N + r]);
    }
}

template <typename V, int R>
__device__ __forceinline__ void twiddle_powers(const TwBase<V, R>& b, V* w) {
    if constexpr (sizeof(V) == 16 || R == 2) {
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = b.t[r - 1];
    } else if constexpr (R == 4) {
        w[1] = b.t[0];
        w[2] = b.t[1];
        w[3] = cmul(w[2], w[1]);
    } else {
        w[1] = b.t[0];
        w[4] = b.t[1];
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
        if constexpr (R == 16) {
            w[8] = cmul(w[4], w[4]);
#pragma unroll
            for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
        }
    }
}

// ---------------------------------------------------------------- one pass
// Twiddle table: tw[t] = exp(-2 pi i t / 2L), t in [0, 2L), followed by the
// pass twiddles of the radix-8 and radix-16 schedules.
template <typename V, int DIR, int E, int LOGL, int LOGC, bool ROWMAJOR, bool SYNC_FIRST, int LR, int LOGNS,
          bool FIRST, bool LAST, class LoadF, class StoreF>
__device__ __forceinline__ void stockham_pass(V* __restrict__ sm, const V* __restrict__ tw, LoadF& load,
                                              StoreF& store) {
    constexpr int R = 1 << LR;
    constexpr int NB = E / R;
    constexpr int L = 1 << LOGL;
    constexpr int LDR = L >> LR;
    constexpr int NS = 1 << LOGNS;
    constexpr int C = 1 << LOGC;
    constexpr int P = (L * C) / E;
    constexpr int LE = Log2<E>::v;
    static_assert(LOGNS % LE == 0, "passes start at multiples of the schedule's radix");
    const V* __restrict__ tp = tw;
    if constexpr (LOGNS > 0) tp = tw + TwpOffset<V, LE, LOGL, LOGNS / LE>::v;
    // Shared-memory indices: element (c, p) sits at spad(ROWMAJOR ? c L + p : p C + c).  Along
    // one butterfly the unpadded index grows by a fixed step S (loads: L/R, stores: NS; times C
    // when the sequences interleave) from a base b whose residue mod the padding period plus
    // any multiple of S stays below the period, so spad(b + r S) = spad(b) + spad(r S): one
    // padded base per butterfly and compile-time offsets.
    constexpr int SLD = ROWMAJOR ? LDR : (LDR << LOGC);
    constexpr int SST = ROWMAJOR ? NS : (NS << LOGC);
    [[maybe_unused]] constexpr int NSM = spad_size<V>(L << LOGC);   // the transform's shared-memory extent
    const int tid = threadIdx.x;
    V v[E];
    int jj[NB], cc[NB];
    TwBase<V, R> twb[LOGNS > 0 ? NB : 1];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int beta = tid + b * P;
        int c, j;
        // tid < P, so j < LDR either way; the mask in the column case states it
        // for the compiler, which then folds q >> log2(LDR) in a first-pass
        // load functor to the constant r (see half_bin)
        if (ROWMAJOR) { j = beta & (LDR - 1); c = beta >> (LOGL - LR); }
        else { c = beta & (C - 1); j = (beta >> LOGC) & (LDR - 1); }
        jj[b] = j;
        cc[b] = c;
        if constexpr (LOGNS > 0) twiddle_base<V, R>(tp, j & (NS - 1), twb[b]);   // in flight across the barrier
        if (FIRST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = load(j + r * LDR, c);
        } else {
            const int b0 = spad<V>(ROWMAJOR ? (c << LOGL) + j : (j << LOGC) + c);
            const V* src = sm + b0;
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[b * R + r] = NUASM_IN_RANGE(b0 + spad<V>(r * SLD), NSM, dbg::kFftLoad) ? src[spad<V>(r * SLD)]
                                                                                        : CTraits<V>::zero();
        }
    }
    if (!FIRST || SYNC_FIRST) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if constexpr (LOGNS > 0) {
            V w[R];
            twiddle_powers<V, R>(twb[b], w);
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], DIR > 0 ? cconj(w[r]) : w[r]);
        }
        Dft<R, DIR, V>::run(v + b * R);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = jj[b], c = cc[b];
        const int k = j & (NS - 1);
        const int base = ((j - k) << LR) + k;
        if (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) store(base + r * NS, c, v[b * R + r]);
        } else {
            const int d0 = spad<V>(ROWMAJOR ? (c << LOGL) + base : (base << LOGC) + c);
            V* dst = sm + d0;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (NUASM_IN_RANGE(d0 + spad<V>(r * SST), NSM, dbg::kFftStore)) dst[spad<V>(r * SST)] = v[b * R + r];
        }
    }
    if (!LAST) __syncthreads();
}

// passes of radix E, then the remainder (LOGL mod log2 E) as one smaller-radix pass
template <typename V, int DIR, int E, int LOGL, int LOGC, bool ROWMAJOR, bool SYNC_FIRST, int I, class LoadF,
          class StoreF, class HookF>
__device__ __forceinline__ void run_passes(V* __restrict__ sm, const V* __restrict__ tw, LoadF& load,
                                           StoreF& store, HookF& after_first) {
    constexpr int LE = Log2<E>::v;
    constexpr int NFULL = LOGL / LE;
    constexpr int REM = LOGL % LE;
    constexpr int NPASS = NFULL + (REM ? 1 : 0);
    if constexpr (I < NPASS) {
        constexpr int LR = I < NFULL ? LE : REM;
        stockham_pass<V, DIR, E, LOGL, LOGC, ROWMAJOR, SYNC_FIRST, LR, I * LE, I == 0, I == NPASS - 1>(sm, tw, load,
                                                                                                     store);
        if constexpr (I == 0) after_first();
        run_passes<V, DIR, E, LOGL, LOGC, ROWMAJOR, SYNC_FIRST, I + 1>(sm, tw, load, store, after_first);
    }
}

// Full transform.  DIR = -1: forward (exp(-2 pi i ...)), +1: inverse, unnormalised.
// The caller synchronises before the call if `sm` still holds data that other
// threads read.  SYNC_FIRST: the first pass synchronises between reading its
// inputs and writing `sm`, so the load functor may read `sm` itself (an
// input staged in the exchange buffer).  `after_first` runs on every thread
// once the first pass has finished reading its inputs (after that pass's
// closing barrier when there are further passes): the load functor's source
// may be reused from then on.
template <typename V, int DIR, int E, int LOGL, int LOGC, bool ROWMAJOR, bool SYNC_FIRST = false, class LoadF,
          class StoreF, class HookF>
__device__ __forceinline__ void block_fft(V* __restrict__ sm, const V* __restrict__ tw, LoadF load, StoreF store,
                                          HookF after_first) {
    run_passes<V, DIR, E, LOGL, LOGC, ROWMAJOR, SYNC_FIRST, 0>(sm, tw, load, store, after_first);
}

template <typename V, int DIR, int E, int LOGL, int LOGC, bool ROWMAJOR, bool SYNC_FIRST = false, class LoadF,
          class StoreF>
__device__ __forceinline__ void block_fft(V* __restrict__ sm, const V* __restrict__ tw, LoadF load, StoreF store) {
    auto none = [] {};
    run_passes<V, DIR, E, LOGL, LOGC, ROWMAJOR, SYNC_FIRST, 0>(sm, tw, load, store, none);
}

}  // namespace nuasm
