// Block-level Stockham FFT engine.
//
// One CTA transforms C independent sequences of power-of-two length L with
// E elements per thread held in registers.  Each pass applies radix-R
// butterflies (R = 16, 8, 4 or 2) in the self-sorting Stockham form
// (decimation in time, natural order in and out): butterfly j reads elements
// j + r L/R, multiplies input r by exp(DIR 2 pi i (j mod Ns) r / (Ns R)),
// applies the length-R DFT and writes (j div Ns) Ns R + (j mod Ns) + r Ns,
// with Ns the product of the radices of the earlier passes.
//
// The first pass reads its inputs through a load functor (global memory,
// another shared buffer, or values computed on the fly: zero padding, folds,
// pre-twiddles) and the last pass writes through a store functor (pruned,
// scattered or fused epilogues), so neither the padded input nor the full
// output ever touches shared memory.  Intermediate passes exchange through
// one padded shared buffer: every thread loads all its inputs, the block
// synchronises, then every thread writes, so the buffer is used in place.
//
// Layout of the shared buffer: ROWMAJOR = true stores sequence c contiguously
// (index c L + p; consecutive threads take consecutive j, which makes row
// loads from global memory coalesced); ROWMAJOR = false interleaves the
// sequences (index p C + c; consecutive threads take consecutive c, which
// makes loads of C adjacent columns of a row-major array coalesced).
#pragma once

#include "common.cuh"

namespace nuasm {

// ---------------------------------------------------------------- DFTs in registers
template <int R, int DIR, typename V> struct Dft;

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
template <int DIR, typename V> __device__ __forceinline__ V w8_3(V a) {
    return mul_i<DIR>(w8_1<DIR>(a));
}

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

// multiply by exp(DIR 2 pi i e / 16), e in [0, 9]
template <int DIR, typename V> __device__ __forceinline__ V w16(V a, int e) {
    using S = typename CTraits<V>::real;
    const S c1 = S(0.92387953251128675613), s1 = S(0.38268343236508977173);
    V w;
    switch (e) {
        case 0: return a;
        case 1: w = CTraits<V>::make(c1, DIR * s1); break;
        case 2: return w8_1<DIR>(a);
        case 3: w = CTraits<V>::make(s1, DIR * c1); break;
        case 4: return mul_i<DIR>(a);
        case 6: return w8_3<DIR>(a);
        case 9: w = CTraits<V>::make(-c1, -DIR * s1); break;
        default: w = CTraits<V>::make(S(1), S(0)); break;
    }
    return cmul(a, w);
}

template <int DIR, typename V> struct Dft<16, DIR, V> {
    __device__ __forceinline__ static void run(V* v) {
        // 16 = 4 x 4: DFT4 over n2 for each n1, twiddle w16^(n1 k2), DFT4 over n1
        V a[16];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            V t[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
            Dft<4, DIR, V>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[4 * k2 + n1] = w16<DIR>(t[k2], n1 * k2);
        }
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            V t[4] = {a[4 * k2], a[4 * k2 + 1], a[4 * k2 + 2], a[4 * k2 + 3]};
            Dft<4, DIR, V>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = t[k1];
        }
    }
};

template <int R> struct Log2;
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<16> { static constexpr int v = 4; };

// ---------------------------------------------------------------- one pass
template <typename V, int DIR, int E, int R, bool ROWMAJOR, class LoadF, class StoreF>
__device__ __forceinline__ void stockham_pass(V* __restrict__ sm, int logL, int logC, int logNs,
                                              bool first, bool last, const V* __restrict__ tw,
                                              int logLt, LoadF& load, StoreF& store) {
    constexpr int NB = E / R;
    constexpr int LR = Log2<R>::v;
    const int P = blockDim.x;
    const int tid = threadIdx.x;
    const int L = 1 << logL;
    const int LdR = L >> LR;
    const int Ns = 1 << logNs;
    V v[E];
    int jj[NB], cc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int beta = tid + b * P;
        int c, j;
        if (ROWMAJOR) { j = beta & (LdR - 1); c = beta >> (logL - LR); }
        else { c = beta & ((1 << logC) - 1); j = beta >> logC; }
        jj[b] = j;
        cc[b] = c;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int p = j + r * LdR;
            if (first) v[b * R + r] = load(p, c);
            else v[b * R + r] = sm[spad<V>(ROWMAJOR ? (c << logL) + p : (p << logC) + c)];
        }
    }
    if (!first) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (logNs > 0) {
            const int k = jj[b] & (Ns - 1);
            const int sh = logLt - logNs - LR;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                V w = __ldg(&tw[(k * r) << sh]);
                if (DIR > 0) w = cconj(w);
                v[b * R + r] = cmul(v[b * R + r], w);
            }
        }
        Dft<R, DIR, V>::run(v + b * R);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = jj[b], c = cc[b];
        const int k = j & (Ns - 1);
        const int base = ((j - k) << LR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int p = base + r * Ns;
            if (last) store(p, c, v[b * R + r]);
            else sm[spad<V>(ROWMAJOR ? (c << logL) + p : (p << logC) + c)] = v[b * R + r];
        }
    }
    if (!last) __syncthreads();
}

// ---------------------------------------------------------------- full transform
// Requires blockDim.x == (L * C) / E.  The caller must synchronise before the
// call if `sm` still holds data other threads read.  DIR = -1: forward
// (exp(-2 pi i ...)), +1: inverse, unnormalised.  `tw` holds exp(-2 pi i t / Lt)
// for t in [0, Lt), Lt = 2^logLt >= L.
template <typename V, int DIR, int E, bool ROWMAJOR, class LoadF, class StoreF>
__device__ void block_fft(V* __restrict__ sm, int logL, int logC, const V* __restrict__ tw,
                          int logLt, LoadF load, StoreF store) {
    constexpr int LE = Log2<E>::v;
    int rem = logL, logNs = 0;
    while (rem > 0) {
        const int lr = rem >= LE ? LE : rem;
        const bool first = logNs == 0, last = rem == lr;
        switch (lr) {
            case 4:
                stockham_pass<V, DIR, E, (E >= 16 ? 16 : 2), ROWMAJOR>(sm, logL, logC, logNs, first,
                                                                       last, tw, logLt, load, store);
                break;
            case 3:
                stockham_pass<V, DIR, E, (E >= 8 ? 8 : 2), ROWMAJOR>(sm, logL, logC, logNs, first, last,
                                                                     tw, logLt, load, store);
                break;
            case 2:
                stockham_pass<V, DIR, E, 4, ROWMAJOR>(sm, logL, logC, logNs, first, last, tw, logLt,
                                                      load, store);
                break;
            default:
                stockham_pass<V, DIR, E, 2, ROWMAJOR>(sm, logL, logC, logNs, first, last, tw, logLt,
                                                      load, store);
                break;
        }
        logNs += lr;
        rem -= lr;
    }
}

}  // namespace nuasm
