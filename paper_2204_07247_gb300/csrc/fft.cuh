// fft.cuh -- warp-owned shared-memory Stockham FFTs for sm_103a.
//
// One warp transforms one complex line of length N (a row of two real fields
// packed as real and imaginary parts, or a column of a half spectrum) held in
// its own slice of shared memory.  Each radix-R stage reads R points at stride
// N/R, applies the twiddles exp(sign 2 pi i (j mod Ns) r / (Ns R)), does a
// length-R DFT in registers and writes the results at
// (j div Ns) Ns R + (j mod Ns) + r Ns (the Stockham autosort recursion: natural
// order, no bit reversal).  Stages ping-pong between two buffers and are
// separated by __syncwarp only: no CTA-wide barrier inside a transform.  (The
// CTA-cooperative variant at the end of this file shares the lines of one unit
// among all warps of a CTA and separates its stages by CTA barriers.)
//
// The transforms are the DFT of Sec. 3.2 (Fourier collocation): forward
// unnormalised with sign -1, inverse with sign +1; the 1/n_pts factor of the
// inverse is applied by the caller.
#pragma once
#include "compat.cuh"

namespace pagd {

// largest line length supported; the global twiddle table holds
// exp(-2 pi i m / kNMax), m < kNMax
constexpr int kLogNMax = 10;
constexpr int kNMax = 1 << kLogNMax;
constexpr int kWarp = PAGD_WARP;

template <class T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };
template <class T> using cx = typename V2<T>::type;

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by S*i (S = -1: by -i, S = +1: by +i)
template <int S, class C> __device__ __forceinline__ C mul_si(C a) {
    return (S < 0) ? C{a.y, -a.x} : C{-a.y, a.x};
}

template <int S, class C> __device__ __forceinline__ void dft2(C* v) {
    C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}

template <int S, class C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_si<S>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <int S, class C> __device__ __forceinline__ void dft8(C* v) {
    using T = decltype(v[0].x);
    const T c = (T)0.70710678118654752440;  // cos(pi/4)
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    // o_k *= exp(S 2 pi i k / 8)
    C w1 = C{c * (o1.x - (T)S * o1.y), c * (o1.y + (T)S * o1.x)};
    C w2 = mul_si<S>(o2);
    C w3 = C{c * (-o3.x - (T)S * o3.y), c * ((T)S * o3.x - o3.y)};
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

template <int R, int S, class C> __device__ __forceinline__ void dftR(C* v) {
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 4) dft4<S>(v[0], v[1], v[2], v[3]);
    else dft8<S>(v);
}

__device__ __forceinline__ void warp_sync() {
#ifndef PAGD_EMU
    __syncwarp();
#endif
}

// One radix-R Stockham stage of one line of length N = 1 << logN, done by the
// lanes of one warp.  Ns = 1 << logNs.  tw: exp(-2 pi i m / (1 << logTw)).
template <int R, int S, class T>
__device__ __forceinline__ void stockham_stage_w(const cx<T>* src, cx<T>* dst, int logN, int logNs,
                                                 const cx<T>* tw, int logTw, int lane) {
    using C = cx<T>;
    constexpr int logR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    const int logNb = logN - logR;  // butterflies = N / R
    const int nb = 1 << logNb;
    const int twshift = logTw - (logNs + logR);  // index scale (1 << logTw) / (Ns R)
    for (int j = lane; j < nb; j += kWarp) {
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = src[j + (r << logNb)];
        const int jm = j & ((1 << logNs) - 1);
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = tw[(jm * r) << twshift];
                if (S > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dftR<R, S>(v);
        const int idxD = ((j - jm) << logR) + jm;
#pragma unroll
        for (int r = 0; r < R; r++) dst[idxD + (r << logNs)] = v[r];
    }
}

// Whole transform of one line by one warp: data in b0 (written by any lane
// before the call); returns 0/1, the buffer holding the result.
template <int S, class T>
__device__ int fft_line_w(cx<T>* b0, cx<T>* b1, int logN, const cx<T>* tw, int logTw, int lane) {
    cx<T>* b[2] = {b0, b1};
    int cur = 0, logNs = 0;
    while (logNs < logN) {
        const int rem = logN - logNs;
        warp_sync();
        if (rem >= 3 && rem != 4) {
            stockham_stage_w<8, S, T>(b[cur], b[cur ^ 1], logN, logNs, tw, logTw, lane);
            logNs += 3;
        } else if (rem >= 2) {
            stockham_stage_w<4, S, T>(b[cur], b[cur ^ 1], logN, logNs, tw, logTw, lane);
            logNs += 2;
        } else {
            stockham_stage_w<2, S, T>(b[cur], b[cur ^ 1], logN, logNs, tw, logTw, lane);
            logNs += 1;
        }
        cur ^= 1;
    }
    warp_sync();
    return cur;
}

}  // namespace pagd

namespace pagd {

// ---------------------------------------------------------------------------
// Compile-time line length: the radix sequence, the per-lane butterfly loops and
// the line loop unroll, so the loads of all lines a warp owns are in flight
// together.  Lines l < nl (nl <= MAXL) sit at `pitch` apart in each buffer.
//
// Padded layout (PAD): point i of a line at i + i / 16, one slot of gap after
// every 16 points.  The first stages of a Stockham transform store at a stride
// of R (and then R^2) points; unpadded, the 32 lanes of a store then share
// 2 (or 4) of the 16 eight-byte bank pairs, a 16-way (4-way) conflict.  With
// the gap they spread over all 16 pairs.  A padded line of n points needs
// n + n / 16 slots.

template <bool P> __host__ __device__ __forceinline__ int pix(int i) { return P ? i + (i >> 4) : i; }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 16; }

template <int R, int S, class T, int LOGN, int LOGNS, int MAXL, bool PS = false, bool PD = false>
__device__ __forceinline__ void stage_fixed(const cx<T>* src, cx<T>* dst, int pitch_s, int pitch_d, int nl,
                                            const cx<T>* tw, int logTw, int lane) {
    using C = cx<T>;
    constexpr int LR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    constexpr int NB = 1 << (LOGN - LR);
    constexpr int NS = 1 << LOGNS;
    constexpr int PER = (NB + kWarp - 1) / kWarp;
    const int twshift = logTw - (LOGNS + LR);
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int j = lane + kWarp * i;
        if ((NB % kWarp) != 0 && j >= NB) break;
        const int jm = j & (NS - 1);
        C w[R];
        if (LOGNS > 0) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                w[r] = tw[(jm * r) << twshift];
                if (S > 0) w[r].y = -w[r].y;
            }
        }
        const int idxD = ((j - jm) << LR) + jm;
#pragma unroll
        for (int l = 0; l < MAXL; l++) {
            if (l < nl) {
                const C* s = src + l * pitch_s;
                C* d = dst + l * pitch_d;
                C v[R];
#pragma unroll
                for (int r = 0; r < R; r++) v[r] = s[pix<PS>(j + r * NB)];
                if (LOGNS > 0) {
#pragma unroll
                    for (int r = 1; r < R; r++) v[r] = cmul(v[r], w[r]);
                }
                dftR<R, S>(v);
#pragma unroll
                for (int r = 0; r < R; r++) d[pix<PD>(idxD + r * NS)] = v[r];
            }
        }
    }
}

// radix of the stage that starts at LOGNS: 8 while at least 3 levels remain
// (4 when exactly 4 do), then 4, then 2
__host__ __device__ constexpr int stage_radix(int logn, int logns) {
    return (logn - logns >= 3 && logn - logns != 4) ? 8 : (logn - logns >= 2 ? 4 : 2);
}
__host__ __device__ constexpr int radix_log(int r) { return r == 2 ? 1 : (r == 4 ? 2 : 3); }

template <int S, class T, int LOGN, int LOGNS, int MAXL, bool PAD = false>
struct FixedStages {
    static __device__ __forceinline__ int run(cx<T>* b0, cx<T>* b1, int pitch, int nl, const cx<T>* tw,
                                              int logTw, int lane, int cur) {
        if constexpr (LOGNS >= LOGN) {
            return cur;
        } else {
            constexpr int R = stage_radix(LOGN, LOGNS);
            warp_sync();
            stage_fixed<R, S, T, LOGN, LOGNS, MAXL, PAD, PAD>(cur ? b1 : b0, cur ? b0 : b1, pitch, pitch, nl, tw,
                                                             logTw, lane);
            return FixedStages<S, T, LOGN, LOGNS + radix_log(R), MAXL, PAD>::run(b0, b1, pitch, nl, tw, logTw, lane,
                                                                                cur ^ 1);
        }
    }
};

// nl lines of length 1 << LOGN in b0 -> result in b0 (returns 0) or b1 (1);
// PAD: both buffers in the padded layout
template <int S, class T, int LOGN, int MAXL, bool PAD = false>
__device__ __forceinline__ int fft_lines_fixed(cx<T>* b0, cx<T>* b1, int pitch, int nl, const cx<T>* tw,
                                               int logTw, int lane) {
    const int r = FixedStages<S, T, LOGN, 0, MAXL, PAD>::run(b0, b1, pitch, nl, tw, logTw, lane, 0);
    warp_sync();
    return r;
}

// The same transform from an unpadded input `in` (lines pitch_in apart, left
// unchanged) into the padded buffers b0 / b1 (lines pitch apart): the first
// stage reads `in` and writes b0.  Returns 0 / 1, the buffer of the result.
template <int S, class T, int LOGN, int MAXL>
__device__ __forceinline__ int fft_lines_fixed_into_padded(const cx<T>* in, int pitch_in, cx<T>* b0, cx<T>* b1,
                                                           int pitch, int nl, const cx<T>* tw, int logTw,
                                                           int lane) {
    constexpr int R = stage_radix(LOGN, 0);
    warp_sync();
    stage_fixed<R, S, T, LOGN, 0, MAXL, false, true>(in, b0, pitch_in, pitch, nl, tw, logTw, lane);
    const int r = FixedStages<S, T, LOGN, radix_log(R), MAXL, true>::run(b0, b1, pitch, nl, tw, logTw, lane, 0);
    warp_sync();
    return r;
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// ---------------------------------------------------------------------------
// CTA-cooperative transforms: all threads of the CTA share the nl lines of one
// unit, the butterflies of a stage dealt round robin over (line, butterfly),
// stages separated by a CTA barrier.  Used where a phase has fewer units than
// warps: the lines of one unit then occupy every SM sub-partition instead of
// one, which is what bounds an FP64 transform on a part with a low FP64 rate.

__device__ __forceinline__ void cta_sync() {
#ifndef PAGD_EMU
    __syncthreads();
#endif
}

template <int R, int S, class T, int LOGN>
__device__ __forceinline__ void stage_coop(const cx<T>* src, cx<T>* dst, int pitch, int nl, int logNs,
                                           const cx<T>* tw, int logTw, int tid, int nthr) {
    using C = cx<T>;
    constexpr int LR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    constexpr int LNB = LOGN - LR;
    constexpr int NB = 1 << LNB;
    const int twshift = logTw - (logNs + LR);
    const int nsm = (1 << logNs) - 1;
    const int tot = nl << LNB;
    for (int it = tid; it < tot; it += nthr) {
        const int l = it >> LNB, j = it & (NB - 1);
        const C* s = src + l * pitch;
        C* d = dst + l * pitch;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = s[j + r * NB];
        const int jm = j & nsm;
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = tw[(jm * r) << twshift];
                if (S > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dftR<R, S>(v);
        const int idxD = ((j - jm) << LR) + jm;
#pragma unroll
        for (int r = 0; r < R; r++) d[idxD + (r << logNs)] = v[r];
    }
}

// nl lines of length 1 << LOGN in b0 (written by any thread before the call)
// -> result in b0 (returns 0) or b1 (1), visible to every thread on return.
// Each stage takes the largest radix (8, 4, 2) whose butterflies still cover
// the nthr threads.
template <int S, class T, int LOGN>
__device__ __noinline__ int fft_lines_coop(cx<T>* b0, cx<T>* b1, int pitch, int nl, const cx<T>* tw, int logTw, int tid,
                              int nthr) {
    cx<T>* b[2] = {b0, b1};
    int cur = 0, logNs = 0;
    while (logNs < LOGN) {
        const int rem = LOGN - logNs;
        int lr = rem >= 3 ? 3 : rem;
        while (lr > 1 && (nl << (LOGN - lr)) < nthr) lr--;
        cta_sync();
        if (lr == 3) stage_coop<8, S, T, LOGN>(b[cur], b[cur ^ 1], pitch, nl, logNs, tw, logTw, tid, nthr);
        else if (lr == 2) stage_coop<4, S, T, LOGN>(b[cur], b[cur ^ 1], pitch, nl, logNs, tw, logTw, tid, nthr);
        else stage_coop<2, S, T, LOGN>(b[cur], b[cur ^ 1], pitch, nl, logNs, tw, logTw, tid, nthr);
        logNs += lr;
        cur ^= 1;
    }
    cta_sync();
    return cur;
}

}  // namespace pagd
