// fft.cuh -- shared-memory Stockham FFTs on many lines at once, for sm_103a.
//
// A CTA holds a set of complex lines (rows of a real field packed in pairs, or
// columns of a half spectrum) in shared memory and transforms all of them
// together: each radix-R stage reads R points of a line at stride N/R, applies
// the twiddles exp(sign 2 pi i (j mod Ns) r / (Ns R)), does a length-R DFT in
// registers and writes the results at (j div Ns) Ns R + (j mod Ns) + r Ns
// (the Stockham autosort recursion, so the output is in natural order and no
// bit reversal is needed).  Stages ping-pong between two buffers.
//
// The transforms are the DFT of Sec. 3.2 (Fourier collocation): forward
// unnormalised with sign -1, inverse with sign +1; the 1/n_pts factor of the
// inverse is applied by the caller.
#pragma once
#include "compat.cuh"

namespace pagd {

// largest line length supported; the twiddle table holds exp(-2 pi i m / kNMax)
constexpr int kLogNMax = 10;
constexpr int kNMax = 1 << kLogNMax;

template <class T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };
template <class T> using cx = typename V2<T>::type;

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }
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

// One radix-R Stockham stage on `nlines` lines of length N = 1 << logN with
// line pitch `pitch` (complex elements).  Ns = 1 << logNs is the length of the
// sub-transforms already combined.  tw: exp(-2 pi i m / kNMax), m < kNMax.
template <int R, int S, class T>
__device__ __forceinline__ void stockham_stage(const cx<T>* __restrict__ src, cx<T>* __restrict__ dst,
                                               int logN, int logNs, int nlines, int pitch,
                                               const cx<T>* __restrict__ tw) {
    using C = cx<T>;
    constexpr int logR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    const int logNb = logN - logR;  // butterflies per line = N / R
    const int nb = 1 << logNb;
    const int total = nb * nlines;
    const int twshift = kLogNMax - (logNs + logR);  // index scale kNMax / (Ns R)
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int line = t >> logNb;
        const int j = t & (nb - 1);
        const C* s = src + line * pitch;
        C* d = dst + line * pitch;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = s[j + (r << logNb)];
        const int jm = j & ((1 << logNs) - 1);
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = ldg(&tw[(jm * r) << twshift]);
                if (S > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dftR<R, S>(v);
        const int idxD = ((j - jm) << logR) + jm;
#pragma unroll
        for (int r = 0; r < R; r++) d[idxD + (r << logNs)] = v[r];
    }
}

// Full transform of all lines: data starts in buf[0]; returns the index (0/1)
// of the buffer holding the result.  Every thread of the CTA must call it.
template <int S, class T>
__device__ int fft_lines(cx<T>* buf0, cx<T>* buf1, int logN, int nlines, int pitch,
                         const cx<T>* __restrict__ tw) {
    cx<T>* b[2] = {buf0, buf1};
    int cur = 0, logNs = 0;
    while (logNs < logN) {
        const int rem = logN - logNs;
        __syncthreads();
        if (rem >= 3 && rem != 4) {
            stockham_stage<8, S, T>(b[cur], b[cur ^ 1], logN, logNs, nlines, pitch, tw);
            logNs += 3;
        } else if (rem >= 2) {
            stockham_stage<4, S, T>(b[cur], b[cur ^ 1], logN, logNs, nlines, pitch, tw);
            logNs += 2;
        } else {
            stockham_stage<2, S, T>(b[cur], b[cur ^ 1], logN, logNs, nlines, pitch, tw);
            logNs += 1;
        }
        cur ^= 1;
    }
    __syncthreads();
    return cur;
}

}  // namespace pagd
