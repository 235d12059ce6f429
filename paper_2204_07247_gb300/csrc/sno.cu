// sno.cu -- a small spectral neural operator that proposes the initial iterate
// of an implicit time step (the learned-guess form of the solver): forward,
// backward and Adam kernels, FP32, for sm_103a.
//
// The paper starts PAGD from the extrapolation u^n + rho (u^n - u^{n-1})
// (Sec. 3.4.2); the network learns the remaining correction
// r = u^{n+1} - (u^n + rho (u^n - u^{n-1})) from (u^n, u^{n-1}), and
// pagd_step_with_guess keeps its proposal only when its first PAGD direction
// is smaller than the extrapolation's.
//
// Network, per sample on an n0 x n1 periodic grid (np = n0 n1 points):
//   a    = [u^n, s_in (u^n - u^{n-1})]                     (2 channels)
//   v_0  = P a + b_P                                        (C channels)
//   z_l  = W_l v_l + b_l + K_l v_l,  v_{l+1} = GELU(z_l),   l = 0 .. L-1
//   out  = Q v_L + b_Q,   guess = extrapolation + s_out out
// with the spectral convolution
//   (K v)[o](x) = sum over kept modes m of w_m Re( sum_c R[o][c][m] F[c][m] e^{i k_m.x} ) / np,
//   F[c][m] = sum_x v[c](x) e^{-i k_m.x},
// kept modes k0 in [-M0/2, M0/2), k1 in [0, M1), w_m = 1 for k1 = 0 and 2
// otherwise (the omitted k1 < 0 half of a real field's spectrum).
//
// Parameters are one flat FP32 array in this order: P [C][2], b_P [C]; for
// each layer W [C][C] (W[o][c]), b [C], R [C][C][M0 M1][2] (R[o][c][m], re, im);
// Q [C], b_Q.  The DFTs over the kept modes are computed directly (two
// separable stages per direction), not with a full FFT.
#include "../../include/pagd_sno.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <new>
#include <string>

namespace {

constexpr int kThr = 256;

struct SnoDims {
    int n0, n1, np, C, L, M0, M1, M;
};

__device__ __forceinline__ float gelu_f(float x) {
    // GELU with the tanh form (Hendrycks and Gimpel, 2016)
    const float k = 0.7978845608028654f;  // sqrt(2 / pi)
    const float u = k * (x + 0.044715f * x * x * x);
    return 0.5f * x * (1.f + tanhf(u));
}
__device__ __forceinline__ float gelu_grad(float x) {
    const float k = 0.7978845608028654f;
    const float u = k * (x + 0.044715f * x * x * x);
    const float t = tanhf(u);
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * k * (1.f + 3.f * 0.044715f * x * x);
}

__device__ __forceinline__ int k0_of(int m0, int M0, int n0) { return m0 < M0 / 2 ? m0 : n0 - M0 + m0; }

// exp(sign 2 pi i j / n) from sincospif
__device__ __forceinline__ float2 cis(int j, int n, float sign) {
    float s, c;
    sincospif(2.f * (float)j / (float)n, &s, &c);
    return make_float2(c, sign * s);
}
// the block's table t[j] = exp(-2 pi i j / n), j < n (conjugate for the inverse)
__device__ __forceinline__ void fill_tw(float2* t, int n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) t[j] = cis(j, n, -1.f);
    __syncthreads();
}

// ---------------------------------------------------------------- lift
// a = [u^n, s_in (u^n - u^{n-1})], v0 = P a + b_P
__global__ void k_lift(SnoDims d, const float* prm, const double* un, const double* unm1, float s_in, float* a,
                       float* v0, int B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (p >= d.np) return;
    const size_t o = (size_t)b * d.np + p;
    const float a0 = (float)un[o], a1 = (float)(s_in * (un[o] - unm1[o]));
    a[((size_t)b * 2 + 0) * d.np + p] = a0;
    a[((size_t)b * 2 + 1) * d.np + p] = a1;
    for (int c = 0; c < d.C; c++)
        v0[((size_t)b * d.C + c) * d.np + p] = prm[2 * c] * a0 + prm[2 * c + 1] * a1 + prm[2 * d.C + c];
}

// ------------------------------------------------- truncated DFT, forward
// stage 1 (last axis): T[r][m1] = sum_x1 X[r][x1] e^{-2 pi i m1 x1 / n1}, one block per row r
__global__ void k_dft_rows(SnoDims d, const float* X, float2* T) {
    __shared__ float2 part[kThr / 32][32];
    extern __shared__ float2 tw[];  // n1 entries
    fill_tw(tw, d.n1);
    const int r = blockIdx.x;
    const float* x = X + (size_t)r * d.n1;
    float2 acc[32];
    for (int m = 0; m < d.M1; m++) acc[m] = make_float2(0.f, 0.f);
    for (int x1 = threadIdx.x; x1 < d.n1; x1 += blockDim.x) {
        const float v = x[x1];
        for (int m = 0; m < d.M1; m++) {
            const float2 e = tw[(m * x1) & (d.n1 - 1)];
            acc[m].x += v * e.x;
            acc[m].y += v * e.y;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int m = 0; m < d.M1; m++) {
        float re = acc[m].x, im = acc[m].y;
        for (int s = 16; s > 0; s >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, s);
            im += __shfl_xor_sync(0xffffffffu, im, s);
        }
        if (lane == 0) part[w][m] = make_float2(re, im);
    }
    __syncthreads();
    if (threadIdx.x < d.M1) {
        float2 s = make_float2(0.f, 0.f);
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            s.x += part[i][threadIdx.x].x;
            s.y += part[i][threadIdx.x].y;
        }
        T[(size_t)r * d.M1 + threadIdx.x] = s;
    }
}

// stage 2 (first axis): F[g][m0][m1] = sum_x0 T[g][x0][m1] e^{-2 pi i k0 x0 / n0}, one block per
// channel g, one thread per mode
__global__ void k_dft_cols(SnoDims d, const float2* T, float2* F) {
    extern __shared__ float2 tw[];  // n0 entries
    fill_tw(tw, d.n0);
    const int g = blockIdx.x, m = threadIdx.x;
    if (m >= d.M) return;
    const int m0 = m / d.M1, m1 = m % d.M1, k0 = k0_of(m0, d.M0, d.n0);
    const float2* t = T + (size_t)g * d.n0 * d.M1 + m1;
    float2 s = make_float2(0.f, 0.f);
    for (int x0 = 0; x0 < d.n0; x0++) {
        const float2 v = t[(size_t)x0 * d.M1];
        const float2 e = tw[(k0 * x0) & (d.n0 - 1)];
        s.x += v.x * e.x - v.y * e.y;
        s.y += v.x * e.y + v.y * e.x;
    }
    F[(size_t)g * d.M + m] = s;
}

// ------------------------------------------------ truncated DFT, inverse
// stage 1 (first axis): U[g][x0][m1] = sum_m0 X[g][m0][m1] e^{+2 pi i k0 x0 / n0}
__global__ void k_idft_cols(SnoDims d, const float2* X, float2* U) {
    extern __shared__ float2 tw[];  // n0 entries
    fill_tw(tw, d.n0);
    const int g = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // x0 * M1 + m1
    if (i >= d.n0 * d.M1) return;
    const int x0 = i / d.M1, m1 = i % d.M1;
    float2 s = make_float2(0.f, 0.f);
    for (int m0 = 0; m0 < d.M0; m0++) {
        const float2 v = X[(size_t)g * d.M + m0 * d.M1 + m1];
        const int k0 = k0_of(m0, d.M0, d.n0);
        float2 e = tw[(k0 * x0) & (d.n0 - 1)];
        e.y = -e.y;
        s.x += v.x * e.x - v.y * e.y;
        s.y += v.x * e.y + v.y * e.x;
    }
    U[(size_t)g * d.n0 * d.M1 + i] = s;
}

// ---------------------------------------------------------------- mixing
// G[b][o][m] = sum_c R[o][c][m] F[b][c][m]
__global__ void k_mix(SnoDims d, const float* R, const float2* F, float2* G) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // o * M + m
    if (i >= d.C * d.M) return;
    const int o = i / d.M, m = i % d.M;
    float2 s = make_float2(0.f, 0.f);
    for (int c = 0; c < d.C; c++) {
        const float* r = R + (((size_t)o * d.C + c) * d.M + m) * 2;
        const float2 f = F[((size_t)b * d.C + c) * d.M + m];
        s.x += r[0] * f.x - r[1] * f.y;
        s.y += r[0] * f.y + r[1] * f.x;
    }
    G[((size_t)b * d.C + o) * d.M + m] = s;
}

// ----------------------------------------------- layer: W v + b + K v, GELU
// One block per (row x0, sample b); U holds the first-axis inverse of G.
__global__ void k_layer(SnoDims d, const float* W, const float* bias, const float2* U, const float* v, float* z,
                        float* vn, int last_act) {
    extern __shared__ float2 su[];  // [C][M1], then the table of n1 twiddles
    __shared__ float sw[32 * 32 + 32];
    float2* tw = su + d.C * d.M1;
    fill_tw(tw, d.n1);
    const int x0 = blockIdx.x, b = blockIdx.y;
    for (int i = threadIdx.x; i < d.C * d.M1; i += blockDim.x) {
        const int o = i / d.M1, m1 = i % d.M1;
        su[i] = U[(((size_t)b * d.C + o) * d.n0 + x0) * d.M1 + m1];
    }
    for (int i = threadIdx.x; i < d.C * d.C; i += blockDim.x) sw[i] = W[i];
    for (int i = threadIdx.x; i < d.C; i += blockDim.x) sw[d.C * d.C + i] = bias[i];
    __syncthreads();
    const float inv = 1.f / (float)d.np;
    for (int x1 = threadIdx.x; x1 < d.n1; x1 += blockDim.x) {
        const size_t p = (size_t)x0 * d.n1 + x1;
        float vin[32];
        for (int c = 0; c < d.C; c++) vin[c] = v[((size_t)b * d.C + c) * d.np + p];
        for (int o = 0; o < d.C; o++) {
            float y = 0.f;
            for (int m1 = 0; m1 < d.M1; m1++) {
                const float2 e = tw[(m1 * x1) & (d.n1 - 1)];  // conjugated below: exp(+i ...)
                const float2 u = su[o * d.M1 + m1];
                y += (m1 == 0 ? 1.f : 2.f) * (u.x * e.x + u.y * e.y);
            }
            float s = sw[d.C * d.C + o] + y * inv;
            for (int c = 0; c < d.C; c++) s += sw[o * d.C + c] * vin[c];
            z[((size_t)b * d.C + o) * d.np + p] = s;
            vn[((size_t)b * d.C + o) * d.np + p] = last_act ? gelu_f(s) : s;
        }
    }
}

// ---------------------------------------------------------- projection
// out = Q v + b_Q.  Inference: guess = un + rho (un - unm1) + s_out out.
// Training: loss and dout = 2 (out - t) / (np B), t = (target - extrapolation) / s_out.
__global__ void k_proj(SnoDims d, const float* Q, const float* v, const double* un, const double* unm1, double rho,
                       double s_out, double* guess, const double* target, float* dout, double* loss, int B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    double l = 0.0;
    if (p < d.np) {
        float o = Q[d.C];
        for (int c = 0; c < d.C; c++) o += Q[c] * v[((size_t)b * d.C + c) * d.np + p];
        const size_t i = (size_t)b * d.np + p;
        const double ext = un[i] + rho * (un[i] - unm1[i]);
        if (guess) guess[i] = ext + s_out * (double)o;
        if (target) {
            const double t = (target[i] - ext) / s_out;
            const double e = (double)o - t;
            l = e * e;
            dout[i] = (float)(2.0 * e / ((double)d.np * B));
        }
    }
    if (loss) {
        for (int s = 16; s > 0; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / ((double)d.np * B));
    }
}

// --------------------------------------------------------------- backward
// Sums over points of per-point products go to per-block partial rows, summed
// by k_sum_rows into the gradient (no float atomics on hot addresses).

// projection: dQ[c] = sum dout v_L[c], db_Q = sum dout; dv_L[c] = Q[c] dout
__global__ void k_proj_back(SnoDims d, const float* Q, const float* v, const float* dout, float* dv, float* part, int B) {
    __shared__ float red[kThr / 32][33];
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    float acc[33];
    for (int c = 0; c <= d.C; c++) acc[c] = 0.f;
    if (p < d.np) {
        const float g = dout[(size_t)b * d.np + p];
        for (int c = 0; c < d.C; c++) {
            const size_t i = ((size_t)b * d.C + c) * d.np + p;
            acc[c] = g * v[i];
            dv[i] = Q[c] * g;
        }
        acc[d.C] = g;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c <= d.C; c++) {
        float x = acc[c];
        for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
        if (lane == 0) red[w][c] = x;
    }
    __syncthreads();
    if (threadIdx.x <= d.C) {
        float s = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i][threadIdx.x];
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (d.C + 1) + threadIdx.x] = s;
    }
}

// layer, pointwise part: dz = dvn GELU'(z) (kept for the weight gradients and
// the spectral part) and dv = W^T dz
__global__ void k_layer_back(SnoDims d, const float* W, const float* z, const float* dvn, float* dz, float* dv,
                             int B) {
    __shared__ float sw[32 * 32];
    for (int i = threadIdx.x; i < d.C * d.C; i += blockDim.x) sw[i] = W[i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (p >= d.np) return;
    float g[32];
    for (int o = 0; o < d.C; o++) {
        const size_t i = ((size_t)b * d.C + o) * d.np + p;
        g[o] = dvn[i] * gelu_grad(z[i]);
        dz[i] = g[o];
    }
    for (int c = 0; c < d.C; c++) {
        float s = 0.f;
        for (int o = 0; o < d.C; o++) s += sw[o * d.C + c] * g[o];
        dv[((size_t)b * d.C + c) * d.np + p] = s;
    }
}

// per row (x0, b) partial sums dW[o][c] = sum dz[o] v[c] and db[o] = sum dz[o]:
// the row is staged in shared memory in chunks, one thread per (o, c)
constexpr int kWChunk = 128;
__global__ void k_wgrad(SnoDims d, const float* dz, const float* v, float* part) {
    __shared__ float sdz[32][kWChunk];
    __shared__ float sv[32][kWChunk];
    const int x0 = blockIdx.x, b = blockIdx.y;
    const int nrow = d.C * d.C + d.C;
    float acc[8];
    for (int q = 0; q < 8; q++) acc[q] = 0.f;
    for (int c0 = 0; c0 < d.n1; c0 += kWChunk) {
        __syncthreads();
        for (int i = threadIdx.x; i < d.C * kWChunk; i += blockDim.x) {
            const int ch = i / kWChunk, x = i % kWChunk;
            const size_t p = ((size_t)b * d.C + ch) * d.np + (size_t)x0 * d.n1 + c0 + x;
            const bool in = c0 + x < d.n1;
            sdz[ch][x] = in ? dz[p] : 0.f;
            sv[ch][x] = in ? v[p] : 0.f;
        }
        __syncthreads();
        for (int q = 0, i = threadIdx.x; i < nrow && q < 8; i += blockDim.x, q++) {
            float s = 0.f;
            if (i < d.C * d.C) {
                const int o = i / d.C, c = i % d.C;
                for (int x = 0; x < kWChunk; x++) s += sdz[o][x] * sv[c][x];
            } else {
                const int o = i - d.C * d.C;
                for (int x = 0; x < kWChunk; x++) s += sdz[o][x];
            }
            acc[q] += s;
        }
    }
    for (int q = 0, i = threadIdx.x; i < nrow && q < 8; i += blockDim.x, q++)
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * nrow + i] = acc[q];
}

// spectral part: dG[b][o][m] = (w_m / np) DFT(dz)[b][o][m] (already in G form);
// dR[o][c][m] += sum_b dG conj(F), dF[b][c][m] = sum_o conj(R) dG
__global__ void k_mix_back(SnoDims d, const float* R, const float2* F, const float2* dZ, float* dR, float2* dF, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // c * M + m
    if (i >= d.C * d.M) return;
    const int c = i / d.M, m = i % d.M, m1 = m % d.M1;
    const float wm = (m1 == 0 ? 1.f : 2.f) / (float)d.np;
    for (int b = 0; b < B; b++) {
        const float2 f = F[((size_t)b * d.C + c) * d.M + m];
        float2 s = make_float2(0.f, 0.f);
        for (int o = 0; o < d.C; o++) {
            float2 g = dZ[((size_t)b * d.C + o) * d.M + m];
            g.x *= wm;
            g.y *= wm;
            const float* r = R + (((size_t)o * d.C + c) * d.M + m) * 2;
            float* dr = dR + (((size_t)o * d.C + c) * d.M + m) * 2;
            dr[0] += g.x * f.x + g.y * f.y;  // dG conj(F)
            dr[1] += g.y * f.x - g.x * f.y;
            s.x += r[0] * g.x + r[1] * g.y;  // conj(R) dG
            s.y += r[0] * g.y - r[1] * g.x;
        }
        dF[((size_t)b * d.C + c) * d.M + m] = s;
    }
}

// dv[g](x) += sum over kept modes of Re(U[g][x0][m1] e^{+2 pi i m1 x1 / n1}) (the adjoint of the
// forward truncated DFT; U is the first-axis inverse of dF, no weights, no 1/np)
__global__ void k_idft_rows_add(SnoDims d, const float2* U, float* dv, int G) {
    extern __shared__ float2 tw[];  // n1 entries
    fill_tw(tw, d.n1);
    const int x0 = blockIdx.x, g = blockIdx.y;
    for (int x1 = threadIdx.x; x1 < d.n1; x1 += blockDim.x) {
        float s = 0.f;
        for (int m1 = 0; m1 < d.M1; m1++) {
            const float2 e = tw[(m1 * x1) & (d.n1 - 1)];  // exp(+i ...) = conj
            const float2 u = U[((size_t)g * d.n0 + x0) * d.M1 + m1];
            s += u.x * e.x + u.y * e.y;
        }
        dv[(size_t)g * d.np + (size_t)x0 * d.n1 + x1] += s;
    }
}

// lift: dP[c][j] = sum dv0[c] a[j], db_P[c] = sum dv0[c]; per-block partials [C][3]
__global__ void k_lift_back(SnoDims d, const float* a, const float* dv0, float* part, int B) {
    __shared__ float red[kThr / 32][96];
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    float a0 = 0.f, a1 = 0.f;
    if (p < d.np) {
        a0 = a[((size_t)b * 2) * d.np + p];
        a1 = a[((size_t)b * 2 + 1) * d.np + p];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c < d.C; c++) {
        const float g = p < d.np ? dv0[((size_t)b * d.C + c) * d.np + p] : 0.f;
        float x0 = g * a0, x1 = g * a1, x2 = g;
        for (int s = 16; s > 0; s >>= 1) {
            x0 += __shfl_xor_sync(0xffffffffu, x0, s);
            x1 += __shfl_xor_sync(0xffffffffu, x1, s);
            x2 += __shfl_xor_sync(0xffffffffu, x2, s);
        }
        if (lane == 0) {
            red[w][3 * c] = x0;
            red[w][3 * c + 1] = x1;
            red[w][3 * c + 2] = x2;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * d.C; i += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += red[q][i];
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (3 * d.C) + i] = s;
    }
}

// out[j] += sum over rows of part[row][j]
__global__ void k_sum_rows(const float* part, int rows, int cols, float* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; r++) s += part[(size_t)r * cols + j];
    out[j] += (float)s;
}

// lift partials are [C][3] = (dP0, dP1, db); the gradient layout is P[C][2] then b_P[C]
__global__ void k_lift_scatter(const float* sums, float* grad, int C) {
    const int c = threadIdx.x;
    if (c >= C) return;
    grad[2 * c] += sums[3 * c];
    grad[2 * c + 1] += sums[3 * c + 1];
    grad[2 * C + c] += sums[3 * c + 2];
}

// Adam (Kingma and Ba, 2015) with bias correction
// the weights as BF16 numbers (round to nearest even), kept in FP32 storage:
// the network computes with them and accumulates in FP32, Adam updates the
// FP32 master copy they are rounded from
__global__ void k_round_bf16(const float* src, float* dst, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct sno_net {
    SnoDims d;
    int batch;
    void* stream;
    char* ws;
    size_t ws_bytes;
    size_t off_a, off_v, off_z, off_F, off_G, off_T, off_U, off_dv, off_dv2, off_dz, off_dout, off_part, off_dF,
        off_loss, off_sums;
    size_t part_rows;
    std::string err;
};

static size_t param_count(const SnoDims& d) {
    return (size_t)3 * d.C + (size_t)d.L * ((size_t)d.C * d.C + d.C + (size_t)2 * d.C * d.C * d.M) + d.C + 1;
}
static size_t off_layer(const SnoDims& d, int l) {
    return (size_t)3 * d.C + (size_t)l * ((size_t)d.C * d.C + d.C + (size_t)2 * d.C * d.C * d.M);
}
static size_t off_Q(const SnoDims& d) { return off_layer(d, d.L); }

static pagd_status sno_fail(sno_net* s, pagd_status st, const char* m) {
    if (s) s->err = m;
    return st;
}

static void plan(sno_net* s) {
    const SnoDims& d = s->d;
    const size_t B = (size_t)s->batch, np = (size_t)d.np;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    s->off_a = take(sizeof(float) * B * 2 * np);
    s->off_v = take(sizeof(float) * B * d.C * np * (d.L + 1));
    s->off_z = take(sizeof(float) * B * d.C * np * d.L);
    s->off_F = take(sizeof(float2) * B * d.C * d.M * d.L);
    s->off_G = take(sizeof(float2) * B * d.C * d.M);
    s->off_T = take(sizeof(float2) * B * d.C * d.n0 * d.M1);
    s->off_U = take(sizeof(float2) * B * d.C * d.n0 * d.M1);
    s->off_dv = take(sizeof(float) * B * d.C * np);
    s->off_dv2 = take(sizeof(float) * B * d.C * np);
    s->off_dz = take(sizeof(float) * B * d.C * np);
    s->off_dout = take(sizeof(float) * B * np);
    const size_t rows_pt = B * (size_t)((np + kThr - 1) / kThr), rows_row = B * (size_t)d.n0;
    s->part_rows = rows_pt > rows_row ? rows_pt : rows_row;
    s->off_part = take(sizeof(float) * s->part_rows * (size_t)(d.C * d.C + d.C + 3 * d.C + 1));
    s->off_dF = take(sizeof(float2) * B * d.C * d.M);
    s->off_loss = take(sizeof(double));
    s->off_sums = take(sizeof(float) * (size_t)(d.C * d.C + d.C + 3 * d.C + 1));
    s->ws_bytes = o;
}

#define CK(x)                                                                       \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) return sno_fail(s, PAGD_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

// the whole forward pass for B samples; activations stay in the workspace
static pagd_status forward(sno_net* s, const float* prm, const double* un, const double* unm1, float s_in, int B) {
    const SnoDims& d = s->d;
    cudaStream_t st = (cudaStream_t)s->stream;
    char* w = s->ws;
    float* a = (float*)(w + s->off_a);
    float* v = (float*)(w + s->off_v);
    float* z = (float*)(w + s->off_z);
    float2* F = (float2*)(w + s->off_F);
    float2* G = (float2*)(w + s->off_G);
    float2* T = (float2*)(w + s->off_T);
    float2* U = (float2*)(w + s->off_U);
    const size_t vs = (size_t)B * d.C * d.np;  // one layer of activations
    const dim3 gp((d.np + kThr - 1) / kThr, B);
    k_lift<<<gp, kThr, 0, st>>>(d, prm, un, unm1, s_in, a, v, B);
    for (int l = 0; l < d.L; l++) {
        const float* L = prm + off_layer(d, l);
        const float* W = L;
        const float* bias = L + d.C * d.C;
        const float* R = L + d.C * d.C + d.C;
        float2* Fl = F + (size_t)l * B * d.C * d.M;
        k_dft_rows<<<B * d.C * d.n0, kThr, sizeof(float2) * d.n1, st>>>(d, v + l * vs, T);
        k_dft_cols<<<B * d.C, d.M, sizeof(float2) * d.n0, st>>>(d, T, Fl);
        k_mix<<<dim3((d.C * d.M + kThr - 1) / kThr, B), kThr, 0, st>>>(d, R, Fl, G);
        k_idft_cols<<<dim3((d.n0 * d.M1 + kThr - 1) / kThr, B * d.C), kThr, sizeof(float2) * d.n0, st>>>(d, G, U);
        k_layer<<<dim3(d.n0, B), kThr, sizeof(float2) * (d.C * d.M1 + d.n1), st>>>(d, W, bias, U, v + l * vs,
                                                                                   z + l * vs, v + (l + 1) * vs, 1);
    }
    CK(cudaGetLastError());
    return PAGD_OK;
}

extern "C" {

pagd_status sno_create(sno_net** out, int n0, int n1, int channels, int layers, int modes0, int modes1, int batch,
                       void* stream) {
    if (!out) return PAGD_EINVAL;
    *out = nullptr;
    auto pow2 = [](int v) { return v >= 8 && v <= 4096 && (v & (v - 1)) == 0; };
    if (!pow2(n0) || !pow2(n1) || channels < 1 || channels > 32 || layers < 1 || layers > 16 || modes0 < 2 ||
        (modes0 & 1) || modes0 > n0 || modes1 < 1 || modes1 > 32 || modes1 > n1 / 2 || modes0 * modes1 > 1024 ||
        batch < 1)
        return PAGD_EINVAL;
    sno_net* s = new (std::nothrow) sno_net();
    if (!s) return PAGD_ENOMEM;
    s->d = SnoDims{n0, n1, n0 * n1, channels, layers, modes0, modes1, modes0 * modes1};
    s->batch = batch;
    s->stream = stream;
    s->ws = nullptr;
    plan(s);
    *out = s;
    return PAGD_OK;
}

pagd_status sno_param_count(const sno_net* s, size_t* n) {
    if (!s || !n) return PAGD_EINVAL;
    *n = param_count(s->d);
    return PAGD_OK;
}

pagd_status sno_workspace_size(const sno_net* s, size_t* bytes) {
    if (!s || !bytes) return PAGD_EINVAL;
    *bytes = s->ws_bytes;
    return PAGD_OK;
}

pagd_status sno_set_workspace(sno_net* s, void* dev, size_t bytes) {
    if (!s || !dev) return PAGD_EINVAL;
    if (((uintptr_t)dev & 255) != 0) return sno_fail(s, PAGD_EINVAL, "workspace not 256-byte aligned");
    if (bytes < s->ws_bytes) return sno_fail(s, PAGD_ENOMEM, "workspace too small");
    s->ws = (char*)dev;
    return PAGD_OK;
}

pagd_status sno_predict(sno_net* s, const float* params, const double* un, const double* unm1, double rho,
                        double s_in, double s_out, int nsamples, double* guess) {
    if (!s || !params || !un || !unm1 || !guess) return PAGD_EINVAL;
    if (!s->ws) return sno_fail(s, PAGD_ESTATE, "no workspace");
    if (nsamples < 1 || nsamples > s->batch) return sno_fail(s, PAGD_EINVAL, "bad sample count");
    pagd_status r = forward(s, params, un, unm1, (float)s_in, nsamples);
    if (r != PAGD_OK) return r;
    const SnoDims& d = s->d;
    const float* vL = (const float*)(s->ws + s->off_v) + (size_t)d.L * nsamples * d.C * d.np;
    k_proj<<<dim3((d.np + kThr - 1) / kThr, nsamples), kThr, 0, (cudaStream_t)s->stream>>>(
        d, params + off_Q(d), vL, un, unm1, rho, s_out, guess, nullptr, nullptr, nullptr, nsamples);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize((cudaStream_t)s->stream));
    return PAGD_OK;
}

pagd_status sno_loss_grad(sno_net* s, const float* params, const double* un, const double* unm1,
                          const double* target, double rho, double s_in, double s_out, int nsamples, float* grad,
                          double* loss) {
    if (!s || !params || !un || !unm1 || !target || !grad) return PAGD_EINVAL;
    if (!s->ws) return sno_fail(s, PAGD_ESTATE, "no workspace");
    if (nsamples < 1 || nsamples > s->batch) return sno_fail(s, PAGD_EINVAL, "bad sample count");
    const SnoDims& d = s->d;
    const int B = nsamples;
    cudaStream_t st = (cudaStream_t)s->stream;
    pagd_status r = forward(s, params, un, unm1, (float)s_in, B);
    if (r != PAGD_OK) return r;
    char* w = s->ws;
    float* a = (float*)(w + s->off_a);
    float* v = (float*)(w + s->off_v);
    float* z = (float*)(w + s->off_z);
    float2* F = (float2*)(w + s->off_F);
    float2* T = (float2*)(w + s->off_T);
    float2* U = (float2*)(w + s->off_U);
    float2* dZ = (float2*)(w + s->off_G);
    float2* dF = (float2*)(w + s->off_dF);
    float* dv = (float*)(w + s->off_dv);
    float* dv2 = (float*)(w + s->off_dv2);
    float* dz = (float*)(w + s->off_dz);
    float* dout = (float*)(w + s->off_dout);
    float* part = (float*)(w + s->off_part);
    float* sums = (float*)(w + s->off_sums);
    double* dloss = (double*)(w + s->off_loss);
    const size_t vs = (size_t)B * d.C * d.np;
    const dim3 gp((d.np + kThr - 1) / kThr, B);
    CK(cudaMemsetAsync(grad, 0, sizeof(float) * param_count(d), st));
    CK(cudaMemsetAsync(dloss, 0, sizeof(double), st));
    const float* Q = params + off_Q(d);
    float* gQ = grad + off_Q(d);
    k_proj<<<gp, kThr, 0, st>>>(d, Q, v + (size_t)d.L * vs, un, unm1, rho, s_out, nullptr, target, dout, dloss, B);
    k_proj_back<<<gp, kThr, 0, st>>>(d, Q, v + (size_t)d.L * vs, dout, dv, part, B);
    k_sum_rows<<<1, 64, 0, st>>>(part, (int)(gp.x * gp.y), d.C + 1, gQ);
    for (int l = d.L - 1; l >= 0; l--) {
        const float* L = params + off_layer(d, l);
        const float* W = L;
        const float* R = L + d.C * d.C + d.C;
        float* gL = grad + off_layer(d, l);
        float* gR = gL + d.C * d.C + d.C;
        const int nrow = d.C * d.C + d.C;
        // pointwise part: dz, dv2 = W^T dz, then dW, db
        k_layer_back<<<gp, kThr, 0, st>>>(d, W, z + (size_t)l * vs, dv, dz, dv2, B);
        k_wgrad<<<dim3(d.n0, B), kThr, 0, st>>>(d, dz, v + (size_t)l * vs, part);
        k_sum_rows<<<(nrow + 63) / 64, 64, 0, st>>>(part, d.n0 * B, nrow, gL);
        // spectral part: DFT(dz) -> dG (weights applied in k_mix_back), dR, dF, dv2 += IDFT(dF)
        k_dft_rows<<<B * d.C * d.n0, kThr, sizeof(float2) * d.n1, st>>>(d, dz, T);
        k_dft_cols<<<B * d.C, d.M, sizeof(float2) * d.n0, st>>>(d, T, dZ);
        k_mix_back<<<(d.C * d.M + kThr - 1) / kThr, kThr, 0, st>>>(d, R, F + (size_t)l * B * d.C * d.M, dZ, gR, dF, B);
        k_idft_cols<<<dim3((d.n0 * d.M1 + kThr - 1) / kThr, B * d.C), kThr, sizeof(float2) * d.n0, st>>>(d, dF, U);
        k_idft_rows_add<<<dim3(d.n0, B * d.C), kThr, sizeof(float2) * d.n1, st>>>(d, U, dv2, B * d.C);
        float* t = dv;
        dv = dv2;
        dv2 = t;
    }
    k_lift_back<<<gp, kThr, 0, st>>>(d, a, dv, part, B);
    CK(cudaMemsetAsync(sums, 0, sizeof(float) * 3 * d.C, st));
    k_sum_rows<<<(3 * d.C + 63) / 64, 64, 0, st>>>(part, (int)(gp.x * gp.y), 3 * d.C, sums);
    k_lift_scatter<<<1, 32, 0, st>>>(sums, grad, d.C);
    CK(cudaGetLastError());
    if (loss) CK(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return PAGD_OK;
}

pagd_status sno_adam_step(sno_net* s, float* params, const float* grad, float* m, float* v, int t, double lr) {
    if (!s || !params || !grad || !m || !v || t < 1 || !(lr > 0.0)) return PAGD_EINVAL;
    const long long n = (long long)param_count(s->d);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<(unsigned)((n + kThr - 1) / kThr), kThr, 0, (cudaStream_t)s->stream>>>(params, grad, m, v, n, (float)lr,
                                                                                   b1, b2, 1e-8f, c1, c2);
    CK(cudaGetLastError());
    return PAGD_OK;
}

pagd_status sno_round_bf16(sno_net* s, const float* master, float* weights) {
    if (!s || !master || !weights) return PAGD_EINVAL;
    const long long n = (long long)param_count(s->d);
    k_round_bf16<<<(unsigned)((n + kThr - 1) / kThr), kThr, 0, (cudaStream_t)s->stream>>>(master, weights, n);
    CK(cudaGetLastError());
    return PAGD_OK;
}

const char* sno_last_error(const sno_net* s) { return s ? s->err.c_str() : "null network"; }

void sno_destroy(sno_net* s) { delete s; }

}  // extern "C"
