// cluster.cuh -- cluster-resident PAGD iterations for small square 2D grids.
//
// On an n x n grid with n = 64, 128 or 256 a device-wide phase has only n / 2
// row units and n / 2 + 1 columns, one per warp on a fraction of the SMs, so
// each phase of the iteration (Algorithm 2: row pass, column pass) costs the
// latency of one unit plus a device-wide barrier.  Here the iterations of one
// base point run inside one thread-block cluster of n / 16 CTAs instead: every
// CTA keeps 16 rows of the physical corrections delta_i, delta_{i-1} and 8
// columns of the spectral states in its shared memory, the transposes between
// the row and the column passes go through distributed shared memory, and the
// phases are separated by cluster barriers.  Nothing of the iteration touches
// global memory except the base fields VBt (and, FCH, Lap VB) that the row
// pass reads, and the norms that the control machine records.
//
// Work per CTA (rank r of the cluster, one unit per warp):
//   row pass     -- row pairs (16 r + 2 w, 16 r + 2 w + 1), w = 0..7;
//   column pass  -- columns k1 = 8 r + w of the half spectrum, except that
//                   unit (r = 0, w = 0) takes columns 0 and n / 2 together:
//                   both are real sequences along the first axis (the row
//                   DFT of real rows at k1 = 0 and n / 2), so they share one
//                   complex transform (z = a + i b, separated by Hermitian
//                   symmetry), and the n / 2 + 1 columns make exactly 8 units
//                   per CTA.
// The arithmetic per point is that of the device-wide phases phase_R and
// phase_CI (same formulas, same iteration precision); the decision after each
// evaluation is ctl_eval, the same function the device-wide control machine
// uses, on the same norm.  When the decision is anything but "iterate on", the
// loop writes its state back to the workspace and hands the control state to
// the device-wide machine, which takes the decision again after the next
// device barrier.
#pragma once
#include "solver.cuh"

#ifndef PAGD_EMU
#include <cooperative_groups.h>
#else
#include <vector>
#endif

namespace pagd {

#ifndef PAGD_EMU
__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#endif

constexpr int kClUnits = 8;              // row pairs and column units per CTA
constexpr int kClRows = 2 * kClUnits;    // rows per CTA
constexpr int kClSlots = kClUnits + 1;   // column slots (slot 8 of CTA 0: column n / 2)
constexpr int kClMaxK = 2;               // fields per pass (FCH)

// cluster size for a fixed line length (0: no cluster mode)
__host__ __device__ constexpr int cl_size_for(int nf) {
    return (nf == 64 || nf == 128 || nf == 256) ? nf / kClRows : 0;
}

// Layout of a CTA's cluster region (byte offsets after the twiddle tables;
// tsz = sizeof(T), K fields per pass).  The two exchange buffers are laid out
// so that what one warp sends to one CTA is a contiguous run (eight 16-byte
// chunks from a row pair, sixteen 8-byte values from a column), and their
// strides are padded so that the local reads spread over all banks:
//   nbx  row pass -> column pass, [pair p][field][slot][rr] (x0 = 2 p + rr),
//        ps complex values per pair;
//   dbx  column pass -> row pass, [k1][field][local row], qs values per k1.
struct ClOff {
    unsigned d[2], s[2], nbx, dbx, scr, part, qc, end;
    int ps, qs;
};
__host__ __device__ inline unsigned cl_take(size_t& q, size_t b) {
    const size_t r = q;
    q += (b + 15) & ~(size_t)15;
    return (unsigned)r;
}
__host__ __device__ inline ClOff cl_offsets(int nf, int K, int tsz) {
    const size_t c = 2 * (size_t)tsz;
    const size_t pitch = (size_t)nf + 2;
    ClOff o;
    o.ps = K * 2 * kClSlots + (K == 2 ? 2 : 0);
    o.qs = K * kClRows + 6;
    size_t q = 0;
    o.d[0] = cl_take(q, (size_t)kClRows * nf * tsz);          // delta, rows x n
    o.d[1] = cl_take(q, (size_t)kClRows * nf * tsz);
    o.s[0] = cl_take(q, (size_t)kClSlots * nf * c);           // delta_hat, slots x n
    o.s[1] = cl_take(q, (size_t)kClSlots * nf * c);
    o.nbx = cl_take(q, (size_t)(nf / 2) * o.ps * c);
    o.dbx = cl_take(q, (size_t)(nf / 2 + 1) * o.qs * c);
    o.scr = cl_take(q, (size_t)kClUnits * 2 * K * pitch * c);  // two K-line buffers per unit
    o.part = cl_take(q, (size_t)kClUnits * 2 * sizeof(double));
    o.qc = cl_take(q, 16 * sizeof(double));
    o.end = (unsigned)q;
    return o;
}

// A CTA's view of the cluster: its rank, the cluster size and, for a pointer
// into its own cluster region, the same address in another CTA's.
struct ClCtx {
    char* base;
    int rank, cs;
#ifdef PAGD_EMU
    char* const* peers;
    template <class X> X* peer(X* p, int r) const { return (X*)(peers[r] + ((char*)p - base)); }
#else
    template <class X> __device__ X* peer(X* p, int r) const {
        return cooperative_groups::this_cluster().map_shared_rank(p, (unsigned)r);
    }
#endif
};

// column k1 of unit u of CTA `rank` (unit 0 of rank 0 also holds column n / 2)
__host__ __device__ inline int cl_col(int rank, int u) { return rank * kClUnits + u; }
// owner CTA and slot of half-spectrum column k (k <= n / 2)
__host__ __device__ inline int cl_owner(int k, int half) { return k < half ? k / kClUnits : 0; }
__host__ __device__ inline int cl_slot(int k, int half) { return k < half ? k % kClUnits : kClUnits; }

// the per-loop constants (betas, scheme coefficients, wavenumber scales) in
// the iteration precision, computed once per loop entry
template <class T> struct ClConst {
    T m2, b0, b2, b4, aim, c0, e2, e4, ts, tau, eta1, eta2, k0s, k1s;
};

template <class T>
__device__ __forceinline__ ClConst<T> cl_const(const Params& P, const Ctl& c) {
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    ClConst<T> q;
    q.m2 = (T)B.m2;
    q.b0 = (T)B.b0;
    q.b2 = (T)B.b2;
    q.b4 = (T)B.b4;
    q.aim = (T)(k.Ai / P.M);
    q.c0 = (T)(1.0 - P.eps);
    q.e2 = (T)(P.eps * P.eps);
    q.e4 = q.e2 * q.e2;
    q.ts = (T)k.ts;
    q.tau = (T)P.tau;
    q.eta1 = (T)P.eta1;
    q.eta2 = (T)P.eta2;
    q.k0s = (T)P.k0sq;
    q.k1s = (T)P.k1sq;
    return q;
}

// kappa at (k1, k0) of an n x n grid from the scales, as kappa_t computes it
template <class T, int NF>
__device__ __forceinline__ T cl_kappa(const ClConst<T>& q, int k1, int k0) {
    const int r0 = (k0 <= (NF >> 1)) ? k0 : k0 - NF;
    return q.k1s * (T)(k1 * k1) + q.k0s * (T)(r0 * r0);
}

// the column-pass point of phase_CI: from the spectral state (sc, sp, g0) and
// the forward column DFT of the row pass's nonlinear terms (in) to the new
// spectral state sn and the outputs d_hat (and, FCH, the spectrum of Lap ybar)
template <class T>
__device__ __forceinline__ void cl_ci_point(const ClConst<T>& q, bool pfc, T l, T ln, T kap, cx<T> sc, cx<T> sp,
                                            cx<T> g0, const cx<T>* in, cx<T>& sn, cx<T>* out) {
    using C = cx<T>;
    const C yh = C{sc.x + l * (sc.x - sp.x), sc.y + l * (sc.y - sp.y)};
    C d{(T)0, (T)0};
    if (kap != (T)0) {
        const T ik = (T)1 / kap;
        const T il = (T)-1 / (q.m2 * ik + q.b0 + q.b2 * kap + q.b4 * kap * kap);
        if (pfc) {
            const T m = q.aim * ik + q.c0 - (T)2 * kap + kap * kap;
            d.x = il * (g0.x + m * yh.x + in[0].x);
            d.y = il * (g0.y + m * yh.y + in[0].y);
        } else {
            const T m = q.aim * ik + q.e4 * kap * kap;
            const T e2k = q.e2 * kap;
            d.x = il * (g0.x + m * yh.x + e2k * in[0].x + in[1].x);
            d.y = il * (g0.y + m * yh.y + e2k * in[0].y + in[1].y);
        }
    }
    sn = C{yh.x + q.ts * d.x, yh.y + q.ts * d.y};
    out[0] = d;
    if (!pfc) {
        const T f = -kap;
        out[1] = C{f * (sn.x + ln * (sn.x - sc.x)), f * (sn.y + ln * (sn.y - sc.y))};
    }
}

// two neighbouring complex values (rows 2 p, 2 p + 1 of one column) as one
// 16-byte store where the element type allows it
__device__ __forceinline__ void cl_st2(float2* p, float2 a, float2 b) {
#ifdef PAGD_EMU
    p[0] = a;
    p[1] = b;
#else
    *(float4*)p = make_float4(a.x, a.y, b.x, b.y);
#endif
}
__device__ __forceinline__ void cl_st2(double2* p, double2 a, double2 b) {
    p[0] = a;
    p[1] = b;
}

// Column pass of iteration it (phase_CI) on this CTA's units.
template <class T, int NF>
__device__ __forceinline__ void cl_col_pass(const Params& P, const Ctl& c, const ClCtx& x, const ClOff& o,
                                            const Tw& tw, int warp, int nwarps, int lane) {
    using C = cx<T>;
    constexpr int LOGN = ilog2c(NF), HALF = NF / 2, PITCH = NF + 2, E = NF / kWarp;
    const int K = k_iter(P.model);
    const bool pfc = P.model == M_PFC;
    const ClConst<T> q = *(const ClConst<T>*)(x.base + o.qc);
    const int it = c.it;
    const T l = (T)lam_at(P, it), ln = (T)lam_at(P, it + 1);
    C* S0 = (C*)(x.base + o.s[it & 1]);        // delta_hat_it
    C* S1 = (C*)(x.base + o.s[(it - 1) & 1]);  // delta_hat_{it-1}, overwritten with delta_hat_{it+1}
    const C* G0 = (const C*)P.C0;              // the base gradient (global, L2-resident)
    const C* NBX = (const C*)(x.base + o.nbx);
    C* DBX = (C*)(x.base + o.dbx);
    const int ps = o.ps, qs = o.qs;
    for (int u = warp; u < kClUnits; u += nwarps) {
        C* b0 = (C*)(x.base + o.scr) + (size_t)u * 2 * K * PITCH;
        C* b1 = b0 + (size_t)K * PITCH;
        const bool pair = (x.rank == 0 && u == 0);
        const int k1 = cl_col(x.rank, u);
        // the base gradient of the unit's column, issued before the transform
        C g0v[E];
        if (!pair) {
#pragma unroll
            for (int i = 0; i < E; i++) g0v[i] = G0[(size_t)k1 * NF + lane + kWarp * i];
        }
        // gather the unit's lines (columns 0 and n/2 packed as z = a + i b: both real)
        for (int f = 0; f < K; f++)
#pragma unroll
            for (int i = 0; i < E; i++) {
                const int x0 = lane + kWarp * i;
                const C* src = NBX + (size_t)(x0 >> 1) * ps + (size_t)(f * kClSlots) * 2 + (x0 & 1);
                b0[(size_t)f * PITCH + x0] = pair ? C{src[0].x, src[2 * kClUnits].x} : src[2 * u];
            }
        const int r = fft_lines_fixed<-1, T, LOGN, kClMaxK>(b0, b1, PITCH, K, tw_of<T>(tw), tw.log, lane);
        C* Xr = r ? b1 : b0;
        C* Xf = r ? b0 : b1;
        if (!pair) {
            const size_t sb = (size_t)u * NF;
#pragma unroll
            for (int i = 0; i < E; i++) {
                const int k0 = lane + kWarp * i;
                C in[kClMaxK], out[kClMaxK];
                for (int f = 0; f < K; f++) in[f] = Xr[(size_t)f * PITCH + k0];
                C sn;
                cl_ci_point<T>(q, pfc, l, ln, cl_kappa<T, NF>(q, k1, k0), S0[sb + k0], S1[sb + k0], g0v[i], in, sn,
                               out);
                S1[sb + k0] = sn;
                for (int f = 0; f < K; f++) Xr[(size_t)f * PITCH + k0] = out[f];
            }
        } else {
            // columns 0 and n/2 from Z = A + i B: A(k) = (Z(k) + conj Z(-k)) / 2,
            // B(k) = (Z(k) - conj Z(-k)) / (2 i); one lane takes k0 and -k0, so
            // the outputs can be made Hermitian (the part the row pass keeps)
            // and packed back in place as A' + i B'
            const size_t sh = (size_t)kClUnits * NF;  // slot of column n/2
            for (int k0 = lane; k0 <= HALF; k0 += kWarp) {
                const int km = (NF - k0) & (NF - 1);
                C A[2][kClMaxK], Bv[2][kClMaxK];
                for (int f = 0; f < K; f++) {
                    const C z = Xr[(size_t)f * PITCH + k0], zm = Xr[(size_t)f * PITCH + km];
                    A[0][f] = C{(T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y)};
                    Bv[0][f] = C{(T)0.5 * (z.y + zm.y), (T)0.5 * (zm.x - z.x)};
                    A[1][f] = C{A[0][f].x, -A[0][f].y};  // value at -k0
                    Bv[1][f] = C{Bv[0][f].x, -Bv[0][f].y};
                }
                C oa[2][kClMaxK], ob[2][kClMaxK];
                const int kk[2] = {k0, km};
                const int ns = (km == k0) ? 1 : 2;  // k0 = 0 and n/2 are their own mirrors
                for (int s = 0; s < ns; s++) {
                    const size_t ia = (size_t)kk[s], ib = sh + (size_t)kk[s];
                    C sn;
                    cl_ci_point<T>(q, pfc, l, ln, cl_kappa<T, NF>(q, 0, kk[s]), S0[ia], S1[ia], G0[ia], A[s], sn,
                                   oa[s]);
                    S1[ia] = sn;
                    cl_ci_point<T>(q, pfc, l, ln, cl_kappa<T, NF>(q, HALF, kk[s]), S0[ib], S1[ib],
                                   G0[(size_t)HALF * NF + kk[s]], Bv[s], sn, ob[s]);
                    S1[ib] = sn;
                }
                if (ns == 1)
                    for (int f = 0; f < K; f++) {
                        oa[1][f] = oa[0][f];
                        ob[1][f] = ob[0][f];
                    }
                for (int f = 0; f < K; f++) {
                    // Hermitian parts a(k0) = (o(k0) + conj o(-k0)) / 2, a(-k0) = conj a(k0)
                    const C a{(T)0.5 * (oa[0][f].x + oa[1][f].x), (T)0.5 * (oa[0][f].y - oa[1][f].y)};
                    const C b{(T)0.5 * (ob[0][f].x + ob[1][f].x), (T)0.5 * (ob[0][f].y - ob[1][f].y)};
                    // w = a + i b at k0, conj(a) + i conj(b) at -k0
                    Xr[(size_t)f * PITCH + k0] = C{a.x - b.y, a.y + b.x};
                    Xr[(size_t)f * PITCH + km] = C{a.x + b.y, b.x - a.y};
                }
            }
        }
        const int r2 = fft_lines_fixed<+1, T, LOGN, kClMaxK>(Xr, Xf, PITCH, K, tw_of<T>(tw), tw.log, lane);
        const C* Yr = r2 ? Xf : Xr;
        // scatter to the row owners: DBX[k1][f][local row], 16 consecutive rows
        // per owner CTA
#pragma unroll 2
        for (int i = 0; i < E; i++) {
            const int x0 = lane + kWarp * i;
            C* dst = x.peer(DBX, x0 / kClRows) + (x0 % kClRows);
            for (int f = 0; f < K; f++) {
                const C w = Yr[(size_t)f * PITCH + x0];
                if (!pair) {
                    dst[(size_t)k1 * qs + f * kClRows] = w;
                } else {
                    dst[f * kClRows] = C{w.x, (T)0};
                    dst[(size_t)HALF * qs + f * kClRows] = C{w.y, (T)0};
                }
            }
        }
        warp_sync();
    }
}

// Row pass of iteration it (phase_R): delta_it = ybar_{it-1} + theta_v s d_{it-1},
// ||d_{it-1}||_inf and sum delta_it (per unit, into the partials), the
// nonlinear terms at ybar_it and their forward row DFT, scattered to the
// column owners.
template <class T, int NF>
__device__ __forceinline__ void cl_row_pass(const Params& P, const Ctl& c, const ClCtx& x, const ClOff& o,
                                            const Tw& tw, int warp, int nwarps, int lane) {
    using C = cx<T>;
    constexpr int LOGN = ilog2c(NF), HALF = NF / 2, PITCH = NF + 2, E = NF / kWarp;
    constexpr int EH = (HALF + 1 + kWarp - 1) / kWarp;
    const int K = k_iter(P.model);
    const bool pfc = P.model == M_PFC;
    const ClConst<T> q = *(const ClConst<T>*)(x.base + o.qc);
    const int it = c.it;
    const T lp = (T)lam_at(P, it - 1), l = (T)lam_at(P, it);
    T* dcur = (T*)(x.base + o.d[it & 1]);          // delta_{it-2} -> delta_it
    const T* dprev = (const T*)(x.base + o.d[(it - 1) & 1]);
    const T* vbt = (const T*)P.VBt;
    const T* lbt = (const T*)P.LBt;
    C* NBX = (C*)(x.base + o.nbx);
    const C* DBX = (const C*)(x.base + o.dbx);
    double* part = (double*)(x.base + o.part);
    const T iscale = (T)P.inv_npts;
    const int ps = o.ps, qs = o.qs;
    for (int u = warp; u < kClUnits; u += nwarps) {
        const int lr0 = 2 * u;                       // local rows lr0, lr0 + 1
        const int r0 = x.rank * kClRows + lr0;       // global rows
        C* b0 = (C*)(x.base + o.scr) + (size_t)u * 2 * K * PITCH;
        C* b1 = b0 + (size_t)K * PITCH;
        // base fields of the two rows (global, L2-resident): issued first
        T vb[2 * E], lb[2 * E];
#pragma unroll
        for (int i = 0; i < E; i++)
#pragma unroll
            for (int rr = 0; rr < 2; rr++) {
                const long long p = (long long)(r0 + rr) * NF + lane + kWarp * i;
                vb[2 * i + rr] = vbt[p];
                lb[2 * i + rr] = pfc ? (T)0 : lbt[p];
            }
        // unpack the half spectra of the two rows into one complex line per field
        for (int f = 0; f < K; f++)
#pragma unroll
            for (int i = 0; i < E; i++) {
                const int xx = lane + kWarp * i;
                const int k = (xx <= HALF) ? xx : NF - xx;
                const C* src = DBX + (size_t)k * qs + f * kClRows + lr0;
                C A = src[0], B = src[1];
                if (xx == 0 || xx == HALF) {
                    A.y = 0;
                    B.y = 0;
                }
                b0[(size_t)f * PITCH + xx] = (xx <= HALF) ? C{A.x - B.y, A.y + B.x} : C{A.x + B.y, B.x - A.y};
            }
        const int r = fft_lines_fixed<+1, T, LOGN, kClMaxK>(b0, b1, PITCH, K, tw_of<T>(tw), tw.log, lane);
        C* Xr = r ? b1 : b0;
        C* Xf = r ? b0 : b1;
        T amax = (T)0;
        double asum = 0.0;
#pragma unroll
        for (int i = 0; i < E; i++)
#pragma unroll
            for (int rr = 0; rr < 2; rr++) {
                const int xx = lane + kWarp * i;
                const size_t lp_ = (size_t)(lr0 + rr) * NF + xx;
                T in[kClMaxK];
                for (int f = 0; f < K; f++) {
                    const C z = Xr[(size_t)f * PITCH + xx];
                    in[f] = (rr ? z.y : z.x) * iscale;
                }
                const T dp = dprev[lp_], dpp = dcur[lp_];
                const T dd = in[0];
                const T de = dp + lp * (dp - dpp) + q.ts * dd;
                dcur[lp_] = de;
                const T ad = fabs(dd);
                amax = (ad > amax || ad != ad) ? ad : amax;
                asum += (double)de;
                const T y = de + l * (de - dp);
                const T b = vb[2 * i + rr];
                T out[kClMaxK];
                if (pfc) {
                    out[0] = y * ((T)3 * b * b + (T)3 * b * y + y * y);
                } else {
                    const T ly = in[1];
                    const T f1b = dF1(b, q.tau), f2b = dF2(b, q.tau);
                    const T df1 = y * ((T)3 * b * b + (T)3 * b * y + y * y + q.tau * ((T)2 * b + y) - (T)1);
                    const T df2 = y * ((T)6 * b + (T)3 * y + (T)2 * q.tau);
                    const T f1n = f1b + df1, f2n = f2b + df2;
                    out[0] = df1;
                    out[1] = -q.e2 * (df2 * lb[2 * i + rr] + (f2n - q.eta1) * ly) + df2 * f1n + (f2b - q.eta2) * df1;
                }
                for (int g = 0; g < K; g++) {
                    C* qq = Xr + (size_t)g * PITCH + xx;
                    if (rr) qq->y = out[g];
                    else qq->x = out[g];
                }
            }
        const int r2 = fft_lines_fixed<-1, T, LOGN, kClMaxK>(Xr, Xf, PITCH, K, tw_of<T>(tw), tw.log, lane);
        const C* Yr = r2 ? Xf : Xr;
        const T hf = (T)0.5;
        // scatter to the column owners: NBX[pair][f][slot][rr], eight slots of
        // one owner side by side
        const size_t pb = (size_t)(r0 >> 1) * ps;
        for (int f = 0; f < K; f++)
#pragma unroll
            for (int i = 0; i < EH; i++) {
                const int k = lane + kWarp * i;
                if (k <= HALF) {
                    const C zk = Yr[(size_t)f * PITCH + k];
                    const C zn = Yr[(size_t)f * PITCH + ((NF - k) & (NF - 1))];
                    C* dst = x.peer(NBX, cl_owner(k, HALF)) + pb + (size_t)(f * kClSlots + cl_slot(k, HALF)) * 2;
                    cl_st2(dst, C{hf * (zk.x + zn.x), hf * (zk.y - zn.y)}, C{hf * (zk.y + zn.y), hf * (zn.x - zk.x)});
                }
            }
        const T wm = warp_max(amax);
        const double ws = warp_sum(asum);
        if (lane == 0) {
            part[2 * u] = (double)wm;
            part[2 * u + 1] = ws;
        }
        warp_sync();
    }
}

// The cluster's ||d||_inf and sum delta of the evaluation just made: every
// warp reduces all CTAs' unit partials in the same order, so every thread of
// the cluster holds the same two values.
__device__ __forceinline__ void cl_reduce(const ClCtx& x, const ClOff& o, int lane, double& nrm, double& sum) {
    const int n = x.cs * kClUnits;
    double m = 0.0, s = 0.0;
    for (int j = lane; j < n; j += kWarp) {
        const double* p = x.peer((double*)(x.base + o.part), j / kClUnits) + 2 * (j % kClUnits);
        const double a = p[0];
        m = (a > m || a != a) ? a : m;
        s += p[1];
    }
    nrm = warp_max(m);
    sum = warp_sum(s);
}

// Load the iteration state of this CTA's rows and columns from the workspace
// (entry at phase CI of iteration c.it) / write it back (exit after phase RI).
template <class T, int NF>
__device__ __forceinline__ void cl_transfer(const Params& P, const Ctl& c, const ClCtx& x, const ClOff& o,
                                            bool load) {
    using C = cx<T>;
    constexpr int HALF = NF / 2;
    const int K = k_iter(P.model);
    const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
    const long long rowbase = (long long)x.rank * kClRows * NF;
    for (int b = 0; b < 2; b++) {
        T* d = (T*)(x.base + o.d[b]);
        T* g = (T*)P.DD[b] + rowbase;
        for (int i = tid; i < kClRows * NF; i += nt) {
            if (load) d[i] = g[i];
            else g[i] = d[i];
        }
    }
    const int nslot = (x.rank == 0) ? kClSlots : kClUnits;
    C* nbx = (C*)(x.base + o.nbx);
    for (int sl = 0; sl < nslot; sl++) {
        const int k1 = (sl == kClUnits) ? HALF : cl_col(x.rank, sl);
        const size_t gi = (size_t)k1 * NF, li = (size_t)sl * NF;
        for (int b = 0; b < 2; b++) {
            C* ls = (C*)(x.base + o.s[b]) + li;
            C* gs = (C*)P.SS[b] + gi;
            for (int i = tid; i < NF; i += nt) {
                if (load) ls[i] = gs[i];
                else gs[i] = ls[i];
            }
        }
        C* gn = (C*)P.NB + (size_t)k1 * P.rows;
        for (int f = 0; f < K; f++)
            for (int i = tid; i < NF; i += nt) {
                C* ln = nbx + (size_t)(i >> 1) * o.ps + (size_t)(f * kClSlots + sl) * 2 + (i & 1);
                if (load) *ln = gn[(size_t)f * P.H + i];
                else gn[(size_t)f * P.H + i] = *ln;
            }
    }
    if (load && threadIdx.x == 0) *(ClConst<T>*)(x.base + o.qc) = cl_const<T>(P, c);
}

// The loop bookkeeping after a row pass (thread 0 of each CTA, on the CTA's
// copy of the control state): the evaluation just made is phase RI of
// iteration it + 1; its norm is recorded (rank 0 only) and the decision taken.
// Returns true to iterate on.
template <class T>
__device__ __forceinline__ bool cl_decide(const Params& P, Ctl& cc, double nrm, double sum, bool writer) {
    cc.ph = PH_RI;
    cc.it++;
    const int bank = cc.step & 1;
    if (writer) {
        P.norms[(size_t)bank * P.nslots + cc.ev] = dbl_bits(nrm);
        P.sums[(size_t)bank * P.nslots + cc.ev] = sum;
    }
    Ctl t = cc;
    ctl_eval<T>(P, t, nrm);
    if (t.ph != PH_CI) return false;
    cc = t;
    return true;
}

#ifdef PAGD_EMU
// The same loop in the CPU emulation: the cluster's CTAs run each pass in
// turn (one thread per warp), each with its own shared-memory region.
template <class T, int NF>
void cluster_iterate_emu(const Params& P, const Ctl& c, const Tw& tw) {
    if constexpr (cl_size_for(NF) == 0) {
        return;
    } else {
        const int cs = P.cl;
        const ClOff o = cl_offsets(NF, k_iter(P.model), (int)sizeof(T));
        std::vector<std::vector<char>> mem((size_t)cs, std::vector<char>((size_t)o.end + 64));
        std::vector<char*> bases((size_t)cs);
        for (int r = 0; r < cs; r++) bases[(size_t)r] = (char*)(((uintptr_t)mem[(size_t)r].data() + 15) & ~(uintptr_t)15);
        auto ctx = [&](int r) {
            ClCtx x;
            x.base = bases[(size_t)r];
            x.rank = r;
            x.cs = cs;
            x.peers = bases.data();
            return x;
        };
        Ctl cc = c;
        for (int r = 0; r < cs; r++) cl_transfer<T, NF>(P, cc, ctx(r), o, true);
        for (;;) {
            for (int r = 0; r < cs; r++) cl_col_pass<T, NF>(P, cc, ctx(r), o, tw, 0, 1, 0);
            cc.it++;
            for (int r = 0; r < cs; r++) cl_row_pass<T, NF>(P, cc, ctx(r), o, tw, 0, 1, 0);
            double nrm, sum;
            cl_reduce(ctx(0), o, 0, nrm, sum);
            cc.it--;
            if (!cl_decide<T>(P, cc, nrm, sum, true)) break;
        }
        for (int r = 0; r < cs; r++) cl_transfer<T, NF>(P, cc, ctx(r), o, false);
        *(Ctl*)P.lctl = cc;
    }
}
#endif

#ifndef PAGD_EMU
// The loop on the device: CTAs of cluster 0 only (the others go straight to
// the device barrier).  c: the control state at phase CI (shared memory);
// wsm: the CTA's warp region; ntr: trace records so far (block 0, thread 0).
// Each CTA keeps its copy of the control state in shared memory; thread 0
// advances it and the others read the few fields the passes need.
template <class T, int NF>
__device__ __noinline__ void cluster_iterate(const Params& P, const Ctl& c, const Tw& tw, char* wsm, int* ntr) {
    if constexpr (cl_size_for(NF) == 0) {
        return;
    } else {
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        if (blockIdx.x >= (unsigned)P.cl) return;  // cluster 0 is blocks 0 .. P.cl - 1
        __shared__ Ctl cc;
        __shared__ int more;
        const ClOff o = cl_offsets(NF, k_iter(P.model), (int)sizeof(T));
        ClCtx x;
        x.base = wsm;
        x.rank = (int)cl.block_rank();
        x.cs = (int)cl.num_blocks();
        const int warp = (int)(threadIdx.x / kWarp), nwarps = (int)(blockDim.x / kWarp), lane = (int)(threadIdx.x % kWarp);
        const bool writer = x.rank == 0 && threadIdx.x == 0;
        if (threadIdx.x == 0) cc = c;
        __syncthreads();
        cl_transfer<T, NF>(P, cc, x, o, true);
        cl.sync();
        for (;;) {
            cl_col_pass<T, NF>(P, cc, x, o, tw, warp, nwarps, lane);
            cl.sync();
            if (writer && P.trace && *ntr < P.trace_cap) {
                P.trace[2 * *ntr] = (unsigned long long)PH_CI;
                P.trace[2 * *ntr + 1] = gtimer_ns();
                (*ntr)++;
            }
            if (threadIdx.x == 0) cc.it++;  // the row pass belongs to iteration it + 1
            __syncthreads();
            cl_row_pass<T, NF>(P, cc, x, o, tw, warp, nwarps, lane);
            cl.sync();
            double nrm, sum;
            cl_reduce(x, o, lane, nrm, sum);
            if (writer && P.trace && *ntr < P.trace_cap) {
                P.trace[2 * *ntr] = (unsigned long long)PH_RI;
                P.trace[2 * *ntr + 1] = gtimer_ns();
                (*ntr)++;
            }
            if (threadIdx.x == 0) {
                cc.it--;  // cl_decide counts the iteration itself (case PH_CI of ctl_step)
                more = cl_decide<T>(P, cc, nrm, sum, writer) ? 1 : 0;
            }
            __syncthreads();
            // every CTA has read the partials before the next row pass writes them
            if (!more) break;
        }
        cl_transfer<T, NF>(P, cc, x, o, false);
        if (writer) *(Ctl*)P.lctl = cc;
        cl.sync();  // no CTA leaves while another may still read its shared memory
    }
}
#endif

}  // namespace pagd
