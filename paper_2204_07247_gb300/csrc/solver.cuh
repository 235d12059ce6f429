// solver.cuh -- the PAGD time step as one persistent cooperative kernel.
//
// One launch runs a "program" (a run of time steps, a DFT, an energy or a mass
// evaluation) as a sequence of phases separated by device-wide barriers.  Every
// CTA evaluates the same control state machine after each barrier, so all CTAs
// agree on the next phase without any host round trip.
//
// Phases are of two kinds, built from warp-owned lines (no CTA-wide barrier
// inside a phase) or, for phases with FP64 work on grids with fewer units than
// warps, from CTA-cooperative units (all warps of a CTA on one unit):
//   row pass    -- per unit of one or two rows: inverse x-DFT of K_in fields
//                  from the column-major half-spectrum buffer, a pointwise
//                  functor, forward x-DFT of K_out fields back to such a buffer;
//   column pass -- per half-spectrum column: forward y-DFT of K_in fields, a
//                  per-wavenumber functor, inverse y-DFT of K_out fields.
//
// The time step (Sec. 3.1.1, Sec. 3.4, Algorithm 2) is solved in a correction
// form: v = VB + delta, where v is the scheme argument breve u (u for BDF2,
// (u + u^n)/2 for MP, Eq. obj:MP), VB is the FP64 argument at the initial guess,
// and the iteration runs on delta in precision T.  With theta_v = 1 (BDF2) or
// 1/2 (MP) the PAGD recurrences in v are
//     ybar_i = delta_i + lambda_i (delta_i - delta_{i-1}),
//     delta_{i+1} = ybar_i + theta_v s d_i,
// where d_i = Lcal^{-1} r_i, r_i = -G'_N(y_i) (Eq. obj:G'), which is Algorithm 2
// rewritten with v = theta_v x + (1 - theta_v) u^n.  G'_N splits into an FP64
// base part C0 = G'_N at VB (computed once per base) and a correction that is
// linear in delta plus the nonlinear difference N(VB + delta) - N(VB), written
// so that every term is proportional to delta (no cancellation in FP32).
#pragma once
#include <type_traits>

#include "fft.cuh"

namespace pagd {

enum { M_PFC = 0, M_FCH = 1 };
enum { S_BDF2 = 0, S_MP = 1, S_LBDF2 = 2, S_LMP = 3 };
enum { P_FP64 = 0, P_MIXED = 1 };
enum { PROG_RUN = 0, PROG_FFT_FWD = 1, PROG_FFT_INV = 2, PROG_ENERGY = 3, PROG_MASS = 4,
       PROG_IMEX = 5, PROG_RHS = 6, PROG_EST = 7, PROG_BARRIER = 8, PROG_PASS = 9 };
enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENOCONV = 4, ST_EPRECOND = 5,
       ST_ENAN = 6, ST_ESTATE = 7, ST_ETIMEOUT = 8 };
enum { FLAG_PRECOND = 1 };

enum Phase {
    PH_B, PH_C, PH_D, PH_E, PH_R1, PH_CI, PH_RI, PH_ACCEPT, PH_FAIL,
    PH_FWD_R, PH_FWD_C, PH_INV_C, PH_INV_R, PH_EN_R, PH_EN_C, PH_EN_R2, PH_MASS,
    PH_IM_R0, PH_IM_C0, PH_IM_R1, PH_IM_C1, PH_IM_R2,
    PH_MF, PH_MI, PH_GS,
    PH_RH_R0, PH_RH_C0, PH_RH_R1, PH_RH_C1, PH_RH_R2, PH_EST,
    PH_NOP,  // an empty phase (barrier probe)
    PH_DONE
};

// device-resident scalars; zeroed by the host before every launch
struct Scal {
    unsigned long long bar_count;  // grid barrier arrivals (monotonic)
    int bar_error, flags;
    int status, steps_done, fail_step, ntrace;
    // averaged-Newton grid sums [bank][field]: banks 0 / 1 by step parity, 2 / 3
    // for the evaluations at a caller's initial guess (probe, re-run)
    double beta_sum[4][2];
    double red[4];
};

struct StepStat {
    int iters, status;
    double resid;
    int used_guess, pad;
};

constexpr int kMaxK = 3;        // fields per pass
// CTA size of the persistent kernels: up to 8 warps (255 registers each fill
// the register file); the launch picks as many as the warps' shared memory
// slices allow
constexpr int kMaxThreads = 256;

// scheme coefficients of one step (see compute_step_coeffs)
struct StepK {
    double a, b, c, thv, ts, Ai, rho, gun, thpc, m2;
};

struct Params {
    int model, scheme, precision, prog;
    // Grid n0 x nm x n1 (2D: nm = 1), n1 the last (fastest) axis.  The row
    // passes transform lines along the last axis: rows = n0 nm of them.  Their
    // half spectra are stored [field][k1][row] (H = h1 rows complex values per
    // field).  In 3D a middle pass transforms along the middle axis and stores
    // [field][k1][km][i0], so the column passes always see ncols = h1 nm
    // contiguous lines of length n0: line l = k1 nm + km.
    int n0, n1, logn0, logn1, h1, logtw;
    int nm, logm, rows, ncols;
    long long H;
    long long npts;
    double k0sq, k1sq, kmsq;  // (2 pi / L)^2 of the first, last and middle axes
    double cellvol;           // product of the spacings
    double eps, eta1, eta2, tau, M;
    double s;
    int n_eta, accel, max_iter, max_recheck, theta_mode;
    // the PFC FP32 iteration passes stage their inputs by asynchronous copies
    // (row_pass_staged / col_pass_staged; fixed line lengths)
    int stage;
    // PROG_PASS: the iteration pass it repeats (PH_RI, PH_CI, PH_MF, PH_MI)
    int pass;
    // the FP32 iteration passes run CTA-cooperative units (phase_R_coop /
    // phase_CI_coop; opt-in, single-instance launches, unstaged passes)
    int coop32;
    double lam[16];      // (1 - eta_j sqrt s) / (1 + eta_j sqrt s)
    double tol, dt, dt_prev0;
    int step0, nsteps, cur0, nslots;  // nslots: norm / sum slots per step parity
    double inv_npts;
    // step coefficients filled on the host: [0] the first step of the run
    // (n = 0), [1] the first step of this launch when n > 0 (previous step
    // dt_prev0), [2] every other step; the device never divides by dt
    StepK kc[3];
    long long warp_bytes;             // shared memory per warp
    // workspace
    double* U[2];
    double* VB;
    double* G64;
    void* VBt;
    void* LBt;
    void* DD[2];
    void* SS[2];
    void* C0;
    void* NB;
    void* DB;
    double2* CL64;
    double2* NB64;
    double2* DB64;
    // 3D only: the middle passes' output, input of the column passes
    void* X;
    double2* X64;
    // reference point of the incremental (FP32-transform) base evaluation: the
    // FP64 spectra of the last evaluated base VB (VR64: v, NR64: PFC v^3 / FCH
    // F'(v), P(v)), its FP64 Laplacian (LB64, FCH) and the last shift (YB)
    double2* VR64;
    double2* NR64;
    double2* WR64;  // FP64 spectrum of A_i v + g at the reference
    double2* GH64;  // FP64 spectrum of the step's history term g (fixed within a step)
    double* LB64;
    void* YB;
    int ref_valid, refresh;
    // the passes with an FP64 line run CTA-cooperative units (single-instance
    // launches with fixed line lengths only)
    int coop;
    // cluster-resident iterations (cluster.cuh): the cluster size (0: off) and
    // the control state the loop hands back to the device-wide machine (a Ctl)
    int cl;
    void* lctl;
    const double2* tw64;
    const float2* tw32;
    Scal* sc;
    double* mass;  // persistent {K, D, R}: mass excess since set_state, this step's change, and
                   // R, ||d_0||_inf of the last step started from the extrapolation (0: none)
    unsigned long long* trace;  // nullable: (phase, globaltimer) pairs, one per completed phase
    int trace_cap;
    unsigned long long* norms;
    double* sums;
    StepStat* stats;
    // caller's initial iterate for the first step of the run (nullable)
    const double* guess;
    // error-estimate program: uh = sum_j est_c[j] est_in[j] (nullable terms)
    const double* est_in[4];
    double est_c[4];
    // program input / output
    const double* in_real;
    double* out_real;
    const double2* in_spec;
    double2* out_spec;
};

struct Ctl {
    int ph, step, it, ev, lastev, cur, rech, fail, best_ev;
    int after, mk, m64;  // 3D middle pass: the phase after it, its fields, FP64 buffers
    int gok;             // GH64 holds this step's g_hat (an exact evaluation made it)
    int bsel;            // bank of the averaged-Newton sums of the current evaluation
    int gmode;           // caller's guess: 0 none, 1 at it (kept when its first direction is no
                         // larger than the record), 2 probing the extrapolation,
                         // 3 iterating from it, 4 iterating from the extrapolation
    double gnorm;        // ||d_0||_inf at the caller's guess
    int acc_used;        // the step pending acceptance started from the caller's guess
    // record of the extrapolation's first direction: evaluation rec_ev of bank
    // rec_bank was one; the next phase B / ACCEPT stores its norm (P.mass[2])
    int rec_pending, rec_ev, rec_bank;
    int acc, acc_cur, acc_it, acc_lastev, acc_ev, reb, ereb, inc, ref_ok, exact_done;
    double resid, base_nrm, best_nrm, acc_resid;
};

// FP32 iterations stop improving once ||d|| reaches about 1e-7 of the FP64
// direction at the base point (the FP32 rounding of C0); the base is moved
// before that floor is reached.
constexpr double kRebaseRatio = 1.0e-6;
constexpr int kStagnation = 12;

// Per-thread pass context: the twiddle tables exp(-2 pi i m / (1 << log))
// staged in shared memory, and how the work of the current phase of one
// instance is split among warps.  wr / wn: this warp's rank among the warps
// working on the instance and their number.  uhi < 0: units are dealt round
// robin by wr / wn (single-instance launches; the rank is CTA-major so that
// every SM gets a busy warp before any SM gets a second); else the warp owns
// the contiguous unit range [ulo, uhi) (batched launches).
struct Tw {
    const double2* t64;
    const float2* t32;
    int log;
    int wr, wn, ulo, uhi;
};

struct URange {
    int b, e, s;
};
__device__ __forceinline__ URange units_of(const Tw& t, int units) {
    if (t.uhi < 0) return URange{t.wr, units, t.wn};
    return URange{t.ulo, t.uhi < units ? t.uhi : units, 1};
}
// the one thread of the instance's warps that writes per-instance scalars
__device__ __forceinline__ bool leader(const Tw& t) { return t.wr == 0 && (threadIdx.x % kWarp) == 0; }
__device__ __forceinline__ long long thread_rank(const Tw& t) {
    return (long long)t.wr * kWarp + (long long)(threadIdx.x % kWarp);
}
__device__ __forceinline__ long long thread_count(const Tw& t) { return (long long)t.wn * kWarp; }
template <class T> __device__ __forceinline__ const cx<T>* tw_of(const Tw& t);
template <> __device__ __forceinline__ const cx<double>* tw_of<double>(const Tw& t) { return t.t64; }
template <> __device__ __forceinline__ const cx<float>* tw_of<float>(const Tw& t) { return t.t32; }

// ---------------------------------------------------------------- helpers


// Scheme coefficients a_n, b_n, c_n (Eqs. obj:BDF2, obj:MP; backward Euler /
// its IMEX version for the first BDF2 / LBDF2 step, Algorithm 3 caption), the
// weight theta_v of the new iterate in breve u, and the extrapolation ratio rho.
// Host side; the device reads the table P.kc.
inline StepK compute_step_coeffs(int scheme, int n, double dt, double dtp, double s, int theta_mode,
                                 double M) {
    StepK k;
    const bool bdf = (scheme == S_BDF2 || scheme == S_LBDF2);
    if (!bdf || n == 0) {
        k.a = 1.0 / dt; k.b = -1.0 / dt; k.c = 0.0;
    } else {
        k.a = 1.0 / dt + 1.0 / (dt + dtp);
        k.b = -1.0 / dt - 1.0 / dtp;
        k.c = 1.0 / dtp - 1.0 / (dt + dtp);
    }
    k.thv = (scheme == S_MP) ? 0.5 : 1.0;
    k.ts = k.thv * s;
    k.Ai = k.a / k.thv;
    k.rho = (n == 0) ? 0.0 : dt / dtp;
    k.gun = k.a * (1.0 - k.thv) / k.thv;
    k.thpc = (scheme == S_MP && theta_mode == 0) ? 0.5 : 1.0;
    k.m2 = k.a / M;
    return k;
}

inline void fill_step_table(Params& P) {
    P.kc[0] = compute_step_coeffs(P.scheme, 0, P.dt, P.dt, P.s, P.theta_mode, P.M);
    P.kc[1] = compute_step_coeffs(P.scheme, P.step0 > 0 ? P.step0 : 1, P.dt, P.dt_prev0, P.s, P.theta_mode, P.M);
    P.kc[2] = compute_step_coeffs(P.scheme, 1, P.dt, P.dt, P.s, P.theta_mode, P.M);
    P.inv_npts = 1.0 / (double)P.npts;
}

__host__ __device__ __forceinline__ const StepK& step_coeffs(const Params& P, int step) {
    const int n = P.step0 + step;
    return P.kc[n == 0 ? 0 : (step == 0 ? 1 : 2)];
}

struct Beta {
    double m2, b0, b2, b4;
};

// Averaged Newton constants (Sec. 3.4.1) from the grid sums over the argument
// of the initial guess of this step.
__device__ __forceinline__ Beta betas(const Params& P, const StepK& k, int bank) {
    Beta B;
    const double inv = P.inv_npts;
    B.m2 = k.m2;
    const double s0 = ldcg(&P.sc->beta_sum[bank][0]) * inv;
    if (P.model == M_PFC) {
        B.b0 = k.thpc * fabs(s0);
        B.b2 = -2.0 * k.thpc;
        B.b4 = k.thpc;
    } else {
        const double s2 = ldcg(&P.sc->beta_sum[bank][1]) * inv;
        const double e2 = P.eps * P.eps;
        B.b0 = k.thpc * fabs(s0);
        B.b2 = k.thpc * fabs(s2);
        B.b4 = k.thpc * e2 * e2;
    }
    return B;
}

__device__ __forceinline__ double lam_at(const Params& P, int i) {
    return P.accel ? P.lam[i % P.n_eta] : 0.0;
}

// last-axis wavenumber index of column-pass line l (l = k1 nm + km)
__host__ __device__ __forceinline__ int kl_of(const Params& P, int l) { return l >> P.logm; }

// kappa = |k|^2 at column-pass line l, first-axis index k0
__device__ __forceinline__ double kappa_at(const Params& P, int l, int k0) {
    const int k1 = l >> P.logm, km = l & (P.nm - 1);
    const int r0 = (k0 <= (P.n0 >> 1)) ? k0 : k0 - P.n0;
    const int rm = (km <= (P.nm >> 1)) ? km : km - P.nm;
    return P.k1sq * (double)k1 * (double)k1 + P.kmsq * (double)rm * (double)rm +
           P.k0sq * (double)r0 * (double)r0;
}

// kappa in the iteration precision (FP32 iterations carry no FP64 arithmetic)
template <class T> __device__ __forceinline__ T kappa_t(const Params& P, int l, int k0) {
    const int k1 = l >> P.logm, km = l & (P.nm - 1);
    const int r0 = (k0 <= (P.n0 >> 1)) ? k0 : k0 - P.n0;
    const int rm = (km <= (P.nm >> 1)) ? km : km - P.nm;
    return (T)P.k1sq * (T)(k1 * k1) + (T)P.kmsq * (T)(rm * rm) + (T)P.k0sq * (T)(r0 * r0);
}

// index of half-spectrum entry (line l, k0) in the row-major API layout
// n0 x nm x h1
__device__ __forceinline__ long long api_spec_index(const Params& P, int l, int k0) {
    const int k1 = l >> P.logm, km = l & (P.nm - 1);
    return ((long long)k0 * P.nm + km) * P.h1 + k1;
}

// double well derivatives, expanded: F'(z) = (z^2 - 1)(z + tau),
// F''(z) = 3 z^2 + 2 tau z - 1, F'''(z) = 6 z + 2 tau, and
// F(z) = z^4/4 + tau z^3/3 - z^2/2 - tau z + (1/2 - 4 tau/3)/2.
template <class T> __device__ __forceinline__ T dF1(T z, T tau) { return (z * z - (T)1) * (z + tau); }
template <class T> __device__ __forceinline__ T dF2(T z, T tau) { return (T)3 * z * z + (T)2 * tau * z - (T)1; }
template <class T> __device__ __forceinline__ T dF3(T z, T tau) { return (T)6 * z + (T)2 * tau; }
__device__ __forceinline__ double Fwell(double z, double tau) {
    return 0.25 * z * z * z * z + tau * z * z * z / 3.0 - 0.5 * z * z - tau * z +
           0.5 * (0.5 - 4.0 * tau / 3.0);
}

__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

// Grid-wide reductions: every warp reduces its lanes with shuffles and lane 0
// publishes the partial with an atomic, so no CTA-wide barrier is needed
// inside a phase (warps of a CTA never wait for each other's units).
__device__ __forceinline__ void publish_sum(double* a, double v) {
    v = warp_sum(v);
    if ((threadIdx.x % kWarp) == 0) atomicAdd(a, v);
}
__device__ __forceinline__ void publish_max(unsigned long long* a, double v) {
    v = warp_max(v);
    if ((threadIdx.x % kWarp) == 0) atomicMax(a, dbl_bits(v));
}

// ---------------------------------------------------------- pass templates

__host__ __device__ __forceinline__ int pitch_of(int n) { return n + 2; }
// A row unit is two rows: the two real lines packed into one complex transform
// are always the same field on neighbouring rows, so both halves have the same
// magnitude (packing two different fields, e.g. d and Lap y, would put the FP32
// rounding of the larger one onto the smaller one).
__host__ __device__ __forceinline__ int row_unit(int, int) { return 2; }

// shared memory of one warp in a row pass / column pass (bytes)
__host__ __device__ __forceinline__ size_t row_warp_smem(int n1, int kin, int szin, int kout, int szout) {
    const int ru = row_unit(kin, kout);
    const int szc = 2 * (szin > szout ? szin : szout);
    return (size_t)kin * ru * n1 * szin + (size_t)kout * ru * n1 * szout + 2 * (size_t)pitch_of(n1) * szc;
}
__host__ __device__ __forceinline__ size_t col_warp_smem(int n0, int k, int sz) {
    return (size_t)(k + 1) * pitch_of(n0) * 2 * sz;
}
// inputs in szi, outputs in szo < szi (separate buffers)
__host__ __device__ __forceinline__ size_t col_warp_smem_mixed(int n0, int kin, int szi, int kout, int szo) {
    return (size_t)(kin + 1) * pitch_of(n0) * 2 * szi + (size_t)(kout + 1) * pitch_of(n0) * 2 * szo;
}

struct WarpCtx {
    int lane;
    char* mem;
};

__device__ __forceinline__ WarpCtx warp_ctx(const Params& P, char* smem) {
    WarpCtx w;
    w.lane = threadIdx.x % kWarp;
    w.mem = smem + (size_t)(threadIdx.x / kWarp) * P.warp_bytes;
    return w;
}

// Row pass.  src/dst: column-major half spectra, field f, column k, row r at
// f*H + k*rows + r.  A unit is ru = 2 rows;
// real line l = f*ru + rr; lines 2j and 2j+1 are packed as the real and
// imaginary parts of complex line j.  fn(p, row, x, const TI* in, TO* out).
template <class TI, class TO, class Fn>
__device__ void row_pass(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src,
                         cx<TO>* dst, char* smem, Fn&& fn) {
    using CI = cx<TI>;
    using CO = cx<TO>;
    const int rows = P.rows, n1 = P.n1, logn1 = P.logn1, half = n1 >> 1;
    const long long H = P.H;
    const int pitch = pitch_of(n1);
    const int ru = row_unit(kin, kout);
    const WarpCtx w = warp_ctx(P, smem);
    TI* Rin = (TI*)w.mem;
    TO* Rout = (TO*)(w.mem + (size_t)kin * ru * n1 * sizeof(TI));
    char* zb = w.mem + (size_t)kin * ru * n1 * sizeof(TI) + (size_t)kout * ru * n1 * sizeof(TO);
    const TI iscale = (TI)P.inv_npts;
    const URange ur = units_of(tw, rows / ru);
    for (int u = ur.b; u < ur.e; u += ur.s) {
        const int r0 = u * ru;
        for (int j = 0; 2 * j < kin * ru; j++) {
            CI* Z0 = (CI*)zb;
            CI* Z1 = Z0 + pitch;
            const int la = 2 * j, lb = 2 * j + 1;
            const CI* sa = src + (size_t)(la / ru) * H + r0 + (la % ru);
            const CI* sb = src + (size_t)(lb / ru) * H + r0 + (lb % ru);
            for (int x = w.lane; x < n1; x += kWarp) {
                const int k = (x <= half) ? x : n1 - x;
                CI A = sa[(size_t)k * rows], B = sb[(size_t)k * rows];
                if (x == 0 || x == half) { A.y = 0; B.y = 0; }
                Z0[x] = (x <= half) ? CI{A.x - B.y, A.y + B.x} : CI{A.x + B.y, B.x - A.y};
            }
            const int res = fft_line_w<+1, TI>(Z0, Z1, logn1, tw_of<TI>(tw), tw.log, w.lane);
            const CI* Zr = res ? Z1 : Z0;
            for (int x = w.lane; x < n1; x += kWarp) {
                const CI z = Zr[x];
                Rin[(size_t)la * n1 + x] = z.x * iscale;
                Rin[(size_t)lb * n1 + x] = z.y * iscale;
            }
            warp_sync();
        }
        for (int x = w.lane; x < n1; x += kWarp) {
            for (int rr = 0; rr < ru; rr++) {
                TI in[kMaxK];
                TO out[kMaxK];
                for (int f = 0; f < kin; f++) in[f] = Rin[(size_t)(f * ru + rr) * n1 + x];
                fn((long long)(r0 + rr) * n1 + x, r0 + rr, x, in, out);
                for (int g = 0; g < kout; g++) Rout[(size_t)(g * ru + rr) * n1 + x] = out[g];
            }
        }
        for (int j = 0; 2 * j < kout * ru; j++) {
            CO* Z0 = (CO*)zb;
            CO* Z1 = Z0 + pitch;
            const int la = 2 * j, lb = 2 * j + 1;
            warp_sync();
            for (int x = w.lane; x < n1; x += kWarp)
                Z0[x] = CO{Rout[(size_t)la * n1 + x], Rout[(size_t)lb * n1 + x]};
            const int res = fft_line_w<-1, TO>(Z0, Z1, logn1, tw_of<TO>(tw), tw.log, w.lane);
            const CO* Zr = res ? Z1 : Z0;
            CO* da = dst + (size_t)(la / ru) * H + r0 + (la % ru);
            CO* db = dst + (size_t)(lb / ru) * H + r0 + (lb % ru);
            const TO hf = (TO)0.5;
            for (int k = w.lane; k <= half; k += kWarp) {
                const CO zk = Zr[k];
                const CO zn = Zr[(n1 - k) & (n1 - 1)];
                da[(size_t)k * rows] = CO{hf * (zk.x + zn.x), hf * (zk.y - zn.y)};
                db[(size_t)k * rows] = CO{hf * (zk.y + zn.y), hf * (zn.x - zk.x)};
            }
        }
        warp_sync();
    }
}

// Column pass over the ncols contiguous lines of length n0: one warp per line.
// fn(k1, k0, in, out); outputs may overwrite inputs of the same point.  The
// forward transforms run in TI, the inverse ones in TO (TO narrower than TI:
// outputs whose size is a small fraction of the inputs', e.g. a direction
// computed from FP64 spectra, go back to physical space in FP32).
template <class TI, class TO, class Fn>
__device__ void col_pass(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src, cx<TO>* dst,
                         char* smem, Fn&& fn) {
    using CI = cx<TI>;
    using CO = cx<TO>;
    constexpr bool same = sizeof(TI) == sizeof(TO);
    const int n0 = P.n0, ncols = P.ncols, logn0 = P.logn0;
    const long long H = P.H;
    const int pitch = pitch_of(n0);
    const int nbi = same ? (kin > kout ? kin : kout) + 1 : kin + 1;
    const WarpCtx w = warp_ctx(P, smem);
    const URange ur = units_of(tw, ncols);
    for (int k1 = ur.b; k1 < ur.e; k1 += ur.s) {
        CI* buf[kMaxK + 1];
        CO* obuf[kMaxK + 1];
        for (int i = 0; i < nbi; i++) buf[i] = (CI*)w.mem + (size_t)i * pitch;
        for (int f = 0; f < kin; f++) {
            const CI* s = src + (size_t)f * H + (size_t)k1 * n0;
            for (int k0 = w.lane; k0 < n0; k0 += kWarp) buf[f][k0] = s[k0];
            const int res = fft_line_w<-1, TI>(buf[f], buf[nbi - 1], logn0, tw_of<TI>(tw), tw.log, w.lane);
            if (res) {
                CI* t = buf[f];
                buf[f] = buf[nbi - 1];
                buf[nbi - 1] = t;
            }
        }
        // outputs: in place of the inputs (same precision) or after them
        for (int i = 0; i <= kout; i++)
            obuf[i] = same ? (CO*)(i < kout ? buf[i] : buf[nbi - 1])
                           : (CO*)((CI*)w.mem + (size_t)nbi * pitch) + (size_t)i * pitch;
        for (int k0 = w.lane; k0 < n0; k0 += kWarp) {
            CI in[kMaxK];
            CO out[kMaxK];
            for (int f = 0; f < kin; f++) in[f] = buf[f][k0];
            fn(k1, k0, in, out);
            for (int g = 0; g < kout; g++) obuf[g][k0] = out[g];
        }
        for (int g = 0; g < kout; g++) {
            const int res = fft_line_w<+1, TO>(obuf[g], obuf[kout], logn0, tw_of<TO>(tw), tw.log, w.lane);
            const CO* r = res ? obuf[kout] : obuf[g];
            CO* d = dst + (size_t)g * H + (size_t)k1 * n0;
            for (int k0 = w.lane; k0 < n0; k0 += kWarp) d[k0] = r[k0];
            warp_sync();
        }
        warp_sync();
    }
}

// ------------------------------------------------- fixed-length pass variants
//
// The same passes with the line length a compile-time constant NF (square
// grids of 64..512): the per-lane loops unroll, every lane issues all its loads
// of a line before using any of them, the lines a warp owns are transformed in
// lockstep, and the pointwise work is split into a batched load step `ld` and an
// apply step `ap`, so the global loads of up to 16 points are in flight at once.

constexpr int kChunk = 16;  // points per batched load
// points per batched load for a load record of `bytes`: at most kChunk and at
// most 384 bytes of records per thread in flight, a power of two
__host__ __device__ constexpr int chunk_for(int bytes, int n) {
    int c = kChunk < n ? kChunk : n;
    while (c > 1 && c * bytes > 384) c >>= 1;
    return c;
}

template <int NF> __host__ __device__ __forceinline__ size_t row_fixed_smem(int kin, int szin, int kout, int szout) {
    return 2 * (size_t)(NF + 2) * ((size_t)kin * 2 * szin + (size_t)kout * 2 * szout);
}
template <int NF> __host__ __device__ __forceinline__ size_t col_fixed_smem(int k, int sz) {
    return 2 * (size_t)(NF + 2) * (size_t)k * 2 * sz;
}

template <class TI, class TO, int NF, class Ld, class Ap>
__device__ void row_pass_fixed(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src,
                               cx<TO>* dst, char* smem, Ld&& ld, Ap&& ap) {
    using CI = cx<TI>;
    using CO = cx<TO>;
    using S = decltype(ld(0ll, 0, 0));
    constexpr int LOGN = ilog2c(NF), HALF = NF / 2, H1 = HALF + 1, PITCH = NF + 2;
    constexpr int E = NF / kWarp, EH = (H1 + kWarp - 1) / kWarp;
    constexpr int GCH = E < 8 ? E : 8;
    constexpr int NPT = 2 * E, PCH = chunk_for((int)sizeof(S), NPT);
    const int rows = P.rows;
    const long long Hs = P.H;
    const WarpCtx w = warp_ctx(P, smem);
    CI* X0 = (CI*)w.mem;
    CI* X1 = X0 + (size_t)kin * PITCH;
    CO* Y0 = (CO*)(X1 + (size_t)kin * PITCH);
    CO* Y1 = Y0 + (size_t)kout * PITCH;
    const TI iscale = (TI)P.inv_npts;
    const URange ur = units_of(tw, rows / 2);
    constexpr int NCH = E / GCH;  // load chunks per field
    for (int u = ur.b; u < ur.e; u += ur.s) {
        const int r0 = 2 * u;
        // the pointwise state of the first chunk is loaded first, so that its
        // latency overlaps the spectra's and the transform's
        S st[PCH];
#pragma unroll
        for (int q = 0; q < PCH; q++) {
            const int i = q >> 1, rr = q & 1;
            const int x = w.lane + kWarp * i;
            st[q] = ld((long long)(r0 + rr) * NF + x, r0 + rr, x);
        }
        // spectra of the kin fields, chunk t = (field, GCH points); FP32 lines
        // load chunk t + 1 before storing chunk t to shared memory (the
        // compiler cannot move a global load above a shared store itself)
        auto load_chunk = [&](int t, CI* a, CI* b) {
            const int l = t / NCH, c = (t % NCH) * GCH;
            const CI* s0 = src + (size_t)l * Hs + r0;
#pragma unroll
            for (int i = 0; i < GCH; i++) {
                const int x = w.lane + kWarp * (c + i);
                const int k = (x <= HALF) ? x : NF - x;
                a[i] = s0[(size_t)k * rows];
                b[i] = s0[(size_t)k * rows + 1];
            }
        };
        auto put_chunk = [&](int t, const CI* a, const CI* b) {
            const int l = t / NCH, c = (t % NCH) * GCH;
#pragma unroll
            for (int i = 0; i < GCH; i++) {
                const int x = w.lane + kWarp * (c + i);
                CI A = a[i], B = b[i];
                if (x == 0 || x == HALF) { A.y = 0; B.y = 0; }
                X0[(size_t)l * PITCH + x] = (x <= HALF) ? CI{A.x - B.y, A.y + B.x} : CI{A.x + B.y, B.x - A.y};
            }
        };
        const int nt = kin * NCH;
        if constexpr (sizeof(TI) == 4) {
            CI a[2][GCH], b[2][GCH];
#pragma unroll
            for (int t = 0; t <= kMaxK * NCH; t++) {
                if (t < nt) load_chunk(t, a[t & 1], b[t & 1]);
                if (t >= 1 && t <= nt) put_chunk(t - 1, a[(t - 1) & 1], b[(t - 1) & 1]);
            }
        } else {
            for (int t = 0; t < nt; t++) {
                CI a[GCH], b[GCH];
                load_chunk(t, a, b);
                put_chunk(t, a, b);
            }
        }
        const CI* Xr = X0;
        if (kin > 0)
            Xr = fft_lines_fixed<+1, TI, LOGN, kMaxK>(X0, X1, PITCH, kin, tw_of<TI>(tw), tw.log, w.lane) ? X1 : X0;
#pragma unroll 1
        for (int c0 = 0; c0 < NPT; c0 += PCH) {
            if (c0 > 0) {
#pragma unroll
                for (int q = 0; q < PCH; q++) {
                    const int i = (c0 + q) >> 1, rr = (c0 + q) & 1;
                    const int x = w.lane + kWarp * i;
                    st[q] = ld((long long)(r0 + rr) * NF + x, r0 + rr, x);
                }
            }
#pragma unroll
            for (int q = 0; q < PCH; q++) {
                const int i = (c0 + q) >> 1, rr = (c0 + q) & 1;
                const int x = w.lane + kWarp * i;
                TI in[kMaxK];
                TO out[kMaxK];
#pragma unroll
                for (int f = 0; f < kMaxK; f++) {
                    if (f < kin) {
                        const CI z = Xr[(size_t)f * PITCH + x];
                        in[f] = (rr ? z.y : z.x) * iscale;
                    }
                }
                ap((long long)(r0 + rr) * NF + x, r0 + rr, x, st[q], in, out);
#pragma unroll
                for (int g = 0; g < kMaxK; g++) {
                    if (g < kout) {
                        CO* qq = Y0 + (size_t)g * PITCH + x;
                        if (rr) qq->y = out[g];
                        else qq->x = out[g];
                    }
                }
            }
        }
        if (kout > 0) {
            const CO* Yr =
                fft_lines_fixed<-1, TO, LOGN, kMaxK>(Y0, Y1, PITCH, kout, tw_of<TO>(tw), tw.log, w.lane) ? Y1 : Y0;
            const TO hf = (TO)0.5;
            for (int g = 0; g < kout; g++) {
                CO* d0 = dst + (size_t)g * Hs + r0;
                const CO* zl = Yr + (size_t)g * PITCH;
#pragma unroll
                for (int i = 0; i < EH; i++) {
                    const int k = w.lane + kWarp * i;
                    if (k <= HALF) {
                        const CO zk = zl[k];
                        const CO zn = zl[(NF - k) & (NF - 1)];
                        d0[(size_t)k * rows] = CO{hf * (zk.x + zn.x), hf * (zk.y - zn.y)};
                        d0[(size_t)k * rows + 1] = CO{hf * (zk.y + zn.y), hf * (zn.x - zk.x)};
                    }
                }
            }
        }
        warp_sync();
    }
}

template <class TI, class TO, int NF, class Ld, class Ap>
__device__ void col_pass_fixed(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src,
                               cx<TO>* dst, char* smem, Ld&& ld, Ap&& ap) {
    using C = cx<TI>;
    using CO = cx<TO>;
    using S = decltype(ld(0, 0));
    constexpr int LOGN = ilog2c(NF), PITCH = NF + 2, E = NF / kWarp;
    constexpr int GCH = E < 8 ? E : 8;
    constexpr int PCH = chunk_for((int)sizeof(S), E);
    const int ncols = P.ncols;
    const long long Hs = P.H;
    const int kl = kin > kout ? kin : kout;
    const WarpCtx w = warp_ctx(P, smem);
    C* B0 = (C*)w.mem;
    C* B1 = B0 + (size_t)kl * PITCH;
    const URange ur = units_of(tw, ncols);
    constexpr int NCH = E / GCH;  // load chunks per field
    for (int k1 = ur.b; k1 < ur.e; k1 += ur.s) {
        // the per-wavenumber state of the first chunk is loaded first, so that
        // its latency overlaps the lines' and the transform's
        S st[PCH];
#pragma unroll
        for (int q = 0; q < PCH; q++) st[q] = ld(k1, w.lane + kWarp * q);
        // lines of the kin fields, chunk t = (field, GCH points); FP32 lines
        // load chunk t + 1 before storing chunk t to shared memory
        auto load_chunk = [&](int t, C* v) {
            const int f = t / NCH, c = (t % NCH) * GCH;
            const C* s = src + (size_t)f * Hs + (size_t)k1 * NF;
#pragma unroll
            for (int i = 0; i < GCH; i++) v[i] = s[w.lane + kWarp * (c + i)];
        };
        auto put_chunk = [&](int t, const C* v) {
            const int f = t / NCH, c = (t % NCH) * GCH;
#pragma unroll
            for (int i = 0; i < GCH; i++) B0[(size_t)f * PITCH + w.lane + kWarp * (c + i)] = v[i];
        };
        const int nt = kin * NCH;
        if constexpr (sizeof(TI) == 4) {
            C v[2][GCH];
#pragma unroll
            for (int t = 0; t <= kMaxK * NCH; t++) {
                if (t < nt) load_chunk(t, v[t & 1]);
                if (t >= 1 && t <= nt) put_chunk(t - 1, v[(t - 1) & 1]);
            }
        } else {
            for (int t = 0; t < nt; t++) {
                C v[GCH];
                load_chunk(t, v);
                put_chunk(t, v);
            }
        }
        const C* Xr = B0;
        C* Xi = B1;
        if (kin > 0) {
            const int r = fft_lines_fixed<-1, TI, LOGN, kMaxK>(B0, B1, PITCH, kin, tw_of<TI>(tw), tw.log, w.lane);
            Xr = r ? B1 : B0;
            Xi = r ? B0 : B1;
        }
        // outputs (TO, PITCH apart) in the buffer the inputs do not occupy;
        // kl lines of TI hold kout lines of TO
        CO* Xo = (CO*)Xi;
#pragma unroll 1
        for (int c0 = 0; c0 < E; c0 += PCH) {
            if (c0 > 0) {
#pragma unroll
                for (int q = 0; q < PCH; q++) st[q] = ld(k1, w.lane + kWarp * (c0 + q));
            }
#pragma unroll
            for (int q = 0; q < PCH; q++) {
                const int k0 = w.lane + kWarp * (c0 + q);
                C in[kMaxK];
                CO out[kMaxK];
#pragma unroll
                for (int f = 0; f < kMaxK; f++)
                    if (f < kin) in[f] = Xr[(size_t)f * PITCH + k0];
                ap(k1, k0, st[q], in, out);
#pragma unroll
                for (int g = 0; g < kMaxK; g++)
                    if (g < kout) Xo[(size_t)g * PITCH + k0] = out[g];
            }
        }
        if (kout > 0) {
            CO* scratch = (CO*)Xr;
            const int r =
                fft_lines_fixed<+1, TO, LOGN, kMaxK>(Xo, scratch, PITCH, kout, tw_of<TO>(tw), tw.log, w.lane);
            const CO* Yr = r ? scratch : Xo;
            for (int g = 0; g < kout; g++) {
                CO* d = dst + (size_t)g * Hs + (size_t)k1 * NF;
#pragma unroll
                for (int i = 0; i < E; i++) d[w.lane + kWarp * i] = Yr[(size_t)g * PITCH + w.lane + kWarp * i];
            }
        }
        warp_sync();
    }
}

// ------------------------------------------- staged FP32 iteration passes
//
// The FP32 row and column passes of the PFC iterations with every input of a
// unit staged in shared memory by asynchronous 16-byte copies (cp.async): a
// warp issues all reads of its next unit (the half-spectrum pieces and the
// pointwise state) before it transforms the current one, so that they are in
// flight while it computes and hold no registers meanwhile.  Two staging slots
// per warp alternate.  The transforms run on two buffers in the padded layout
// (fft.cuh: no bank conflicts in the strided stages).  Selected on the host
// (Params::stage) where a warp's slice of shared memory, sized for the FP64
// phases, holds them; K fields per line (PFC: 1), NS arrays of pointwise state.
//
// Row unit: rows r0, r0 + 1.  Slot = K x (N/2 + 1) 16-byte pieces (the two
// rows' coefficients at k, adjacent in the [k][row] layout) + NS x 2 rows of
// FP32 state.  The pointwise step writes its outputs over its inputs (each
// point reads all of its fields before writing any).  Column unit: line k1.
// Slot = K lines of the input spectrum + NS lines of complex state, pitch N;
// the first stage of the forward transform reads the slot's lines.

__host__ __device__ constexpr size_t row_staged_smem(int n, int k, int ns, int slots) {
    return 2 * (size_t)k * (size_t)padded_len(n) * 8 +
           (size_t)slots * ((size_t)k * (size_t)(n / 2 + 1) * 16 + (size_t)ns * 2 * n * 4);
}
__host__ __device__ constexpr size_t col_staged_smem(int n, int k, int ns, int slots) {
    return 2 * (size_t)k * (size_t)padded_len(n) * 8 + (size_t)slots * (size_t)(k + ns) * n * 8;
}
// staging slots per model: PFC (one field) prefetches the next unit into a
// second slot; FCH (two fields, four state arrays) has room for one slot,
// which still puts all of a unit's reads in flight at once
__host__ __device__ constexpr int staged_slots(int model) { return model == 0 ? 2 : 1; }
__host__ __device__ constexpr int staged_row_state(int model) { return model == 0 ? 3 : 4; }

template <int NF, int K, int NS, int SLOTS, class Ap>
__device__ void row_pass_staged(const Params& P, const Tw& tw, const float2* src, float2* dst,
                                const float* const* sp, char* smem, Ap&& ap) {
    constexpr int LOGN = ilog2c(NF), HALF = NF / 2, H1 = HALF + 1, PP = padded_len(NF), E = NF / kWarp;
    constexpr int SLOT = K * H1 * 16 + NS * 2 * NF * 4;  // bytes
    const int rows = P.rows;
    const long long Hs = P.H;
    const WarpCtx w = warp_ctx(P, smem);
    float2* X0 = (float2*)w.mem;
    float2* X1 = X0 + K * PP;
    char* slots = (char*)(X1 + K * PP);
    const float iscale = (float)P.inv_npts;
    const URange ur = units_of(tw, rows / 2);
    auto issue = [&](int u, int s) {
        const int r0 = 2 * u;
        float4* sq = (float4*)(slots + (size_t)s * SLOT);
        float* st = (float*)(sq + K * H1);
#pragma unroll
        for (int f = 0; f < K; f++)
            for (int k = w.lane; k < H1; k += kWarp)
                cp_async16(sq + f * H1 + k, src + (size_t)f * Hs + (size_t)k * rows + r0);
#pragma unroll
        for (int a = 0; a < NS; a++)
            for (int j = w.lane; j < NF / 2; j += kWarp)
                cp_async16(st + a * 2 * NF + 4 * j, sp[a] + (size_t)r0 * NF + 4 * j);
    };
    if (SLOTS == 2 && ur.b < ur.e) issue(ur.b, 0);
    if (SLOTS == 2) cp_async_commit();
    int s = 0;
    for (int u = ur.b; u < ur.e; u += ur.s, s ^= (SLOTS - 1)) {
        const int r0 = 2 * u;
        if constexpr (SLOTS == 2) {
            // this unit's copies were issued with the previous unit
            if (u + ur.s < ur.e) issue(u + ur.s, s ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            issue(u, 0);
            cp_async_commit();
            cp_async_wait<0>();
        }
        warp_sync();
        const float4* sq = (const float4*)(slots + (size_t)s * SLOT);
        const float* st = (const float*)(sq + K * H1);
        // the two rows' half spectra -> one complex line (real part row r0)
#pragma unroll
        for (int f = 0; f < K; f++) {
#pragma unroll
            for (int i = 0; i < E; i++) {
                const int x = w.lane + kWarp * i;
                const int k = (x <= HALF) ? x : NF - x;
                const float4 v = sq[f * H1 + k];
                float2 A{v.x, v.y}, B{v.z, v.w};
                if (x == 0 || x == HALF) { A.y = 0.f; B.y = 0.f; }
                X0[f * PP + pix<true>(x)] =
                    (x <= HALF) ? float2{A.x - B.y, A.y + B.x} : float2{A.x + B.y, B.x - A.y};
            }
        }
        const int r = fft_lines_fixed<+1, float, LOGN, K, true>(X0, X1, PP, K, tw.t32, tw.log, w.lane);
        float2* Xr = r ? X1 : X0;
        float2* Xo = r ? X0 : X1;
#pragma unroll
        for (int i = 0; i < E; i++) {
            const int x = w.lane + kWarp * i;
            const int px = pix<true>(x);
#pragma unroll
            for (int rr = 0; rr < 2; rr++) {
                float sv[NS], in[K], out[K];
#pragma unroll
                for (int a = 0; a < NS; a++) sv[a] = st[a * 2 * NF + rr * NF + x];
#pragma unroll
                for (int f = 0; f < K; f++) {
                    const float2 z = Xr[f * PP + px];
                    in[f] = (rr ? z.y : z.x) * iscale;
                }
                ap((long long)(r0 + rr) * NF + x, r0 + rr, x, sv, in, out);
#pragma unroll
                for (int g = 0; g < K; g++) {
                    if (rr) Xr[g * PP + px].y = out[g];
                    else Xr[g * PP + px].x = out[g];
                }
            }
        }
        const int r2 = fft_lines_fixed<-1, float, LOGN, K, true>(Xr, Xo, PP, K, tw.t32, tw.log, w.lane);
        const float2* Yr = r2 ? Xo : Xr;
#pragma unroll
        for (int g = 0; g < K; g++) {
            float4* d0 = (float4*)(dst + (size_t)g * Hs + r0);
            const float2* zl = Yr + g * PP;
            for (int k = w.lane; k <= HALF; k += kWarp) {
                const float2 zk = zl[pix<true>(k)], zn = zl[pix<true>((NF - k) & (NF - 1))];
                d0[(size_t)k * (rows / 2)] =
                    float4{0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y), 0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x)};
            }
        }
        warp_sync();
    }
    cp_async_wait<0>();
    warp_sync();
}

template <int NF, int K, int NS, int SLOTS, class Ap>
__device__ void col_pass_staged(const Params& P, const Tw& tw, const float2* src, float2* dst,
                                const float2* const* sc, char* smem, Ap&& ap) {
    constexpr int LOGN = ilog2c(NF), PP = padded_len(NF), E = NF / kWarp;
    constexpr int SLOT = (K + NS) * NF * 8;  // bytes
    const int ncols = P.ncols;
    const long long Hs = P.H;
    const WarpCtx w = warp_ctx(P, smem);
    float2* B0 = (float2*)w.mem;
    float2* B1 = B0 + K * PP;
    char* slots = (char*)(B1 + K * PP);
    const URange ur = units_of(tw, ncols);
    auto issue = [&](int k1, int s) {
        float2* sl = (float2*)(slots + (size_t)s * SLOT);
#pragma unroll
        for (int f = 0; f < K; f++)
            for (int j = w.lane; j < NF / 2; j += kWarp)
                cp_async16(sl + f * NF + 2 * j, src + (size_t)f * Hs + (size_t)k1 * NF + 2 * j);
#pragma unroll
        for (int a = 0; a < NS; a++)
            for (int j = w.lane; j < NF / 2; j += kWarp)
                cp_async16(sl + (K + a) * NF + 2 * j, sc[a] + (size_t)k1 * NF + 2 * j);
    };
    if (SLOTS == 2 && ur.b < ur.e) issue(ur.b, 0);
    if (SLOTS == 2) cp_async_commit();
    int s = 0;
    for (int k1 = ur.b; k1 < ur.e; k1 += ur.s, s ^= (SLOTS - 1)) {
        if constexpr (SLOTS == 2) {
            if (k1 + ur.s < ur.e) issue(k1 + ur.s, s ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            issue(k1, 0);
            cp_async_commit();
            cp_async_wait<0>();
        }
        warp_sync();
        const float2* sl = (const float2*)(slots + (size_t)s * SLOT);
        const float2* st = sl + K * NF;
        const int r = fft_lines_fixed_into_padded<-1, float, LOGN, K>(sl, NF, B0, B1, PP, K, tw.t32, tw.log, w.lane);
        float2* Xr = r ? B1 : B0;
        float2* Xi = r ? B0 : B1;
#pragma unroll
        for (int i = 0; i < E; i++) {
            const int k0 = w.lane + kWarp * i;
            const int pk = pix<true>(k0);
            float2 sv[NS], in[K], out[K];
#pragma unroll
            for (int a = 0; a < NS; a++) sv[a] = st[a * NF + k0];
#pragma unroll
            for (int f = 0; f < K; f++) in[f] = Xr[f * PP + pk];
            ap(k1, k0, sv, in, out);
#pragma unroll
            for (int g = 0; g < K; g++) Xi[g * PP + pk] = out[g];
        }
        const float2* Yr = fft_lines_fixed<+1, float, LOGN, K, true>(Xi, Xr, PP, K, tw.t32, tw.log, w.lane) ? Xr : Xi;
#pragma unroll
        for (int g = 0; g < K; g++) {
            float4* d = (float4*)(dst + (size_t)g * Hs + (size_t)k1 * NF);
            const float2* y = Yr + g * PP;
            for (int j = w.lane; j < NF / 2; j += kWarp) {
                const int q = pix<true>(2 * j);  // 2j and 2j + 1 share a 16-point group
                d[j] = float4{y[q].x, y[q].y, y[q + 1].x, y[q + 1].y};
            }
        }
        warp_sync();
    }
    cp_async_wait<0>();
    warp_sync();
}

// ------------------------------------------------ CTA-cooperative variants
//
// The same passes with one unit per CTA: the threads of the CTA load the
// unit's lines, transform them together (fft_lines_coop), share the pointwise
// work and store, with CTA barriers in between.  For phases with fewer units
// than warps (a 256^2 grid has 128 row units and 129 columns): the work of a
// unit then runs on all four SM sub-partitions, which is what an FP64 line
// needs on a part whose FP64 rate per sub-partition is low.  Shared memory is
// the CTA's slice region (one unit needs no more than one warp's slice).

constexpr int kCoopChunk = 4;  // points per thread whose loads are in flight together

template <class TI, class TO, int NF, class Ld, class Ap>
__device__ void row_pass_coop(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src, cx<TO>* dst,
                              char* smem, Ld&& ld, Ap&& ap) {
    using CI = cx<TI>;
    using CO = cx<TO>;
    using S = decltype(ld(0ll, 0, 0));
    constexpr int LOGN = ilog2c(NF), HALF = NF / 2, H1 = HALF + 1, PITCH = NF + 2;
    const int rows = P.rows;
    const long long Hs = P.H;
    const int tid = threadIdx.x, nthr = blockDim.x;
    CI* X0 = (CI*)smem;
    CI* X1 = X0 + (size_t)kin * PITCH;
    CO* Y0 = (CO*)(X1 + (size_t)kin * PITCH);
    CO* Y1 = Y0 + (size_t)kout * PITCH;
    const TI iscale = (TI)P.inv_npts;
    for (int u = blockIdx.x; u < rows / 2; u += gridDim.x) {
        const int r0 = 2 * u;
        // inverse x-DFT inputs: complex line x of field l packs rows r0, r0 + 1
        for (int it = tid; it < kin * NF; it += nthr) {
            const int l = it >> LOGN, x = it & (NF - 1);
            const int k = (x <= HALF) ? x : NF - x;
            const CI* s0 = src + (size_t)l * Hs + (size_t)k * rows + r0;
            CI A = s0[0], B = s0[1];
            if (x == 0 || x == HALF) { A.y = 0; B.y = 0; }
            X0[(size_t)l * PITCH + x] = (x <= HALF) ? CI{A.x - B.y, A.y + B.x} : CI{A.x + B.y, B.x - A.y};
        }
        const CI* Xr = X0;
        if (kin > 0) Xr = fft_lines_coop<+1, TI, LOGN>(X0, X1, PITCH, kin, tw_of<TI>(tw), tw.log, tid, nthr) ? X1 : X0;
        // pointwise: point q = rr NF + x of the unit (consecutive threads, consecutive x)
        for (int q0 = 0; q0 < 2 * NF; q0 += nthr * kCoopChunk) {
            S st[kCoopChunk];
#pragma unroll
            for (int c = 0; c < kCoopChunk; c++) {
                const int q = q0 + tid + nthr * c;
                if (q < 2 * NF) {
                    const int rr = q >> LOGN, x = q & (NF - 1);
                    st[c] = ld((long long)(r0 + rr) * NF + x, r0 + rr, x);
                }
            }
#pragma unroll
            for (int c = 0; c < kCoopChunk; c++) {
                const int q = q0 + tid + nthr * c;
                if (q < 2 * NF) {
                    const int rr = q >> LOGN, x = q & (NF - 1);
                    TI in[kMaxK];
                    TO out[kMaxK];
#pragma unroll
                    for (int f = 0; f < kMaxK; f++) {
                        if (f < kin) {
                            const CI z = Xr[(size_t)f * PITCH + x];
                            in[f] = (rr ? z.y : z.x) * iscale;
                        }
                    }
                    ap((long long)(r0 + rr) * NF + x, r0 + rr, x, st[c], in, out);
#pragma unroll
                    for (int g = 0; g < kMaxK; g++) {
                        if (g < kout) {
                            CO* qq = Y0 + (size_t)g * PITCH + x;
                            if (rr) qq->y = out[g];
                            else qq->x = out[g];
                        }
                    }
                }
            }
        }
        if (kout > 0) {
            const CO* Yr = fft_lines_coop<-1, TO, LOGN>(Y0, Y1, PITCH, kout, tw_of<TO>(tw), tw.log, tid, nthr) ? Y1 : Y0;
            const TO hf = (TO)0.5;
            for (int it = tid; it < kout * H1; it += nthr) {
                const int g = it / H1, k = it - g * H1;
                CO* d0 = dst + (size_t)g * Hs + r0;
                const CO* zl = Yr + (size_t)g * PITCH;
                const CO zk = zl[k];
                const CO zn = zl[(NF - k) & (NF - 1)];
                d0[(size_t)k * rows] = CO{hf * (zk.x + zn.x), hf * (zk.y - zn.y)};
                d0[(size_t)k * rows + 1] = CO{hf * (zk.y + zn.y), hf * (zn.x - zk.x)};
            }
        }
        cta_sync();  // the next unit reuses the buffers
    }
}

template <class TI, class TO, int NF, class Ld, class Ap>
__device__ void col_pass_coop(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src, cx<TO>* dst,
                              char* smem, Ld&& ld, Ap&& ap) {
    using C = cx<TI>;
    using CO = cx<TO>;
    using S = decltype(ld(0, 0));
    constexpr int LOGN = ilog2c(NF), PITCH = NF + 2;
    const int ncols = P.ncols;
    const long long Hs = P.H;
    const int kl = kin > kout ? kin : kout;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C* B0 = (C*)smem;
    C* B1 = B0 + (size_t)kl * PITCH;
    for (int k1 = blockIdx.x; k1 < ncols; k1 += gridDim.x) {
        for (int it = tid; it < kin * NF; it += nthr) {
            const int f = it >> LOGN, x = it & (NF - 1);
            B0[(size_t)f * PITCH + x] = src[(size_t)f * Hs + (size_t)k1 * NF + x];
        }
        const C* Xr = B0;
        C* Xi = B1;
        if (kin > 0) {
            const int r = fft_lines_coop<-1, TI, LOGN>(B0, B1, PITCH, kin, tw_of<TI>(tw), tw.log, tid, nthr);
            Xr = r ? B1 : B0;
            Xi = r ? B0 : B1;
        }
        CO* Xo = (CO*)Xi;
        for (int q0 = 0; q0 < NF; q0 += nthr * kCoopChunk) {
            S st[kCoopChunk];
#pragma unroll
            for (int c = 0; c < kCoopChunk; c++) {
                const int k0 = q0 + tid + nthr * c;
                if (k0 < NF) st[c] = ld(k1, k0);
            }
#pragma unroll
            for (int c = 0; c < kCoopChunk; c++) {
                const int k0 = q0 + tid + nthr * c;
                if (k0 < NF) {
                    C in[kMaxK];
                    CO out[kMaxK];
#pragma unroll
                    for (int f = 0; f < kMaxK; f++)
                        if (f < kin) in[f] = Xr[(size_t)f * PITCH + k0];
                    ap(k1, k0, st[c], in, out);
#pragma unroll
                    for (int g = 0; g < kMaxK; g++)
                        if (g < kout) Xo[(size_t)g * PITCH + k0] = out[g];
                }
            }
        }
        if (kout > 0) {
            CO* scratch = (CO*)Xr;
            const int r = fft_lines_coop<+1, TO, LOGN>(Xo, scratch, PITCH, kout, tw_of<TO>(tw), tw.log, tid, nthr);
            const CO* Yr = r ? scratch : Xo;
            for (int it = tid; it < kout * NF; it += nthr) {
                const int g = it >> LOGN, x = it & (NF - 1);
                dst[(size_t)g * Hs + (size_t)k1 * NF + x] = Yr[(size_t)g * PITCH + x];
            }
        }
        cta_sync();
    }
}

// Only passes with an FP64 line have the cooperative variant: an FP32 line is
// latency-bound, not rate-bound, on one sub-partition, and the extra code
// costs the FP32 passes registers.
template <class TI, class TO> constexpr bool kHasCoop = sizeof(TI) == 8 || sizeof(TO) == 8;
// NF | kNoCoop: line length NF without the cooperative variants (batched
// launches, whose warps own their units, never use them)
constexpr int kNoCoop = 1 << 20;

// ------------------------------------------------------- middle axis (3D)
//
// S = -1: forward along the middle axis, [f][k1][i0 nm + i1] -> [f][k1][km][i0];
// S = +1: inverse, [f][k1][km][i0] -> [f][k1][i0 nm + i1] (no scaling: the
// row passes apply 1/n_pts).  A unit is kMidG consecutive i0 of one k1 plane:
// its kMidG lines are contiguous on the row side, and on the transposed side
// every km holds kMidG neighbouring values.
constexpr int kMidG = 2;

// sz: bytes of a real scalar (8 for FP64 lines)
__host__ __device__ __forceinline__ size_t mid_warp_smem(int nm, int sz) {
    return (size_t)2 * kMidG * pitch_of(nm) * 2 * sz;
}
__host__ __device__ __forceinline__ int mid_units(const Params& P) { return P.h1 * (P.n0 / kMidG); }

template <class T, int S, int NF>
__device__ void mid_pass(const Params& P, const Tw& tw, int k, const cx<T>* src, cx<T>* dst, char* smem) {
    using C = cx<T>;
    constexpr int L = NF & (kNoCoop - 1);  // fixed line length of the launch (0: runtime)
    // values per lane loaded before any of them is stored to shared memory
    // (the compiler cannot move a global load above a shared store itself)
    constexpr int CH = sizeof(T) == 4 ? 16 : 8;
    const int nm = P.nm, logm = P.logm, n0 = P.n0, rows = P.rows, gpp = P.n0 / kMidG;
    const long long H = P.H;
    const int pitch = pitch_of(nm);
    const int nv = kMidG * nm;
    const WarpCtx w = warp_ctx(P, smem);
    C* B0 = (C*)w.mem;
    C* B1 = B0 + (size_t)kMidG * pitch;
    const URange ur = units_of(tw, P.h1 * gpp);
    for (int u = ur.b; u < ur.e; u += ur.s) {
        const int k1 = u / gpp, i0 = (u - k1 * gpp) * kMidG;
        for (int f = 0; f < k; f++) {
            const C* sf = src + (size_t)f * H;
            C* df = dst + (size_t)f * H;
            const size_t rowbase = (size_t)k1 * rows + (size_t)i0 * nm;    // [k1][i0][i1]
            const size_t colbase = (size_t)k1 * nm * n0 + (size_t)i0;      // [k1][km][i0]
            for (int j0 = 0; j0 < nv; j0 += CH * kWarp) {
                C v[CH];
#pragma unroll
                for (int q = 0; q < CH; q++) {
                    const int j = j0 + w.lane + q * kWarp;
                    if (j < nv) {
                        if (S < 0) v[q] = sf[rowbase + j];
                        else v[q] = sf[colbase + (size_t)(j / kMidG) * n0 + (j % kMidG)];
                    }
                }
#pragma unroll
                for (int q = 0; q < CH; q++) {
                    const int j = j0 + w.lane + q * kWarp;
                    if (j < nv) {
                        if (S < 0) {
                            B0[(j >> logm) * pitch + (j & (nm - 1))] = v[q];
                        } else {
                            const int km = j / kMidG, g = j - km * kMidG;
                            B0[g * pitch + km] = v[q];
                        }
                    }
                }
            }
            int r = 0;
            if constexpr (L > 0) {
                if (nm == L) {
                    // cubic grid: both lines in lockstep through the fixed-length stages
                    r = fft_lines_fixed<S, T, ilog2c(L), kMidG>(B0, B1, pitch, kMidG, tw_of<T>(tw), tw.log, w.lane);
                } else {
                    for (int g = 0; g < kMidG; g++)
                        r = fft_line_w<S, T>(B0 + g * pitch, B1 + g * pitch, logm, tw_of<T>(tw), tw.log, w.lane);
                }
            } else {
                for (int g = 0; g < kMidG; g++)
                    r = fft_line_w<S, T>(B0 + g * pitch, B1 + g * pitch, logm, tw_of<T>(tw), tw.log, w.lane);
            }
            const C* Br = r ? B1 : B0;
            for (int j = w.lane; j < nv; j += kWarp) {
                if (S < 0) {
                    const int km = j / kMidG, g = j - km * kMidG;
                    df[colbase + (size_t)km * n0 + g] = Br[g * pitch + km];
                } else {
                    const int g = j >> logm, i1 = j & (nm - 1);
                    df[rowbase + j] = Br[g * pitch + i1];
                }
            }
            warp_sync();
        }
    }
}

// The FP32 middle passes of cubic grids with their inputs staged as in the
// iteration passes: a unit (kMidG lines of one field) is 16-byte pieces, each
// two neighbouring lines' values at one position (row side: i1 pairs of one
// line; transposed side: the kMidG values at one km), copied by cp.async into
// one of two slots while the warp transforms the previous unit; transforms in
// the padded layout.
__host__ __device__ constexpr size_t mid_staged_smem(int n) {
    return 2 * (size_t)kMidG * (size_t)padded_len(n) * 8 + 2 * (size_t)n * 16;
}

template <int NF, int S>
__device__ void mid_pass_staged(const Params& P, const Tw& tw, int k, const float2* src, float2* dst, char* smem) {
    constexpr int LOGN = ilog2c(NF), PP = padded_len(NF);
    static_assert(kMidG == 2, "a 16-byte piece holds kMidG FP32 complex values");
    const int n0 = P.n0, rows = P.rows, gpp = P.n0 / kMidG;
    const long long H = P.H;
    const WarpCtx w = warp_ctx(P, smem);
    float2* B0 = (float2*)w.mem;
    float2* B1 = B0 + kMidG * PP;
    float4* slots = (float4*)(B1 + kMidG * PP);  // 2 x NF pieces
    const URange ur = units_of(tw, P.h1 * gpp);
    auto issue = [&](int u, int f, int s) {
        const int k1 = u / gpp, i0 = (u - k1 * gpp) * kMidG;
        const float2* sf = src + (size_t)f * H;
        float4* sl = slots + s * NF;
        if (S < 0) {
            const float2* rb = sf + (size_t)k1 * rows + (size_t)i0 * NF;  // [k1][i0][i1]
            for (int j = w.lane; j < NF; j += kWarp) cp_async16(sl + j, rb + 2 * j);
        } else {
            const float2* cb = sf + (size_t)k1 * NF * n0 + i0;  // [k1][km][i0]
            for (int km = w.lane; km < NF; km += kWarp) cp_async16(sl + km, cb + (size_t)km * n0);
        }
    };
    int u = ur.b, f = 0, s = 0;
    if (u < ur.e && k > 0) issue(u, 0, 0);
    cp_async_commit();
    while (u < ur.e && k > 0) {
        int un = u, fn = f + 1;
        if (fn == k) {
            fn = 0;
            un = u + ur.s;
        }
        if (un < ur.e) issue(un, fn, s ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        warp_sync();
        const float2* sl = (const float2*)(slots + s * NF);
#pragma unroll 4
        for (int j = w.lane; j < kMidG * NF; j += kWarp) {
            if (S < 0) B0[(j / NF) * PP + pix<true>(j % NF)] = sl[j];         // line g = j / NF
            else B0[(j % kMidG) * PP + pix<true>(j / kMidG)] = sl[j];         // km = j / kMidG
        }
        const int r = fft_lines_fixed<S, float, LOGN, kMidG, true>(B0, B1, PP, kMidG, tw.t32, tw.log, w.lane);
        const float2* Br = r ? B1 : B0;
        const int k1 = u / gpp, i0 = (u - k1 * gpp) * kMidG;
        float2* df = dst + (size_t)f * H;
        if (S < 0) {
            float4* cb = (float4*)(df + (size_t)k1 * NF * n0 + i0);
            for (int km = w.lane; km < NF; km += kWarp) {
                const float2 a = Br[pix<true>(km)], b = Br[PP + pix<true>(km)];
                cb[(size_t)km * (n0 / 2)] = float4{a.x, a.y, b.x, b.y};
            }
        } else {
            float4* rb = (float4*)(df + (size_t)k1 * rows + (size_t)i0 * NF);
            for (int j = w.lane; j < NF; j += kWarp) {
                const int g = (2 * j) / NF, q = pix<true>((2 * j) % NF);  // i1 and i1 + 1 share a group
                const float2 a = Br[g * PP + q], b = Br[g * PP + q + 1];
                rb[j] = float4{a.x, a.y, b.x, b.y};
            }
        }
        warp_sync();
        u = un;
        f = fn;
        s ^= 1;
    }
    cp_async_wait<0>();
    warp_sync();
}

// Column passes read the last row pass's output and write the next row pass's
// input: in 2D NB -> DB directly; in 3D the middle passes sit between, so the
// column passes read X (forward middle output) and write NB (inverse middle
// input), and the inverse middle pass writes DB.
__device__ __forceinline__ const double2* csrc64(const Params& P) { return P.nm > 1 ? P.X64 : P.NB64; }
__device__ __forceinline__ double2* cdst64(const Params& P) { return P.nm > 1 ? P.NB64 : P.DB64; }
template <class T> __device__ __forceinline__ const cx<T>* csrcT(const Params& P) {
    return (const cx<T>*)(P.nm > 1 ? P.X : P.NB);
}
template <class T> __device__ __forceinline__ cx<T>* cdstT(const Params& P) {
    return (cx<T>*)(P.nm > 1 ? P.NB : P.DB);
}

// dispatch: NF = 0 runs the runtime-length passes (NF may carry kNoCoop)
// COOP: the pass has the CTA-cooperative variant (by default when it has an
// FP64 line; phases with FP64 pointwise work on T lines ask for it too)
template <class TI, class TO, int NF, bool COOP = kHasCoop<TI, TO>, class Ld, class Ap>
__device__ __forceinline__ void rowp(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src,
                                     cx<TO>* dst, char* smem, Ld&& ld, Ap&& ap) {
    constexpr int L = NF & (kNoCoop - 1);
    if constexpr (L == 0) {
        row_pass<TI, TO>(P, tw, kin, kout, src, dst, smem,
                         [&](long long p, int row, int x, const TI* in, TO* out) {
                             const auto s = ld(p, row, x);
                             ap(p, row, x, s, in, out);
                         });
    } else {
        if constexpr (COOP && !(NF & kNoCoop)) {
            if (P.coop) {
                row_pass_coop<TI, TO, L>(P, tw, kin, kout, src, dst, smem, ld, ap);
                return;
            }
        }
        row_pass_fixed<TI, TO, L>(P, tw, kin, kout, src, dst, smem, ld, ap);
    }
}

template <class TI, class TO, int NF, bool COOP = kHasCoop<TI, TO>, class Ld, class Ap>
__device__ __forceinline__ void colp2(const Params& P, const Tw& tw, int kin, int kout, const cx<TI>* src,
                                      cx<TO>* dst, char* smem, Ld&& ld, Ap&& ap) {
    constexpr int L = NF & (kNoCoop - 1);
    if constexpr (L == 0) {
        col_pass<TI, TO>(P, tw, kin, kout, src, dst, smem, [&](int k1, int k0, const cx<TI>* in, cx<TO>* out) {
            const auto s = ld(k1, k0);
            ap(k1, k0, s, in, out);
        });
    } else {
        if constexpr (COOP && !(NF & kNoCoop)) {
            if (P.coop) {
                col_pass_coop<TI, TO, L>(P, tw, kin, kout, src, dst, smem, ld, ap);
                return;
            }
        }
        col_pass_fixed<TI, TO, L>(P, tw, kin, kout, src, dst, smem, ld, ap);
    }
}
template <class T, int NF, bool COOP = kHasCoop<T, T>, class Ld, class Ap>
__device__ __forceinline__ void colp(const Params& P, const Tw& tw, int kin, int kout, const cx<T>* src,
                                     cx<T>* dst, char* smem, Ld&& ld, Ap&& ap) {
    colp2<T, T, NF, COOP>(P, tw, kin, kout, src, dst, smem, ld, ap);
}

struct Nil {};

// ------------------------------------------------------------ phase bodies
//
// The FP32 iteration phases (R, CI) are inlined into the persistent kernel
// (PAGD_HOT), where the parameters are constant-bank operands; the base
// evaluations (exact and incremental, both with FP64 work per point) and the
// programs are functions of their own (PAGD_COLD), so that their larger
// working sets are allocated separately and do not spill registers in the hot
// phases.
#ifndef PAGD_HOT
#define PAGD_HOT __forceinline__
#endif
#ifndef PAGD_COLD
#define PAGD_COLD __noinline__
#endif

// number of fields in the iteration passes: PFC transforms v^3 differences and
// inverts d; FCH transforms (dF', dP) and inverts (d, Lap ybar)
__host__ __device__ __forceinline__ int k_iter(int model) { return model == M_PFC ? 1 : 2; }
__host__ __device__ __forceinline__ int k_base(int model) { return model == M_PFC ? 3 : 2; }

// Phase B: (1) the pending acceptance of the previous step, (2) either the new
// step's initial guess (Sec. 3.4.2: extrapolation of the two previous solutions),
// base argument VB, history term g and preconditioner sums, or a move of the
// base to the current candidate (mixed precision), (3) the forward x-DFT of the
// FP64 base fields (VB, g[, VB^3]).
// INC: incremental base evaluation (FP32-mixed).  Instead of (VB, g[, VB^3]) in
// FP64 it transforms, in T, the fields that are small at the new base: the
// linear residual W = A_i VB + g = a x + b u^n + c u^{n-1} (O(u_t)), the shift
// y = VB_new - VB_old from the reference point, and (PFC) the nonlinear change
// VB_new^3 - VB_old^3 = y (3 r^2 + 3 r y + y^2), r = VB_old.
template <class T, int NF, bool INC>
__device__ __forceinline__ void phase_B_impl(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red) {
    using TO = typename std::conditional<INC, T, double>::type;
    const StepK& k = step_coeffs(P, c.step);
    const int bank = c.step & 1;
    T* vbt = (T*)P.VBt;
    T* d0 = (T*)P.DD[0];
    T* d1 = (T*)P.DD[1];
    const long long gt = thread_rank(tw);
    const long long gs = thread_count(tw);
    // acceptance of step c.step - 1 (same scheme, so the same theta_v).  The
    // FP64 mean of the correction and the running mass excess K are removed; the
    // exact change sum(u^{n+1} - u^n) is fed back into K (error feedback keeps
    // the rounding of the removal from accumulating over steps).
    const T* dacc = (const T*)P.DD[c.acc_it & 1];
    const double macc =
        c.acc ? ldcg(&P.sums[(size_t)(bank ^ 1) * P.nslots + c.acc_lastev]) / (double)P.npts +
                    ldcg(&P.mass[0]) / (double)P.npts
              : 0.0;
    double dmass = 0.0;
    // rebase: the candidate of this step
    const T* dreb = (const T*)P.DD[c.it & 1];
    const double mreb = c.reb ? ldcg(&P.sums[(size_t)bank * P.nslots + c.lastev]) / (double)P.npts : 0.0;
    // a new step clears its bank's norm and sum slots (a restart of the same
    // step from another initial guess keeps counting in them)
    if (!c.reb && c.gmode != 2 && c.gmode != 3 && c.gmode != 4) {
        for (long long q = gt; q < P.nslots; q += gs) {
            P.norms[(size_t)bank * P.nslots + q] = 0ull;
            P.sums[(size_t)bank * P.nslots + q] = 0.0;
        }
        if (gt == 0) {
            P.sc->beta_sum[bank ^ 1][0] = 0.0;
            P.sc->beta_sum[bank ^ 1][1] = 0.0;
        }
    }
    if (c.rec_pending && leader(tw)) P.mass[2] = bits_dbl(ldcg(&P.norms[(size_t)c.rec_bank * P.nslots + c.rec_ev]));
    if (c.acc && leader(tw)) {
        P.stats[c.step - 1].iters = c.acc_ev;
        P.stats[c.step - 1].status = ST_OK;
        P.stats[c.step - 1].resid = c.acc_resid;
        P.stats[c.step - 1].used_guess = c.acc_used;
        P.sc->steps_done = c.step;
    }
    double s0 = 0.0, s2 = 0.0;
    const float c1e = (float)(1.0 - P.eps), tauf = (float)P.tau, eta1f = (float)P.eta1, eta2f = (float)P.eta2,
                e2f = (float)(P.eps * P.eps);
    const int kb = k_base(P.model);
    const bool pfc = P.model == M_PFC;
    const bool reb = c.reb != 0, acc = c.acc != 0;
    const double ith = 1.0 / k.thv, wth = 1.0 - k.thv;
    double* U0 = P.U[c.cur];
    double* U1 = P.U[c.cur ^ 1];
    struct St { double vb, g, a, b, d; };
    T* yb = (T*)P.YB;
    cx<TO>* dst = INC ? (cx<TO>*)P.NB : (cx<TO>*)P.NB64;
    const double Ai = k.Ai;
    // an exact re-evaluation within a step reuses the step's g_hat (GH64)
    const bool gcached = !INC && reb && c.gok;
    const bool use_guess = !reb && (c.gmode == 1 || c.gmode == 3);
    const double gshift = use_guess ? ldcg(&P.sc->red[2]) * P.inv_npts : 0.0;
    const int kout = ((INC && reb) || gcached) ? kb - 1 : kb;
    rowp<double, TO, NF>(
        P, tw, 0, kout, (const double2*)nullptr, dst, smem,
        [&](long long p, int, int) {
            St s;
            s.vb = P.VB[p];
            s.g = P.G64[p];
            s.d = reb ? (double)dreb[p] : (acc ? (double)dacc[p] : 0.0);
            s.a = reb ? 0.0 : U0[p];   // (before acceptance) u^n of the previous step if acc
            s.b = reb ? 0.0 : U1[p];
            return s;
        },
        [&](long long p, int, int, const St& s, const double*, TO* out) {
            double vb, g;
            if (reb) {
                vb = s.vb + (s.d - mreb);
                g = s.g;
            } else {
                double a = s.a, b = s.b;
                if (acc) {
                    // U1 is the previous step's u^n; the accepted u^{n+1} goes to U0
                    const double va = s.vb + (s.d - macc);
                    a = (va - wth * s.b) * ith;
                    U0[p] = a;
                    dmass += a - s.b;
                }
                // initial iterate (Sec. 3.4.2): extrapolation, or the caller's
                // guess moved to the mass of u^n
                const double x0 = use_guess ? P.guess[p] + gshift : a + k.rho * (a - b);
                vb = k.thv * x0 + (1.0 - k.thv) * a;
                g = k.b * a + k.c * b - k.gun * a;
                P.G64[p] = g;
                // averaged-Newton sums: preconditioner constants, FP32 is enough
                const float vf = (float)vb;
                if (pfc) {
                    s0 += (double)(3.0f * vf * vf + c1e);
                } else {
                    const float f1 = dF1(vf, tauf), f2 = dF2(vf, tauf), f3 = dF3(vf, tauf);
                    s0 += (double)(f2 * f2 - eta2f * f2 + f3 * f1);
                    s2 += (double)(e2f * (f2 - eta1f));
                }
            }
            P.VB[p] = vb;
            vbt[p] = (T)vb;
            d0[p] = (T)0;
            d1[p] = (T)0;
            if constexpr (INC) {
                // a rebase keeps g, so W moves by A_i y (added spectrally); a new
                // step transforms its W
                const double y = vb - s.vb, r = s.vb;
                yb[p] = (T)y;
                const int o = reb ? 0 : 1;
                if (!reb) out[0] = (TO)(Ai * vb + g);
                out[o] = (TO)y;
                if (pfc) {
                    const TO yt = (TO)y, rt = (TO)r;
                    out[o + 1] = yt * ((TO)3 * rt * rt + (TO)3 * rt * yt + yt * yt);
                }
            } else {
                out[0] = vb;
                if (!gcached) out[1] = g;
                if (pfc) out[gcached ? 1 : 2] = vb * vb * vb;
            }
        });
    if (!reb) {
        publish_sum(&P.sc->beta_sum[c.bsel][0], s0);
        if (!pfc) {
            publish_sum(&P.sc->beta_sum[c.bsel][1], s2);
        }
    }
    if (acc) {
        publish_sum(&P.mass[1], dmass);
    }
}

template <class T, int NF>
__device__ PAGD_COLD void phase_B_exact(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red) {
    phase_B_impl<T, NF, false>(P, c, tw, smem, red);
}
template <class T, int NF>
__device__ PAGD_COLD void phase_B_inc(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red) {
    phase_B_impl<T, NF, true>(P, c, tw, smem, red);
}

// Spectral base gradient C0 = G'_N(VB) (Eqs. misc07 / obj:G'), its
// preconditioned direction d0 and the first correction delta_1 = theta_v s d0.
template <class T>
__device__ __forceinline__ void base_direction(const Params& P, const StepK& k, const Beta& B,
                                               int k1, int k0, double kap, double2 G, double2& d) {
    const long long idx = (long long)k1 * P.n0 + k0;
    cx<T>* C0 = (cx<T>*)P.C0;
    cx<T>* S0 = (cx<T>*)P.SS[0];
    cx<T>* S1 = (cx<T>*)P.SS[1];
    if (kap == 0.0) {
        G = double2{0.0, 0.0};
        d = double2{0.0, 0.0};
    } else {
        const double Lk = B.m2 / kap + B.b0 + B.b2 * kap + B.b4 * kap * kap;
        if (!(Lk > 0.0)) atomicOr(&P.sc->flags, FLAG_PRECOND);
        const double il = -1.0 / Lk;
        d = double2{il * G.x, il * G.y};
    }
    C0[idx] = cx<T>{(T)G.x, (T)G.y};
    S0[idx] = cx<T>{(T)0, (T)0};
    S1[idx] = cx<T>{(T)(k.ts * d.x), (T)(k.ts * d.y)};
}

template <class T, int NF>
__device__ PAGD_COLD void phase_C(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    if (leader(tw)) {
        // fold the last acceptance's mass change into the running excess
        P.mass[0] += P.mass[1];
        P.mass[1] = 0.0;
    }
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    const int kb = k_base(P.model);
    const double iM = 1.0 / P.M;
    const double e4 = P.eps * P.eps * P.eps * P.eps;
    const bool gcached = c.ereb && c.gok;  // g_hat from GH64, not among the inputs
    const int kin = gcached ? kb - 1 : kb;
    auto ldg_hat = [&](int k1, int k0) {
        return gcached ? P.GH64[(long long)k1 * P.n0 + k0] : double2{0.0, 0.0};
    };
    if (P.model == M_PFC) {
        // the direction is small: its inverse transforms run in T
        colp2<double, T, NF>(P, tw, kin, 1, csrc64(P), cdstT<T>(P), smem, ldg_hat,
                         [&](int k1, int k0, const double2& gh, const double2* in, cx<T>* out) {
                             const double kap = kappa_at(P, k1, k0);
                             const double2 v = in[0], g = gcached ? gh : in[1], nl = in[gcached ? 1 : 2];
                             if (!gcached) P.GH64[(long long)k1 * P.n0 + k0] = g;
                             P.VR64[(long long)k1 * P.n0 + k0] = v;
                             P.NR64[(long long)k1 * P.n0 + k0] = nl;
                             P.WR64[(long long)k1 * P.n0 + k0] = double2{k.Ai * v.x + g.x, k.Ai * v.y + g.y};
                             double2 G{0.0, 0.0};
                             if (kap != 0.0) {
                                 const double Lh = 1.0 - P.eps - 2.0 * kap + kap * kap;
                                 const double ik = iM / kap;
                                 G.x = (k.Ai * v.x + g.x) * ik + Lh * v.x + nl.x;
                                 G.y = (k.Ai * v.y + g.y) * ik + Lh * v.y + nl.y;
                             }
                             double2 d;
                             base_direction<T>(P, k, B, k1, k0, kap, G, d);
                             out[0] = cx<T>{(T)d.x, (T)d.y};
                         });
    } else {
        colp<double, NF>(P, tw, kin, 1, csrc64(P), cdst64(P), smem, ldg_hat,
                         [&](int k1, int k0, const double2& gh, const double2* in, double2* out) {
                             const double kap = kappa_at(P, k1, k0);
                             const double2 v = in[0], g = gcached ? gh : in[1];
                             if (!gcached) P.GH64[(long long)k1 * P.n0 + k0] = g;
                             P.VR64[(long long)k1 * P.n0 + k0] = v;
                             P.WR64[(long long)k1 * P.n0 + k0] = double2{k.Ai * v.x + g.x, k.Ai * v.y + g.y};
                             double2 G{0.0, 0.0};
                             if (kap != 0.0) {
                                 const double ik = iM / kap;
                                 G.x = (k.Ai * v.x + g.x) * ik + e4 * kap * kap * v.x;
                                 G.y = (k.Ai * v.y + g.y) * ik + e4 * kap * kap * v.y;
                             }
                             P.CL64[(long long)k1 * P.n0 + k0] = G;
                             out[0] = double2{-kap * v.x, -kap * v.y};
                         });
    }
}

// FCH: physical Lap VB, then forward x-DFT of (F'(VB), P(VB)) where
// P = -eps^2 (F'' - eta1) Lap v + (F'' - eta2) F'  (the non-Laplacian part of mu).
template <class T, int NF>
__device__ PAGD_COLD void phase_D(const Params& P, const Tw& tw, char* smem) {
    T* lbt = (T*)P.LBt;
    const double e2 = P.eps * P.eps;
    rowp<double, double, NF>(P, tw, 1, 2, P.DB64, P.NB64, smem,
                             [&](long long p, int, int) { return P.VB[p]; },
                             [&](long long p, int, int, const double& vb, const double* in, double* out) {
                                 const double lb = in[0];
                                 lbt[p] = (T)lb;
                                 P.LB64[p] = lb;
                                 const double f1 = dF1(vb, P.tau), f2 = dF2(vb, P.tau);
                                 out[0] = f1;
                                 out[1] = -e2 * (f2 - P.eta1) * lb + (f2 - P.eta2) * f1;
                             });
}

template <class T, int NF>
__device__ PAGD_COLD void phase_E(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    const double e2 = P.eps * P.eps;
    const double l1 = lam_at(P, 1);
    // the direction (and Lap of the first correction) are small: inverse in T
    colp2<double, T, NF>(P, tw, 2, 2, csrc64(P), cdstT<T>(P), smem,
                     [&](int k1, int k0) { return P.CL64[(long long)k1 * P.n0 + k0]; },
                     [&](int k1, int k0, const double2& lin, const double2* in, cx<T>* out) {
                         const double kap = kappa_at(P, k1, k0);
                         const long long idx = (long long)k1 * P.n0 + k0;
                         P.NR64[idx] = in[0];
                         P.NR64[idx + P.H] = in[1];
                         double2 G{0.0, 0.0};
                         if (kap != 0.0) {
                             G.x = lin.x + e2 * kap * in[0].x + in[1].x;
                             G.y = lin.y + e2 * kap * in[0].y + in[1].y;
                         }
                         double2 d;
                         base_direction<T>(P, k, B, k1, k0, kap, G, d);
                         out[0] = cx<T>{(T)d.x, (T)d.y};
                         const double f = -kap * (1.0 + l1) * k.ts;
                         out[1] = cx<T>{(T)(f * d.x), (T)(f * d.y)};
                     });
}

// Incremental base evaluation, column part: the FP64 reference spectra move to
// the new base (v_hat += y_hat, PFC: N_hat += dN_hat) and the base gradient is
// assembled in FP64 from them and the T-transformed small fields.
template <class T, int NF>
__device__ PAGD_COLD void phase_CN(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    using C = cx<T>;
    if (leader(tw)) {
        P.mass[0] += P.mass[1];
        P.mass[1] = 0.0;
    }
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    const bool reb = c.ereb != 0;
    const int kb = k_base(P.model);
    const int kin = reb ? kb - 1 : kb;
    const int o = reb ? 0 : 1;  // in[o] = y_hat, in[o + 1] = dN_hat (PFC), in[0] = W_hat (new step)
    const double iM = 1.0 / P.M, Ai = k.Ai;
    const double e4 = P.eps * P.eps * P.eps * P.eps;
    const bool pfc = P.model == M_PFC;
    struct St { double2 v, n, w; };
    colp<T, NF, true>(
        P, tw, kin, 1, csrcT<T>(P), cdstT<T>(P), smem,
        [&](int k1, int k0) {
            const long long idx = (long long)k1 * P.n0 + k0;
            return St{P.VR64[idx], pfc ? P.NR64[idx] : double2{0.0, 0.0}, P.WR64[idx]};
        },
        [&](int k1, int k0, const St& s, const C* in, C* out) {
            const long long idx = (long long)k1 * P.n0 + k0;
            const double kap = kappa_at(P, k1, k0);
            const double2 yh{(double)in[o].x, (double)in[o].y};
            const double2 v{s.v.x + yh.x, s.v.y + yh.y};
            P.VR64[idx] = v;
            const double2 w = reb ? double2{s.w.x + Ai * yh.x, s.w.y + Ai * yh.y}
                                  : double2{(double)in[0].x, (double)in[0].y};
            P.WR64[idx] = w;
            if (pfc) {
                const double2 nl{s.n.x + (double)in[o + 1].x, s.n.y + (double)in[o + 1].y};
                P.NR64[idx] = nl;
                double2 G{0.0, 0.0};
                if (kap != 0.0) {
                    const double Lh = 1.0 - P.eps - 2.0 * kap + kap * kap;
                    const double ik = iM / kap;
                    G.x = w.x * ik + Lh * v.x + nl.x;
                    G.y = w.y * ik + Lh * v.y + nl.y;
                }
                double2 d;
                base_direction<T>(P, k, B, k1, k0, kap, G, d);
                out[0] = C{(T)d.x, (T)d.y};
            } else {
                double2 G{0.0, 0.0};
                if (kap != 0.0) {
                    const double ik = iM / kap;
                    G.x = w.x * ik + e4 * kap * kap * v.x;
                    G.y = w.y * ik + e4 * kap * kap * v.y;
                }
                P.CL64[idx] = G;
                const T f = (T)(-kap);
                out[0] = C{f * in[o].x, f * in[o].y};
            }
        });
}

// FCH incremental: Lap VB_new = Lap VB_old + Lap y (FP64 physical), then the T
// transforms of the nonlinear changes F'(VB_new) - F'(VB_old) and
// P(VB_new) - P(VB_old), written as the iteration's difference formulas.
template <class T, int NF>
__device__ PAGD_COLD void phase_DN(const Params& P, const Tw& tw, char* smem) {
    using C = cx<T>;
    T* lbt = (T*)P.LBt;
    const T* yb = (const T*)P.YB;
    const T tau = (T)P.tau, e2 = (T)(P.eps * P.eps), eta1 = (T)P.eta1, eta2 = (T)P.eta2;
    struct St { double vb, lb; T y; };
    rowp<T, T, NF, true>(
        P, tw, 1, 2, (const C*)P.DB, (C*)P.NB, smem,
        [&](long long p, int, int) { return St{P.VB[p], P.LB64[p], yb[p]}; },
        [&](long long p, int, int, const St& s, const T* in, T* out) {
            const T ly = in[0];
            const double lbn = s.lb + (double)ly;
            P.LB64[p] = lbn;
            lbt[p] = (T)lbn;
            const T y = s.y;
            const T b = (T)(s.vb - (double)s.y);
            const T lb = (T)s.lb;
            const T f1b = dF1(b, tau), f2b = dF2(b, tau);
            const T df1 = y * ((T)3 * b * b + (T)3 * b * y + y * y + tau * ((T)2 * b + y) - (T)1);
            const T df2 = y * ((T)6 * b + (T)3 * y + (T)2 * tau);
            const T f1n = f1b + df1, f2n = f2b + df2;
            out[0] = df1;
            out[1] = -e2 * (df2 * lb + (f2n - eta1) * ly) + df2 * f1n + (f2b - eta2) * df1;
        });
}

template <class T, int NF>
__device__ PAGD_COLD void phase_EN(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    using C = cx<T>;
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    const double e2 = P.eps * P.eps;
    const double l1 = lam_at(P, 1);
    const long long H = P.H;
    struct St { double2 lin, f1, pp; };
    colp<T, NF, true>(
        P, tw, 2, 2, csrcT<T>(P), cdstT<T>(P), smem,
        [&](int k1, int k0) {
            const long long idx = (long long)k1 * P.n0 + k0;
            return St{P.CL64[idx], P.NR64[idx], P.NR64[idx + H]};
        },
        [&](int k1, int k0, const St& s, const C* in, C* out) {
            const long long idx = (long long)k1 * P.n0 + k0;
            const double kap = kappa_at(P, k1, k0);
            const double2 f1{s.f1.x + (double)in[0].x, s.f1.y + (double)in[0].y};
            const double2 pp{s.pp.x + (double)in[1].x, s.pp.y + (double)in[1].y};
            P.NR64[idx] = f1;
            P.NR64[idx + H] = pp;
            double2 G{0.0, 0.0};
            if (kap != 0.0) {
                G.x = s.lin.x + e2 * kap * f1.x + pp.x;
                G.y = s.lin.y + e2 * kap * f1.y + pp.y;
            }
            double2 d;
            base_direction<T>(P, k, B, k1, k0, kap, G, d);
            out[0] = C{(T)d.x, (T)d.y};
            const double f = -kap * (1.0 + l1) * k.ts;
            out[1] = C{(T)(f * d.x), (T)(f * d.y)};
        });
}

// Constants of the iteration row pass at iteration it of the step.
template <class T> struct RowK {
    T lp, l, ts, tau, e2, eta1, eta2;
};
template <class T> __device__ __forceinline__ RowK<T> row_consts(const Params& P, const Ctl& c) {
    const StepK& k = step_coeffs(P, c.step);
    return RowK<T>{(T)lam_at(P, c.it - 1), (T)lam_at(P, c.it), (T)k.ts, (T)P.tau, (T)(P.eps * P.eps),
                   (T)P.eta1,            (T)P.eta2};
}

// One point of the iteration row pass: delta_{i+1} from the direction
// (Algorithm 2's update in the correction form) written over delta_{i-1}, the
// max-norm and sum accumulators, the extrapolated iterate y and the nonlinear
// term(s) at it (PFC: (b + y)^3 - b^3; FCH: the differences of F' and of the
// second variation's nonlinear part).
template <class T, class TI, bool PFC>
__device__ __forceinline__ void row_point(const RowK<T>& q, T* dcur, long long p, T dp, T dpp, T b, T lb,
                                          const TI* in, T* out, TI& amax, double& asum) {
    const TI dd = in[0];
    const T de = dp + q.lp * (dp - dpp) + q.ts * (T)dd;
    dcur[p] = de;
    const TI ad = fabs(dd);
    amax = (ad > amax || ad != ad) ? ad : amax;
    asum += (double)de;
    const T y = de + q.l * (de - dp);
    if (PFC) {
        out[0] = y * ((T)3 * b * b + (T)3 * b * y + y * y);
    } else {
        const T tau = q.tau;
        const T ly = (T)in[1];
        const T f1b = dF1(b, tau), f2b = dF2(b, tau);
        const T df1 = y * ((T)3 * b * b + (T)3 * b * y + y * y + tau * ((T)2 * b + y) - (T)1);
        const T df2 = y * ((T)6 * b + (T)3 * y + (T)2 * tau);
        const T f1n = f1b + df1, f2n = f2b + df2;
        out[0] = df1;
        out[1] = -q.e2 * (df2 * lb + (f2n - q.eta1) * ly) + df2 * f1n + (f2b - q.eta2) * df1;
    }
}

// The FP32 iteration row pass with staged inputs (row_pass_staged): its own
// function, so that its registers are allocated apart from the general
// pass's.  PFC: one field, state delta_i, delta_{i-1}, base; FCH: two fields
// (the direction and its Laplacian), and the base's Laplacian as fourth state.
template <int NF, bool PFC>
__device__ __noinline__ void phase_R_staged(const Params& P, const Ctl& c, const Tw& tw, char* smem,
                                            const float2* src) {
    constexpr int K = PFC ? 1 : 2, NS = staged_row_state(PFC ? 0 : 1), SL = staged_slots(PFC ? 0 : 1);
    const RowK<float> q = row_consts<float>(P, c);
    const int bank = c.step & 1;
    float* dcur = (float*)P.DD[c.it & 1];
    const float* sp[4] = {(const float*)P.DD[(c.it - 1) & 1], dcur, (const float*)P.VBt, (const float*)P.LBt};
    float amax = 0.f;
    double asum = 0.0;
    row_pass_staged<NF, K, NS, SL>(P, tw, src, (float2*)P.NB, sp, smem,
                                   [&](long long p, int, int, const float* sv, const float* in, float* out) {
                                       row_point<float, float, PFC>(q, dcur, p, sv[0], sv[1], sv[2],
                                                                    NS > 3 ? sv[NS > 3 ? 3 : 0] : 0.f, in, out,
                                                                    amax, asum);
                                   });
    publish_max(&P.norms[(size_t)bank * P.nslots + c.ev], (double)amax);
    publish_sum(&P.sums[(size_t)bank * P.nslots + c.ev], asum);
}

// The FP32 iteration row pass with CTA-cooperative units (row_pass_coop), an
// opt-in alternative (Params::coop32) for grids with fewer row units than
// SMs, where one warp per unit leaves most of an SM idle.
template <int NF>
__device__ __noinline__ void phase_R_coop(const Params& P, const Ctl& c, const Tw& tw, char* smem, const float2* src) {
    const RowK<float> q = row_consts<float>(P, c);
    const int bank = c.step & 1;
    float* dcur = (float*)P.DD[c.it & 1];
    const float* dprev = (const float*)P.DD[(c.it - 1) & 1];
    const float* vbt = (const float*)P.VBt;
    const float* lbt = (const float*)P.LBt;
    const int K = k_iter(P.model);
    const bool pfc = P.model == M_PFC;
    float amax = 0.f;
    double asum = 0.0;
    struct St { float dp, dpp, b, lb; };
    row_pass_coop<float, float, NF>(
        P, tw, K, K, src, (float2*)P.NB, smem,
        [&](long long p, int, int) { return St{dprev[p], dcur[p], vbt[p], pfc ? 0.f : lbt[p]}; },
        [&](long long p, int, int, const St& s, const float* in, float* out) {
            if (pfc) row_point<float, float, true>(q, dcur, p, s.dp, s.dpp, s.b, s.lb, in, out, amax, asum);
            else row_point<float, float, false>(q, dcur, p, s.dp, s.dpp, s.b, s.lb, in, out, amax, asum);
        });
    // every warp publishes its threads' norm and sum
    publish_max(&P.norms[(size_t)bank * P.nslots + c.ev], (double)amax);
    publish_sum(&P.sums[(size_t)bank * P.nslots + c.ev], asum);
}

// Iteration row pass (R1 reads the FP64 base direction, RI the T one):
// delta_it = ybar_{it-1} + theta_v s d_{it-1}; ||d_{it-1}||_inf; then the
// nonlinear differences at ybar_it and their forward x-DFT.
template <class TI, class T, int NF>
__device__ PAGD_HOT void phase_R(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red,
                        const cx<TI>* src) {
    if constexpr (sizeof(TI) == 4 && sizeof(T) == 4 && (NF & (kNoCoop - 1)) != 0) {
        if (P.stage) {
            if (P.model == M_PFC) phase_R_staged<NF & (kNoCoop - 1), true>(P, c, tw, smem, (const float2*)src);
            else phase_R_staged<NF & (kNoCoop - 1), false>(P, c, tw, smem, (const float2*)src);
            return;
        }
        if constexpr (!(NF & kNoCoop)) {
            if (P.coop32) {
                phase_R_coop<NF>(P, c, tw, smem, (const float2*)src);
                return;
            }
        }
    }
    const RowK<T> q = row_consts<T>(P, c);
    const int it = c.it;
    const int bank = c.step & 1;
    T* dcur = (T*)P.DD[it & 1];
    const T* dprev = (const T*)P.DD[(it - 1) & 1];
    const T* vbt = (const T*)P.VBt;
    const T* lbt = (const T*)P.LBt;
    const int K = k_iter(P.model);
    TI amax = (TI)0;
    double asum = 0.0;
    const bool pfc = P.model == M_PFC;
    struct St { T dp, dpp, b, lb; };
    rowp<TI, T, NF>(
        P, tw, K, K, src, (cx<T>*)P.NB, smem,
        [&](long long p, int, int) {
            St s;
            s.dp = dprev[p];
            s.dpp = dcur[p];
            s.b = vbt[p];
            s.lb = pfc ? (T)0 : lbt[p];
            return s;
        },
        [&](long long p, int, int, const St& s, const TI* in, T* out) {
            if (pfc) row_point<T, TI, true>(q, dcur, p, s.dp, s.dpp, s.b, s.lb, in, out, amax, asum);
            else row_point<T, TI, false>(q, dcur, p, s.dp, s.dpp, s.b, s.lb, in, out, amax, asum);
        });
    publish_max(&P.norms[(size_t)bank * P.nslots + c.ev], (double)amax);
    publish_sum(&P.sums[(size_t)bank * P.nslots + c.ev], asum);
}

// Constants of the iteration column pass: the momentum factors, theta_v s, the
// preconditioner's coefficients (averaged-Newton betas, Sec. 3.4.1) and the
// linear part's in the iteration precision.
template <class T> struct ColK {
    T l, ln, ts, m2, b0, b2, b4, aim, c0, e2, e4;
};
template <class T> __device__ __forceinline__ ColK<T> col_consts(const Params& P, const Ctl& c) {
    const StepK& k = step_coeffs(P, c.step);
    const Beta B = betas(P, k, c.bsel);
    const T e2 = (T)(P.eps * P.eps);
    return ColK<T>{(T)lam_at(P, c.it), (T)lam_at(P, c.it + 1), (T)k.ts, (T)B.m2, (T)B.b0, (T)B.b2, (T)B.b4,
                   (T)(k.Ai / P.M),   (T)(1.0 - P.eps),       e2,       e2 * e2};
}

// One wavenumber of the iteration column pass: ybar_hat, the spectral residual
// (Eq. obj:G' with the zero mode removed), d_hat = r_hat / Lcal_hat (Algorithm
// 2), the spectral state update written over the older state, and the outputs
// to transform (d_hat; FCH also the Laplacian of ybar_{it+1}).
template <class T, bool PFC>
__device__ __forceinline__ void col_point(const Params& P, const ColK<T>& q, cx<T>* sprev, int k1, int k0, cx<T> sc,
                                          cx<T> sp, cx<T> g0, const cx<T>* in, cx<T>* out) {
    using C = cx<T>;
    const long long idx = (long long)k1 * P.n0 + k0;
    const T kap = kappa_t<T>(P, k1, k0);
    const C yh = C{sc.x + q.l * (sc.x - sp.x), sc.y + q.l * (sc.y - sp.y)};
    C d{(T)0, (T)0};
    if (kap != (T)0) {
        const T ik = (T)1 / kap;
        const T il = (T)-1 / (q.m2 * ik + q.b0 + q.b2 * kap + q.b4 * kap * kap);
        if (PFC) {
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
    const C sn = C{yh.x + q.ts * d.x, yh.y + q.ts * d.y};
    sprev[idx] = sn;
    out[0] = d;
    if (!PFC) {
        const T f = -kap;
        out[1] = C{f * (sn.x + q.ln * (sn.x - sc.x)), f * (sn.y + q.ln * (sn.y - sc.y))};
    }
}

// The FP32 iteration column pass with staged inputs (col_pass_staged): K
// fields out (PFC: the direction; FCH: also the Laplacian of ybar_{it+1}).
template <int NF, bool PFC>
__device__ __noinline__ void phase_CI_staged(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    constexpr int K = PFC ? 1 : 2, SL = staged_slots(PFC ? 0 : 1);
    const ColK<float> q = col_consts<float>(P, c);
    float2* sprev = (float2*)P.SS[(c.it - 1) & 1];
    const float2* sc3[3] = {(const float2*)P.SS[c.it & 1], sprev, (const float2*)P.C0};
    col_pass_staged<NF, K, 3, SL>(P, tw, csrcT<float>(P), cdstT<float>(P), sc3, smem,
                                  [&](int k1, int k0, const float2* sv, const float2* in, float2* out) {
                                      col_point<float, PFC>(P, q, sprev, k1, k0, sv[0], sv[1], sv[2], in, out);
                                  });
}

// The FP32 iteration column pass with CTA-cooperative units (col_pass_coop).
template <int NF>
__device__ __noinline__ void phase_CI_coop(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    const ColK<float> q = col_consts<float>(P, c);
    const float2* scur = (const float2*)P.SS[c.it & 1];
    float2* sprev = (float2*)P.SS[(c.it - 1) & 1];
    const float2* C0 = (const float2*)P.C0;
    const int K = k_iter(P.model);
    const bool pfc = P.model == M_PFC;
    struct St { float2 sc, sp, g0; };
    col_pass_coop<float, float, NF>(
        P, tw, K, K, csrcT<float>(P), cdstT<float>(P), smem,
        [&](int k1, int k0) {
            const long long idx = (long long)k1 * P.n0 + k0;
            return St{scur[idx], sprev[idx], C0[idx]};
        },
        [&](int k1, int k0, const St& s, const float2* in, float2* out) {
            if (pfc) col_point<float, true>(P, q, sprev, k1, k0, s.sc, s.sp, s.g0, in, out);
            else col_point<float, false>(P, q, sprev, k1, k0, s.sc, s.sp, s.g0, in, out);
        });
}

// Iteration column pass: ybar_hat, spectral residual, preconditioned
// direction and spectral state update (col_point), and the inverse y-DFT of d
// (and of Lap ybar_{it+1} for FCH).
template <class T, int NF>
__device__ PAGD_HOT void phase_CI(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    using C = cx<T>;
    if constexpr (sizeof(T) == 4 && (NF & (kNoCoop - 1)) != 0) {
        if (P.stage) {
            if (P.model == M_PFC) phase_CI_staged<NF & (kNoCoop - 1), true>(P, c, tw, smem);
            else phase_CI_staged<NF & (kNoCoop - 1), false>(P, c, tw, smem);
            return;
        }
        if constexpr (!(NF & kNoCoop)) {
            if (P.coop32) {
                phase_CI_coop<NF>(P, c, tw, smem);
                return;
            }
        }
    }
    const ColK<T> q = col_consts<T>(P, c);
    const int it = c.it;
    const C* scur = (const C*)P.SS[it & 1];
    C* sprev = (C*)P.SS[(it - 1) & 1];
    const C* C0 = (const C*)P.C0;
    const int K = k_iter(P.model);
    const bool pfc = P.model == M_PFC;
    struct St { C sc, sp, g0; };
    colp<T, NF>(
        P, tw, K, K, csrcT<T>(P), cdstT<T>(P), smem,
        [&](int k1, int k0) {
            const long long idx = (long long)k1 * P.n0 + k0;
            return St{scur[idx], sprev[idx], C0[idx]};
        },
        [&](int k1, int k0, const St& s, const C* in, C* out) {
            if (pfc) col_point<T, true>(P, q, sprev, k1, k0, s.sc, s.sp, s.g0, in, out);
            else col_point<T, false>(P, q, sprev, k1, k0, s.sc, s.sp, s.g0, in, out);
        });
}

// Accept of the last step of a launch: u^{n+1} = (VB + delta - mean(delta)
// - (1 - theta_v) u^n) / theta_v, written over u^{n-1}.  (Earlier steps are
// accepted inside the next step's phase B.)  The mean of delta is zero in exact
// arithmetic (Remark on discrete mass conservation) and is removed in FP64.
template <class T>
__device__ PAGD_COLD void phase_accept(const Params& P, const Ctl& c, const Tw& tw, double* red) {
    const StepK& k = step_coeffs(P, c.step);
    const int bank = c.step & 1;
    const T* dc = (const T*)P.DD[c.it & 1];
    const double* un = P.U[c.cur];
    double* unew = P.U[c.cur ^ 1];
    const double m = (ldcg(&P.sums[(size_t)bank * P.nslots + c.lastev]) + ldcg(&P.mass[0])) / (double)P.npts;
    const long long gt = thread_rank(tw);
    const long long gs = thread_count(tw);
    const double ith = 1.0 / k.thv, w = (1.0 - k.thv);
    double dmass = 0.0;
    for (long long p = gt; p < P.npts; p += gs) {
        const double v = P.VB[p] + ((double)dc[p] - m);
        const double a = un[p];
        const double x = (v - w * a) * ith;
        unew[p] = x;
        dmass += x - a;
        if (P.out_real) P.out_real[p] = x;
    }
    publish_sum(&P.mass[1], dmass);
    if (c.rec_pending && leader(tw)) P.mass[2] = bits_dbl(ldcg(&P.norms[(size_t)c.rec_bank * P.nslots + c.rec_ev]));
    if (leader(tw)) {
        P.stats[c.step].iters = c.ev;
        P.stats[c.step].status = ST_OK;
        P.stats[c.step].resid = c.resid;
        P.stats[c.step].used_guess = c.gmode == 1 || c.gmode == 3;
        P.sc->steps_done = c.step + 1;
    }
}

inline __device__ void phase_fail(const Params& P, const Ctl& c, const Tw& tw) {
    if (leader(tw)) {
        P.sc->status = c.fail;
        P.sc->fail_step = c.step;
        P.stats[c.step].iters = c.ev;
        P.stats[c.step].status = c.fail;
        P.stats[c.step].resid = c.resid;
    }
}

// ------------------------------------------------ DFT / energy / mass programs

template <int NF>
__device__ PAGD_COLD void phase_fwd_r(const Params& P, const Tw& tw, char* smem) {
    rowp<double, double, NF>(P, tw, 0, 1, (const double2*)nullptr, P.NB64, smem,
                             [&](long long p, int, int) { return P.in_real[p]; },
                             [&](long long, int, int, const double& u, const double*, double* out) { out[0] = u; });
}
template <int NF>
__device__ PAGD_COLD void phase_fwd_c(const Params& P, const Tw& tw, char* smem) {
    colp<double, NF>(P, tw, 1, 0, csrc64(P), (double2*)nullptr, smem, [&](int, int) { return Nil{}; },
                     [&](int k1, int k0, const Nil&, const double2* in, double2*) {
                         P.out_spec[api_spec_index(P, k1, k0)] = in[0];
                     });
}
template <int NF>
__device__ PAGD_COLD void phase_inv_c(const Params& P, const Tw& tw, char* smem) {
    colp<double, NF>(P, tw, 0, 1, (const double2*)nullptr, cdst64(P), smem,
                     [&](int k1, int k0) { return P.in_spec[api_spec_index(P, k1, k0)]; },
                     [&](int, int, const double2& v, const double2*, double2* out) { out[0] = v; });
}
template <int NF>
__device__ PAGD_COLD void phase_inv_r(const Params& P, const Tw& tw, char* smem) {
    rowp<double, double, NF>(P, tw, 1, 0, P.DB64, (double2*)nullptr, smem,
                             [&](long long, int, int) { return Nil{}; },
                             [&](long long p, int, int, const Nil&, const double* in, double*) {
                                 P.out_real[p] = in[0];
                             });
}

// energy (Eqs. obj:PFC-egy / obj:FCHegy with Fourier differentiation and the
// trapezoidal rule): red[0] pointwise part, red[1] spectral part
template <int NF>
__device__ PAGD_COLD void phase_en_r(const Params& P, const Tw& tw, char* smem, double* red) {
    double acc = 0.0;
    const bool pfc = P.model == M_PFC;
    rowp<double, double, NF>(P, tw, 0, 1, (const double2*)nullptr, P.NB64, smem,
                             [&](long long p, int, int) { return P.in_real[p]; },
                             [&](long long, int, int, const double& u, const double*, double* out) {
                                 out[0] = u;
                                 if (pfc) acc += 0.25 * u * u * u * u + 0.5 * (1.0 - P.eps) * u * u;
                             });
    if (pfc) {
        publish_sum(&P.sc->red[0], acc);
    }
}
template <int NF>
__device__ PAGD_COLD void phase_en_c(const Params& P, const Tw& tw, char* smem, double* red) {
    double acc = 0.0;
    const bool pfc = P.model == M_PFC;
    const int half = P.n1 >> 1;
    colp<double, NF>(P, tw, 1, pfc ? 0 : 1, csrc64(P), cdst64(P), smem, [&](int, int) { return Nil{}; },
                     [&](int k1, int k0, const Nil&, const double2* in, double2* out) {
                         const double kap = kappa_at(P, k1, k0);
                         const int kl = kl_of(P, k1);
                         const double w = (kl == 0 || kl == half) ? 1.0 : 2.0;
                         const double a2 = in[0].x * in[0].x + in[0].y * in[0].y;
                         if (pfc) {
                             acc += w * (-kap + 0.5 * kap * kap) * a2;
                         } else {
                             acc += w * kap * a2;
                             out[0] = double2{-kap * in[0].x, -kap * in[0].y};
                         }
                     });
    publish_sum(&P.sc->red[1], acc);
}
template <int NF>
__device__ PAGD_COLD void phase_en_r2(const Params& P, const Tw& tw, char* smem, double* red) {
    double acc = 0.0;
    const double e2 = P.eps * P.eps;
    rowp<double, double, NF>(P, tw, 1, 0, P.DB64, (double2*)nullptr, smem,
                             [&](long long p, int, int) { return P.in_real[p]; },
                             [&](long long, int, int, const double& u, const double* in, double*) {
                                 const double w = e2 * in[0] - dF1(u, P.tau);
                                 acc += 0.5 * w * w - P.eta2 * Fwell(u, P.tau);
                             });
    publish_sum(&P.sc->red[0], acc);
}
// Mass shift of the caller's initial guess: the discrete solution keeps the
// mass of u^n and every PAGD update has zero mean, so the initial iterate is
// the guess moved to that mass; red[2] = sum(u^n - guess).
inline __device__ void phase_gs(const Params& P, const Ctl& c, const Tw& tw) {
    double acc = 0.0;
    const double* un = P.U[c.cur];
    const long long gt = thread_rank(tw);
    const long long gs = thread_count(tw);
    for (long long p = gt; p < P.npts; p += gs) acc += un[p] - P.guess[p];
    publish_sum(&P.sc->red[2], acc);
}

inline __device__ void phase_mass(const Params& P, const Tw& tw, double* red) {
    double acc = 0.0;
    const long long gt = thread_rank(tw);
    const long long gs = thread_count(tw);
    for (long long p = gt; p < P.npts; p += gs) acc += P.in_real[p];
    publish_sum(&P.sc->red[0], acc);
}

// ------------------------------------------- right-hand side and estimate
//
// R(v) = M Lap mu(v) (the gradient flow of Sec. 2, sampled by the AM3
// estimator of Sec. 3.1.2), in FP64: PFC mu_hat = N_hat + (1 - eps - 2 kappa +
// kappa^2) v_hat with N = v^3; FCH mu_hat = eps^4 kappa^2 v_hat +
// eps^2 kappa F'_hat + P_hat, P = -eps^2 (F'' - eta1) Lap v + (F'' - eta2) F'.
template <int NF>
__device__ PAGD_COLD void phase_rh_r0(const Params& P, const Tw& tw, char* smem) {
    const bool pfc = P.model == M_PFC;
    rowp<double, double, NF>(P, tw, 0, pfc ? 2 : 1, (const double2*)nullptr, P.NB64, smem,
                             [&](long long p, int, int) { return P.in_real[p]; },
                             [&](long long, int, int, const double& v, const double*, double* out) {
                                 out[0] = v;
                                 if (pfc) out[1] = v * v * v;
                             });
}
template <int NF>
__device__ PAGD_COLD void phase_rh_c0(const Params& P, const Tw& tw, char* smem) {
    const bool pfc = P.model == M_PFC;
    colp<double, NF>(P, tw, pfc ? 2 : 1, 1, csrc64(P), cdst64(P), smem, [&](int, int) { return Nil{}; },
                     [&](int k1, int k0, const Nil&, const double2* in, double2* out) {
                         const double kap = kappa_at(P, k1, k0);
                         if (pfc) {
                             const double Lh = 1.0 - P.eps - 2.0 * kap + kap * kap;
                             const double f = -P.M * kap;
                             out[0] = double2{f * (in[1].x + Lh * in[0].x), f * (in[1].y + Lh * in[0].y)};
                         } else {
                             P.CL64[(long long)k1 * P.n0 + k0] = in[0];
                             out[0] = double2{-kap * in[0].x, -kap * in[0].y};
                         }
                     });
}
template <int NF>
__device__ PAGD_COLD void phase_rh_r1(const Params& P, const Tw& tw, char* smem) {
    const double e2 = P.eps * P.eps;
    rowp<double, double, NF>(P, tw, 1, 2, P.DB64, P.NB64, smem,
                             [&](long long p, int, int) { return P.in_real[p]; },
                             [&](long long, int, int, const double& v, const double* in, double* out) {
                                 const double f1 = dF1(v, P.tau), f2 = dF2(v, P.tau);
                                 out[0] = f1;
                                 out[1] = -e2 * (f2 - P.eta1) * in[0] + (f2 - P.eta2) * f1;
                             });
}
template <int NF>
__device__ PAGD_COLD void phase_rh_c1(const Params& P, const Tw& tw, char* smem) {
    const double e2 = P.eps * P.eps, e4 = e2 * e2;
    colp<double, NF>(P, tw, 2, 1, csrc64(P), cdst64(P), smem,
                     [&](int k1, int k0) { return P.CL64[(long long)k1 * P.n0 + k0]; },
                     [&](int k1, int k0, const double2& v, const double2* in, double2* out) {
                         const double kap = kappa_at(P, k1, k0);
                         const double f = -P.M * kap;
                         const double mr = e4 * kap * kap * v.x + e2 * kap * in[0].x + in[1].x;
                         const double mi = e4 * kap * kap * v.y + e2 * kap * in[0].y + in[1].y;
                         out[0] = double2{f * mr, f * mi};
                     });
}
// Error estimate of adaptive stepping: uh = sum_j c_j in_j (the AM3 or midAB2
// higher-order value), red[0] = sum (ut - uh)^2, red[1] = sum uh^2 (the cell
// volume cancels in their ratio); ut = in_real.
inline __device__ void phase_est(const Params& P, const Tw& tw) {
    double e = 0.0, h = 0.0;
    const long long gt = thread_rank(tw);
    const long long gs = thread_count(tw);
    for (long long p = gt; p < P.npts; p += gs) {
        double uh = 0.0;
        for (int j = 0; j < 4; j++)
            if (P.est_in[j]) uh += P.est_c[j] * P.est_in[j][p];
        const double d = P.in_real[p] - uh;
        e += d * d;
        h += uh * uh;
    }
    publish_sum(&P.sc->red[0], e);
    publish_sum(&P.sc->red[1], h);
}

// ------------------------------------------------------ linear IMEX step
//
// Eq. eqn:FCH-semidis-simplicit with the splits of Sec. 3.1.1, solved per
// wavenumber (Sec. 3.3), in FP64:
//   IM_R0: ubreve (extrapolation) and the forward x-DFT of
//          (N(ubreve) or ubreve, u^n, u^{n-1})
//   IM_C0: (PFC) solve; (FCH) keep u^n, u^{n-1} spectra, inverse y-DFT of -kappa ubreve
//   IM_R1: (FCH) Lap ubreve physical, forward x-DFT of (F'(ub), Q(ub))
//   IM_C1: (FCH) solve
//   IM_R2: inverse x-DFT of u^{n+1} -> written over u^{n-1}
template <int NF>
__device__ PAGD_COLD void phase_im_r0(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    const StepK& k = step_coeffs(P, c.step);
    const double* un = P.U[c.cur];
    const double* um = P.U[c.cur ^ 1];
    const bool pfc = P.model == M_PFC;
    const bool lmp = P.scheme == S_LMP;
    rowp<double, double, NF>(P, tw, 0, 3, (const double2*)nullptr, P.NB64, smem,
                             [&](long long p, int, int) { return double2{un[p], um[p]}; },
                             [&](long long p, int, int, const double2& ab, const double*, double* out) {
                                 const double a = ab.x, b = ab.y;
                                 const double ub = lmp ? 0.5 * ((2.0 + k.rho) * a - k.rho * b)
                                                       : a + k.rho * (a - b);
                                 P.VB[p] = ub;
                                 out[0] = pfc ? ub * ub * ub - P.eps * ub : ub;
                                 out[1] = a;
                                 out[2] = b;
                             });
}
// per-wavenumber solve; nh = N_hat(ubreve)
__device__ __forceinline__ double2 imex_solve(const Params& P, const StepK& k, double kap,
                                              double2 nh, double2 un, double2 um) {
    const double M = P.M;
    double Lh;
    if (P.model == M_PFC) Lh = (1.0 - kap) * (1.0 - kap);
    else {
        const double e2 = P.eps * P.eps;
        Lh = e2 * e2 * kap * kap + kap + (1.0 - 2.0 * P.tau * P.tau + P.eta2);
    }
    const double half = (P.scheme == S_LMP) ? 0.5 : 1.0;
    double rx = -k.b * un.x - k.c * um.x - M * kap * nh.x;
    double ry = -k.b * un.y - k.c * um.y - M * kap * nh.y;
    if (P.scheme == S_LMP) {
        rx -= M * kap * 0.5 * Lh * un.x;
        ry -= M * kap * 0.5 * Lh * un.y;
    }
    const double den = k.a + M * kap * half * Lh;
    return double2{rx / den, ry / den};
}
template <int NF>
__device__ PAGD_COLD void phase_im_c0(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    const StepK& k = step_coeffs(P, c.step);
    if (P.model == M_PFC) {
        colp<double, NF>(P, tw, 3, 1, csrc64(P), cdst64(P), smem, [&](int, int) { return Nil{}; },
                         [&](int k1, int k0, const Nil&, const double2* in, double2* out) {
                             const double kap = kappa_at(P, k1, k0);
                             out[0] = imex_solve(P, k, kap, in[0], in[1], in[2]);
                         });
    } else {
        colp<double, NF>(P, tw, 3, 1, csrc64(P), cdst64(P), smem, [&](int, int) { return Nil{}; },
                         [&](int k1, int k0, const Nil&, const double2* in, double2* out) {
                             const double kap = kappa_at(P, k1, k0);
                             const long long idx = (long long)k1 * P.n0 + k0;
                             P.CL64[idx] = in[1];
                             P.CL64[idx + P.H] = in[2];
                             out[0] = double2{-kap * in[0].x, -kap * in[0].y};
                         });
    }
}
template <int NF>
__device__ PAGD_COLD void phase_im_r1(const Params& P, const Tw& tw, char* smem) {
    // N(u) = -kappa0 u - eps^2 Lap F'(u) - (eps^2 (F'' - eta1) - kappa2) Lap u + (F'' - eta2) F'
    const double e2 = P.eps * P.eps, kap0 = 1.0 - 2.0 * P.tau * P.tau + P.eta2;
    rowp<double, double, NF>(P, tw, 1, 2, P.DB64, P.NB64, smem,
                             [&](long long p, int, int) { return P.VB[p]; },
                             [&](long long, int, int, const double& ub, const double* in, double* out) {
                                 const double lu = in[0];
                                 const double f1 = dF1(ub, P.tau), f2 = dF2(ub, P.tau);
                                 out[0] = f1;
                                 out[1] = -kap0 * ub - (e2 * (f2 - P.eta1) - 1.0) * lu + (f2 - P.eta2) * f1;
                             });
}
template <int NF>
__device__ PAGD_COLD void phase_im_c1(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    const StepK& k = step_coeffs(P, c.step);
    const double e2 = P.eps * P.eps;
    struct St { double2 un, um; };
    colp<double, NF>(P, tw, 2, 1, csrc64(P), cdst64(P), smem,
                     [&](int k1, int k0) {
                         const long long idx = (long long)k1 * P.n0 + k0;
                         return St{P.CL64[idx], P.CL64[idx + P.H]};
                     },
                     [&](int k1, int k0, const St& s, const double2* in, double2* out) {
                         const double kap = kappa_at(P, k1, k0);
                         // -eps^2 Lap F' -> + eps^2 kappa F'_hat
                         const double2 nh{e2 * kap * in[0].x + in[1].x, e2 * kap * in[0].y + in[1].y};
                         out[0] = imex_solve(P, k, kap, nh, s.un, s.um);
                     });
}
template <int NF>
__device__ PAGD_COLD void phase_im_r2(const Params& P, const Ctl& c, const Tw& tw, char* smem) {
    double* unew = P.U[c.cur ^ 1];
    const bool last = (c.step + 1 == P.nsteps) && P.out_real;
    rowp<double, double, NF>(P, tw, 1, 0, P.DB64, (double2*)nullptr, smem,
                             [&](long long, int, int) { return Nil{}; },
                             [&](long long p, int, int, const Nil&, const double* in, double*) {
                                 unew[p] = in[0];
                                 if (last) P.out_real[p] = in[0];
                             });
    if (leader(tw)) {
        P.stats[c.step].iters = 0;
        P.stats[c.step].status = ST_OK;
        P.stats[c.step].resid = 0.0;
        P.sc->steps_done = c.step + 1;
    }
}

// ------------------------------------------------------------ control

// Whether the next base evaluation is incremental: FP32-mixed only, once a
// reference point exists, except for the first evaluation of every refresh-th
// step, which recomputes the reference spectra exactly in FP64.  The
// incremental evaluation errs by about 1e-7 of the base shift, so it only seeds
// iterations: the first acceptance check of every step is an exact FP64
// evaluation (the caller passes new_step = 0 and requires exact_done).
__host__ __device__ inline int inc_eval(const Params& P, int ref_ok, int gstep, int new_step) {
    if (P.precision != P_MIXED || !ref_ok) return 0;
    if (new_step && P.refresh > 0 && gstep % P.refresh == 0) return 0;
    return 1;
}

__host__ __device__ inline Ctl ctl_init(const Params& P) {
    Ctl c;
    c.step = 0; c.it = 0; c.ev = 0; c.lastev = 0; c.cur = P.cur0; c.rech = 0; c.fail = 0;
    c.best_ev = 0; c.acc = 0; c.acc_cur = 0; c.acc_it = 0; c.acc_lastev = 0; c.acc_ev = 0; c.reb = 0;
    c.ref_ok = P.ref_valid;
    c.exact_done = 0;
    c.ereb = 0;
    c.after = PH_DONE; c.mk = 0; c.m64 = 1;
    c.gok = 0;
    c.bsel = 0;  // bank of the launch's first step (c.step & 1)
    c.gmode = 0;
    c.gnorm = 0.0;
    c.acc_used = 0;
    c.rec_pending = 0; c.rec_ev = 0; c.rec_bank = 0;
    c.inc = inc_eval(P, c.ref_ok, P.step0, 1);
    c.resid = 0.0; c.base_nrm = 0.0; c.best_nrm = 0.0; c.acc_resid = 0.0;
    switch (P.prog) {
        case PROG_RUN:
            c.ph = (P.nsteps > 0) ? PH_B : PH_DONE;
            if (P.nsteps > 0 && P.guess) {
                c.ph = PH_GS;  // the guess's mass shift first
                c.gmode = 1;
                c.bsel = 2;
            }
            break;
        case PROG_IMEX: c.ph = (P.nsteps > 0) ? PH_IM_R0 : PH_DONE; break;
        case PROG_FFT_FWD: c.ph = PH_FWD_R; break;
        case PROG_FFT_INV: c.ph = PH_INV_C; break;
        case PROG_ENERGY: c.ph = PH_EN_R; break;
        case PROG_RHS: c.ph = PH_RH_R0; break;
        case PROG_EST: c.ph = PH_EST; break;
        case PROG_BARRIER: c.ph = (P.nsteps > 0) ? PH_NOP : PH_DONE; break;
        case PROG_PASS:
            // one iteration pass repeated on the buffers of the last step, as
            // iteration 1 of the step (a middle pass in the iterations' form:
            // the iteration fields, in T)
            c.ph = (P.nsteps > 0) ? P.pass : PH_DONE;
            c.it = 1;
            c.ev = 1;
            c.m64 = 0;
            c.mk = k_iter(P.model);
            break;
        default: c.ph = PH_MASS; break;
    }
    return c;
}

// phases by pass type, for the 3D middle passes and the batched schedule
__host__ __device__ inline bool phase_is_col(int ph) {
    return ph == PH_C || ph == PH_E || ph == PH_CI || ph == PH_IM_C0 || ph == PH_IM_C1 || ph == PH_FWD_C ||
           ph == PH_INV_C || ph == PH_EN_C || ph == PH_RH_C0 || ph == PH_RH_C1;
}
__host__ __device__ inline bool phase_is_mid(int ph) { return ph == PH_MF || ph == PH_MI; }
// row passes that read a half spectrum written by the column pass before them
__host__ __device__ inline bool row_reads_spectrum(int ph) {
    return ph == PH_D || ph == PH_R1 || ph == PH_RI || ph == PH_INV_R || ph == PH_EN_R2 || ph == PH_IM_R1 ||
           ph == PH_IM_R2 || ph == PH_RH_R1 || ph == PH_RH_R2;
}

// 3D: put a middle pass between a row pass and the column pass after it (MF)
// and between a column pass and a row pass that reads its output (MI).  pph,
// pinc, preb: the phase that just ran and its incremental / rebase flags,
// which fix the number of spectral fields it wrote and their buffer set.
__host__ __device__ inline void mid_insert(const Params& P, int pph, int pinc, int preb, int pgok, Ctl& c) {
    const int nx = c.ph;
    const int K = k_iter(P.model), kb = k_base(P.model);
    int k = 0, m64 = 1, ph = -1;
    if (!phase_is_col(pph) && !phase_is_mid(pph) && phase_is_col(nx)) {
        ph = PH_MF;
        switch (pph) {
            case PH_B: k = (preb && (pinc || pgok)) ? kb - 1 : kb; m64 = !pinc; break;
            case PH_D: k = 2; m64 = !pinc; break;
            case PH_R1:
            case PH_RI: k = K; m64 = 0; break;
            case PH_IM_R0: k = 3; break;
            case PH_IM_R1: k = 2; break;
            case PH_RH_R0: k = (P.model == M_PFC) ? 2 : 1; break;
            case PH_RH_R1: k = 2; break;
            default: k = 1; break;  // FWD_R, EN_R
        }
    } else if (phase_is_col(pph) && row_reads_spectrum(nx)) {
        ph = PH_MI;
        switch (pph) {
            case PH_C: k = 1; m64 = (P.model == M_FCH) && !pinc; break;  // PFC: direction in T
            case PH_E: k = 2; m64 = 0; break;
            case PH_CI: k = K; m64 = 0; break;
            default: k = 1; break;  // INV_C, EN_C, IM_C0, IM_C1
        }
    }
    if (ph < 0) return;
    c.after = nx;
    c.ph = ph;
    c.mk = k;
    c.m64 = m64;
}

// The decision after an evaluation (phase R1 or RI of the evaluation numbered
// c.ev) whose ||d||_inf is nrm: accept, fail, probe the other initial guess,
// move the base, or iterate on (c.ph = PH_CI).  Shared by the device-wide phase
// sequence and the cluster-resident iteration loop, so both take the same
// decisions from the same norms.
template <class T>
__device__ void ctl_eval(const Params& P, Ctl& c, double nrm) {
    const bool t64 = sizeof(T) == 8;
    const int bank = c.step & 1;
    c.lastev = c.ev;
    c.ev++;
    c.resid = nrm;
    if (!(nrm <= 1.0e300)) { c.fail = ST_ENAN; c.ph = PH_FAIL; return; }
    if (c.ph == PH_R1 || nrm < c.best_nrm) { c.best_nrm = nrm; c.best_ev = c.ev; }
    if (c.ph == PH_R1) c.base_nrm = nrm;
    // the first direction of a step from the extrapolation (Sec. 3.4.2): the
    // record a caller's guess is judged against
    if (c.ph == PH_R1 && !c.ereb && (c.gmode == 0 || c.gmode == 2 || c.gmode == 4)) {
        c.rec_pending = 1;
        c.rec_ev = c.lastev;
        c.rec_bank = bank;
    }
    const double rec = (c.ph == PH_R1 && c.gmode == 1 && !c.ereb) ? ldcg(&P.mass[2]) : 0.0;
    if (c.ph == PH_R1 && c.gmode == 1 && !c.ereb && rec > 0.0 && nrm <= rec) {
        c.gmode = 3;  // the guess is kept: no second probe, it iterates on from here
    }
    const bool fp32_norm = P.precision == P_MIXED && !t64 && c.ph == PH_RI;
    // Only an exact FP64 evaluation certifies a step.  An incremental
    // base evaluation (T transforms of the shift from the reference
    // point) errs by about 1e-7 of that shift, so when its norm reaches
    // tol the base moves there and is evaluated exactly.
    const bool inc_norm = c.ph == PH_R1 && c.inc;
    if (nrm <= P.tol && !fp32_norm && !inc_norm) {
        if (c.step + 1 < P.nsteps) {
            // accepted inside the next step's phase B
            c.acc = 1;
            c.acc_cur = c.cur;
            c.acc_it = c.it;
            c.acc_lastev = c.lastev;
            c.acc_ev = c.ev;
            c.acc_resid = nrm;
            c.acc_used = c.gmode == 1 || c.gmode == 3;
            c.step++;
            c.cur ^= 1;
            c.exact_done = 0;
            c.gok = 0;
            c.gmode = 0;
            c.bsel = c.step & 1;
            c.inc = t64 ? 0 : inc_eval(P, c.ref_ok, P.step0 + c.step, 1);
            c.ph = PH_B;
        } else {
            c.ph = PH_ACCEPT;
        }
    } else if (c.ev >= P.max_iter || c.ev + 1 >= P.nslots) {
        c.fail = ST_ENOCONV;
        c.ph = PH_FAIL;
    } else if (c.ph == PH_R1 && c.gmode == 1 && rec > 0.0 && nrm > rec) {
        // the guess's first direction is larger than the extrapolation's was
        // on the last step: start this step over from the extrapolation
        c.gmode = 4;
        c.bsel = bank;
        c.inc = t64 ? 0 : inc_eval(P, c.ref_ok, P.step0 + c.step, 1);
        c.ph = PH_B;
    } else if (c.ph == PH_R1 && c.gmode == 1 && !(rec > 0.0)) {
        // no record yet: the first direction at the extrapolated guess as
        // well, and the smaller of the two is kept
        c.gnorm = nrm;
        c.gmode = 2;
        c.bsel = bank;
        c.inc = t64 ? 0 : inc_eval(P, c.ref_ok, P.step0 + c.step, 1);
        c.ph = PH_B;
    } else if (c.ph == PH_R1 && c.gmode == 2 && nrm > c.gnorm) {
        c.gmode = 3;  // back to the caller's guess
        c.bsel = 3;
        c.inc = t64 ? 0 : inc_eval(P, c.ref_ok, P.step0 + c.step, 1);
        c.ph = PH_B;
    } else if ((fp32_norm && (nrm <= P.tol || nrm <= kRebaseRatio * c.base_nrm ||
                              c.ev - c.best_ev >= kStagnation)) ||
               (inc_norm && nrm <= P.tol)) {
        if (c.rech >= P.max_recheck) { c.fail = ST_ENOCONV; c.ph = PH_FAIL; return; }
        c.rech++;
        c.reb = 1;
        // a rebase that may accept is evaluated exactly; one that only
        // moves the base past the FP32 floor may be incremental
        c.inc = (nrm <= P.tol || !c.exact_done) ? 0 : inc_eval(P, c.ref_ok, P.step0 + c.step, 0);
        c.ph = PH_B;
    } else {
        c.ph = PH_CI;
    }
}

template <class T>
__device__ void ctl_step(const Params& P, Ctl& c);

// Decide the next phase.  Runs identically in every thread of every CTA after a
// grid barrier; only device-global values that were final before the barrier
// are read.
template <class T>
__device__ void ctl_advance(const Params& P, Ctl& c) {
    if (P.prog == PROG_PASS) {
        c.step++;
        if (c.step >= P.nsteps) c.ph = PH_DONE;
        return;
    }
    if (phase_is_mid(c.ph)) {
        c.ph = c.after;
        return;
    }
    const int pph = c.ph, pinc = c.inc, preb = c.reb, pgok = c.gok;
    ctl_step<T>(P, c);
    if (P.nm > 1) mid_insert(P, pph, pinc, preb, pgok, c);
}

template <class T>
__device__ void ctl_step(const Params& P, Ctl& c) {
    const int bank = c.step & 1;
    switch (c.ph) {
        case PH_GS: c.ph = PH_B; break;
        case PH_B:
            // a new step restarts the counts, except the repeated new-step
            // evaluations of the guess probe (they count in the step's cost)
            if (!c.reb && c.gmode != 2 && c.gmode != 3 && c.gmode != 4) { c.ev = 0; c.rech = 0; }
            c.rec_pending = 0;  // phase B stored it
            c.ereb = c.reb;  // the evaluation started by B is a rebase (kept through C..E)
            c.acc = 0;
            c.reb = 0;
            c.ph = PH_C;
            break;
        case PH_C:
            if (!c.inc) c.gok = 1;  // GH64 now holds this step's g_hat
            if (P.model == M_FCH) { c.ph = PH_D; break; }
            [[fallthrough]];
        case PH_E:
            c.ref_ok = 1;
            if (!c.inc) c.exact_done = 1;
            if (!(fabs(ldcg(&P.sc->beta_sum[c.bsel][0])) + fabs(ldcg(&P.sc->beta_sum[c.bsel][1])) <= 1.0e300)) {
                c.fail = ST_ENAN;  // non-finite initial guess
                c.ph = PH_FAIL;
                break;
            }
            if (ldcg(&P.sc->flags) & FLAG_PRECOND) { c.fail = ST_EPRECOND; c.ph = PH_FAIL; break; }
            c.ph = PH_R1;
            c.it = 1;
            break;
        case PH_D: c.ph = PH_E; break;
        case PH_R1:
        case PH_RI: ctl_eval<T>(P, c, bits_dbl(ldcg(&P.norms[(size_t)bank * P.nslots + c.ev]))); break;
        case PH_CI: c.ph = PH_RI; c.it++; break;
        case PH_ACCEPT: c.step++; c.cur ^= 1; c.ph = PH_DONE; break;
        case PH_IM_R2:
            c.step++;
            c.cur ^= 1;
            c.ph = (c.step >= P.nsteps) ? PH_DONE : PH_IM_R0;
            break;
        case PH_IM_R0: c.ph = PH_IM_C0; break;
        case PH_IM_C0: c.ph = (P.model == M_PFC) ? PH_IM_R2 : PH_IM_R1; break;
        case PH_IM_R1: c.ph = PH_IM_C1; break;
        case PH_IM_C1: c.ph = PH_IM_R2; break;
        case PH_FWD_R: c.ph = PH_FWD_C; break;
        case PH_INV_C: c.ph = PH_INV_R; break;
        case PH_EN_R: c.ph = PH_EN_C; break;
        case PH_EN_C: c.ph = (P.model == M_PFC) ? PH_DONE : PH_EN_R2; break;
        case PH_RH_R0: c.ph = PH_RH_C0; break;
        case PH_RH_C0: c.ph = (P.model == M_PFC) ? PH_RH_R2 : PH_RH_R1; break;
        case PH_RH_R1: c.ph = PH_RH_C1; break;
        case PH_RH_C1: c.ph = PH_RH_R2; break;
        case PH_NOP:
            c.step++;
            c.ph = (c.step >= P.nsteps) ? PH_DONE : PH_NOP;
            break;
        default: c.ph = PH_DONE; break;
    }
}

// Every phase but the iteration and middle passes.  PAGD_DISPATCH chooses
// whether this switch is inlined into the kernel (default) or is one outlined
// call site, which keeps the calls' register saving out of the hot passes.
#ifndef PAGD_DISPATCH
#define PAGD_DISPATCH __forceinline__
#endif
template <class T, int NF>
__device__ PAGD_DISPATCH void exec_cold(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red) {
    switch (c.ph) {
        case PH_B:
            if (c.inc) phase_B_inc<T, NF>(P, c, tw, smem, red);
            else phase_B_exact<T, NF>(P, c, tw, smem, red);
            break;
        case PH_C:
            if (c.inc) phase_CN<T, NF>(P, c, tw, smem);
            else phase_C<T, NF>(P, c, tw, smem);
            break;
        case PH_D:
            if (c.inc) phase_DN<T, NF>(P, tw, smem);
            else phase_D<T, NF>(P, tw, smem);
            break;
        case PH_E:
            if (c.inc) phase_EN<T, NF>(P, c, tw, smem);
            else phase_E<T, NF>(P, c, tw, smem);
            break;
        case PH_ACCEPT: phase_accept<T>(P, c, tw, red); break;
        case PH_FAIL: phase_fail(P, c, tw); break;
        case PH_FWD_R: phase_fwd_r<NF>(P, tw, smem); break;
        case PH_FWD_C: phase_fwd_c<NF>(P, tw, smem); break;
        case PH_INV_C: phase_inv_c<NF>(P, tw, smem); break;
        case PH_INV_R: phase_inv_r<NF>(P, tw, smem); break;
        case PH_EN_R: phase_en_r<NF>(P, tw, smem, red); break;
        case PH_EN_C: phase_en_c<NF>(P, tw, smem, red); break;
        case PH_EN_R2: phase_en_r2<NF>(P, tw, smem, red); break;
        case PH_MASS: phase_mass(P, tw, red); break;
        case PH_GS: phase_gs(P, c, tw); break;
        case PH_RH_R0: phase_rh_r0<NF>(P, tw, smem); break;
        case PH_RH_C0: phase_rh_c0<NF>(P, tw, smem); break;
        case PH_RH_R1: phase_rh_r1<NF>(P, tw, smem); break;
        case PH_RH_C1: phase_rh_c1<NF>(P, tw, smem); break;
        case PH_RH_R2: phase_inv_r<NF>(P, tw, smem); break;
        case PH_EST: phase_est(P, tw); break;
        case PH_IM_R0: phase_im_r0<NF>(P, c, tw, smem); break;
        case PH_IM_C0: phase_im_c0<NF>(P, c, tw, smem); break;
        case PH_IM_R1: phase_im_r1<NF>(P, tw, smem); break;
        case PH_IM_C1: phase_im_c1<NF>(P, c, tw, smem); break;
        case PH_IM_R2: phase_im_r2<NF>(P, c, tw, smem); break;
        default: break;
    }
}

// the FP32 middle passes of a cubic grid run staged (mid_pass_staged) when
// the launch stages its iteration passes; returns whether it ran them (only
// fixed line lengths instantiate the staged pass)
template <class T, int NF, int S>
__device__ __forceinline__ bool mid_pass_staged_if(const Params& P, const Tw& tw, int k, const void* src, void* dst,
                                                   char* smem) {
    if constexpr (sizeof(T) == 4 && (NF & (kNoCoop - 1)) != 0) {
        if (P.stage && P.nm == (NF & (kNoCoop - 1))) {
            mid_pass_staged<NF & (kNoCoop - 1), S>(P, tw, k, (const float2*)src, (float2*)dst, smem);
            return true;
        }
    }
    return false;
}

template <class T, int NF>
__device__ __forceinline__ void exec_phase(const Params& P, const Ctl& c, const Tw& tw, char* smem, double* red) {
    switch (c.ph) {
        case PH_R1:
        case PH_RI: phase_R<T, T, NF>(P, c, tw, smem, red, (const cx<T>*)P.DB); break;
        case PH_CI: phase_CI<T, NF>(P, c, tw, smem); break;
        case PH_MF:
            if (c.m64) mid_pass<double, -1, NF>(P, tw, c.mk, P.NB64, P.X64, smem);
            else if (!mid_pass_staged_if<T, NF, -1>(P, tw, c.mk, P.NB, P.X, smem))
                mid_pass<T, -1, NF>(P, tw, c.mk, (const cx<T>*)P.NB, (cx<T>*)P.X, smem);
            break;
        case PH_MI:
            if (c.m64) mid_pass<double, +1, NF>(P, tw, c.mk, P.NB64, P.DB64, smem);
            else if (!mid_pass_staged_if<T, NF, +1>(P, tw, c.mk, P.NB, P.DB, smem))
                mid_pass<T, +1, NF>(P, tw, c.mk, (const cx<T>*)P.NB, (cx<T>*)P.DB, smem);
            break;
        default: exec_cold<T, NF>(P, c, tw, smem, red); break;
    }
}

// shared memory per warp needed by any phase (bytes, 16-byte multiple);
// nf = 0: runtime-length passes, else the fixed-length ones; nm: middle axis
inline size_t warp_smem_bytes(int n0, int n1, int model, int tsize, int nf, int nm = 1) {
    size_t m = 0;
    auto upd = [&](size_t v) { if (v > m) m = v; };
    if (nm > 1) upd(mid_warp_smem(nm, 8));  // middle passes (3D), FP64 worst case
    const int ki = k_iter(model);
    if (nf == 0) {
        upd(row_warp_smem(n1, 0, 8, 3, 8));            // B (PFC: 3 fields) / IMEX R0
        upd(row_warp_smem(n1, 1, 8, 2, 8));            // D / IMEX R1 / energy / DFT
        upd(row_warp_smem(n1, 0, 8, 1, 8));
        upd(row_warp_smem(n1, ki, 8, ki, tsize));      // R1
        upd(row_warp_smem(n1, ki, tsize, ki, tsize));  // RI
        upd(col_warp_smem(n0, 3, 8));                  // C / IMEX C0
        upd(col_warp_smem(n0, 2, 8));                  // E
        upd(col_warp_smem(n0, ki, tsize));             // CI
        upd(col_warp_smem_mixed(n0, 3, 8, 1, tsize));  // exact C (PFC): FP64 in, direction out
        upd(col_warp_smem_mixed(n0, 2, 8, 2, tsize));  // exact E (FCH)
    } else {
        const size_t p = (size_t)(nf + 2);
        auto rowf = [&](int kin, int szin, int kout, int szout) {
            return 2 * p * ((size_t)kin * 2 * szin + (size_t)kout * 2 * szout);
        };
        auto colf = [&](int k, int sz) { return 2 * p * (size_t)k * 2 * sz; };
        upd(rowf(0, 8, 3, 8));
        upd(rowf(1, 8, 2, 8));
        upd(rowf(ki, 8, ki, tsize));
        upd(rowf(ki, tsize, ki, tsize));
        upd(colf(3, 8));
        upd(colf(2, 8));
        upd(colf(ki, tsize));
    }
    return (m + 15) & ~(size_t)15;
}

// twiddle tables in shared memory: 1 << logtw entries, FP64 then FP32
__host__ __device__ inline size_t tw_smem_bytes(int logtw) { return ((size_t)1 << logtw) * (16 + 8); }

// the fixed line length used for an n0 x n1 grid (0: runtime-length passes)
inline int fixed_len(int n0, int n1) {
    if (n0 != n1) return 0;
    return (n0 == 64 || n0 == 128 || n0 == 256 || n0 == 512) ? n0 : 0;
}

// ------------------------------------------------------------ batched launches
//
// One persistent launch can advance many independent instances (see
// batch.cuh).  The work of a global phase is laid out on a cost axis: instance
// i covers [G_i, G_i + units_i q_i), q_i the points one unit touches, and warp w
// of the grid takes [C_w, C_{w+1}), C_w = floor(total w / NW).

struct BatchParams {
    Params* PI;  // device array of count instance parameter blocks
    int count, logtw;
    Scal* sc;    // barrier state of the launch
    // nullable: one (mask of the phases run, globaltimer) record per global
    // phase, the count in *ntrace
    unsigned long long* trace;
    int trace_cap;
    int* ntrace;
    const double2* tw64;
    const float2* tw32;
};

// work units of a phase and the points one unit touches: column lines, middle
// groups, or row pairs (also for the pointwise phases)
__host__ __device__ inline int phase_units(const Params& P, int ph) {
    return phase_is_col(ph) ? P.ncols : phase_is_mid(ph) ? mid_units(P) : P.rows / 2;
}
__host__ __device__ inline int unit_cost(const Params& P, int ph) {
    return phase_is_col(ph) ? P.n0 : phase_is_mid(ph) ? kMidG * P.nm : 2 * P.n1;
}
// Device time per point of a member's current phase, in units of a PFC FP32
// iteration pass, measured on GB300 with pure phases of batched launches.
// PFC (96 members): exact base row / column passes 8.8x / 7.8x, incremental
// ones ~2/3 of that, the last step's accept 5x.  FCH (8 members of 512^2): its
// iteration passes carry two fields, about 2x a PFC pass per point; relative
// to them, exact base passes 4.5-5x, incremental B / C / D / E
// 4.0 / 2.3 / 1.7 / 3.2x, accept 1.5x.  The batched
// launch lays members out on a cost axis of points x this weight, so that a
// global phase mixing members in FP64 base evaluations with members in FP32
// iterations gives every warp about the same time of work.  Only the dealing
// of units to warps depends on it.
__host__ __device__ inline int phase_weight(const Params& P, const Ctl& c) {
    const bool t64 = P.precision != P_MIXED;
    if (P.model == M_FCH && !t64) {
        switch (c.ph) {
            case PH_B: return c.inc ? 8 : 10;
            case PH_C: return c.inc ? 5 : 10;
            case PH_D: return c.inc ? 3 : 10;
            case PH_E: return c.inc ? 6 : 10;
            case PH_R1:
            case PH_RI:
            case PH_CI: return 2;
            case PH_MF:
            case PH_MI: return c.m64 ? 3 * (c.mk > 0 ? c.mk : 1) : 2;
            case PH_ACCEPT: return 3;
            default: return 4;
        }
    }
    switch (c.ph) {
        case PH_B: return c.inc ? 6 : 9;
        case PH_C:
        case PH_D:
        case PH_E: return c.inc ? 5 : 8;
        case PH_R1:
        case PH_RI:
        case PH_CI: return t64 ? 3 : 1;
        case PH_MF:
        case PH_MI: return (c.m64 || t64) ? 3 * (c.mk > 0 ? c.mk : 1) : 1;
        case PH_ACCEPT: return 5;
        default: return t64 ? 4 : 2;
    }
}
__host__ __device__ inline long long weighted_unit_cost(const Params& P, const Ctl& c) {
    return (long long)unit_cost(P, c.ph) * phase_weight(P, c);
}

// the fixed line lengths compiled into the batched kernel (others: runtime length)
__host__ __device__ inline int batch_nf(int n0, int n1) {
    if (n0 != n1) return 0;
    return (n0 == 128 || n0 == 256 || n0 == 512) ? n0 : 0;
}

// warp owning cost position x (C_w <= x < C_{w+1})
__host__ __device__ inline long long cost_owner(long long x, long long total, long long nw) {
    return ((x + 1) * nw - 1) / total;
}
__host__ __device__ inline long long cost_start(long long w, long long total, long long nw) {
    return (total * w) / nw;
}

constexpr int kIdleRank = 1 << 28;  // rank * 32 exceeds any point count (< 2^32)

// Tw of warp gw for instance i whose work is [g, g + cost) on the cost axis.
__host__ __device__ inline void batch_split(Tw& t, long long gw, long long nw, long long total, long long g,
                                            long long cost, int units, int q) {
    // Members spread over many warps with very many units each (3D grids):
    // their units are dealt round robin over the warps whose slice starts
    // inside the member ([ra, rb]; every warp is in at most one such group), as
    // in a single-instance launch, so that neighbouring units (which share
    // 32-byte sectors of the half spectra) run at the same time instead of one
    // after the other on one warp.  Members with a share of a few warps keep
    // contiguous ranges (measured better for 2D members up to 512^2; a member
    // smaller than one warp's share would otherwise land on one warp on top of
    // that warp's own slice).
    const long long ra = (g * nw + total - 1) / total, rb = ((g + cost) * nw + total - 1) / total - 1;
    if (rb - ra + 1 >= 16 && (long long)units >= 32 * (rb - ra + 1)) {
        if (gw < ra || gw > rb) {
            t.wr = kIdleRank;
            t.wn = 1;
            t.ulo = 0;
            t.uhi = 0;
            return;
        }
        t.wr = (int)(gw - ra);
        t.wn = (int)(rb - ra + 1);
        t.ulo = 0;
        t.uhi = -1;
        return;
    }
    const long long wa = cost_owner(g, total, nw), wb = cost_owner(g + cost - 1, total, nw);
    if (gw < wa || gw > wb) {
        // a warp of a CTA that works on the instance but owns none of it: it
        // joins the CTA's barriers and reductions only.  Its thread rank is
        // past every point and slot index and its stride is nonzero, so every
        // strided loop is empty; it is not the leader; its unit range is empty.
        t.wr = kIdleRank;
        t.wn = 1;
        t.ulo = 0;
        t.uhi = 0;
        return;
    }
    t.wr = (int)(gw - wa);
    t.wn = (int)(wb - wa + 1);
    const long long c0 = cost_start(gw, total, nw) - g, c1 = cost_start(gw + 1, total, nw) - g;
    long long lo = c0 <= 0 ? 0 : (c0 + q - 1) / q;
    long long hi = c1 <= 0 ? 0 : (c1 + q - 1) / q;
    if (lo > units) lo = units;
    if (hi > units) hi = units;
    t.ulo = (int)lo;
    t.uhi = (int)hi;
}

// shared memory of the batched kernel besides the twiddles and the warp slices
__host__ __device__ inline size_t batch_ctl_bytes(int count) {
    const size_t c = (size_t)count * sizeof(Ctl) + (size_t)(count + 1) * sizeof(long long);
    return (c + 15) & ~(size_t)15;
}

}  // namespace pagd
