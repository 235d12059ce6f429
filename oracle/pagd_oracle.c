/*
 * pagd_oracle.c -- plain, slow, FP64 CPU oracle for the PAGD time step of
 * Park, Salgado & Wise, "Benchmark computations of the phase field crystal and
 * functionalized Cahn-Hilliard equations via fully implicit, Nesterov
 * accelerated schemes" (arXiv 2204.07247).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, import or
 * call this file: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes, each function citing the passage it follows:
 *   - its own iterative radix-2 complex FFT (powers of two) and a brute-force
 *     DFT used only to pin the FFT (Sec. 3.2, the DFT and Eq. def:frac-Lap);
 *   - the PFC and FCH chemical potentials and discrete energies (Sec. 2.1
 *     Eq. obj:PFC-egy / eqn:PFCsystem; Sec. 2.2 Eq. obj:FCHegy / eqn:FCHsystem);
 *   - the fully implicit schemes BDF2 (backward Euler first step) and MP
 *     (Sec. 3.1.1, Eqs. eqn:FCH-semidis-implicit, obj:BDF2, obj:MP);
 *   - the objective G_N and its projected gradient (Sec. 3.4, Proposition,
 *     Eqs. obj:FCH-mini-objv, misc07, obj:G');
 *   - the averaged Newton preconditioner (Sec. 3.4.1);
 *   - PGD and PAGD with sweeping friction (Algorithms 1 and 2);
 *   - the linear IMEX schemes LBDF2 / LMP (Eq. eqn:FCH-semidis-simplicit and
 *     Sec. 3.3).
 *
 * Conventions (readings of the paper where it leaves a choice open):
 *   - grid: n[0] x ... x n[dim-1] points, index n[dim-1] fastest, spacing
 *     h_d = L_d / n_d (the paper's "h = 1/N" is read as L/N);
 *   - DFT unnormalised forward (sign -1), inverse sign +1 divided by n_pts;
 *   - wavenumber k_d = 2 pi r_d / L_d with r_d = i_d for i_d <= n_d/2 and
 *     i_d - n_d otherwise; kappa = |k|^2 (even multipliers only, so the
 *     Nyquist sign does not matter);
 *   - the loop of Algorithms 1/2 stops after the first iteration whose
 *     search direction satisfies ||d_i||_inf <= tol;
 *   - for MP the preconditioner's energy terms carry the factor 1/2 of the
 *     second variation of 2 E((v+u^n)/2) unless theta_mode = 1 (literal form).
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PFC 0
#define ORC_FCH 1
#define ORC_BDF2 0
#define ORC_MP 1
#define ORC_LBDF2 2
#define ORC_LMP 3

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOCONV 4
#define ORC_EPRECOND 5
#define ORC_ENAN 6

typedef double complex cplx;

typedef struct {
    int model;      /* ORC_PFC or ORC_FCH */
    int dim;        /* 2 or 3 */
    int n[3];       /* points per axis, powers of two, n[dim-1] fastest */
    double L[3];    /* domain lengths */
    double eps;     /* PFC epsilon / FCH interface thickness epsilon */
    double eta1, eta2, tau; /* FCH material parameters and well asymmetry */
    double M;       /* mobility */
    int scheme;     /* ORC_BDF2 .. ORC_LMP */
    double s;       /* PAGD / PGD step size */
    int n_eta;      /* length of the sweeping friction list */
    double eta[16]; /* sweeping friction list */
    int max_iter;   /* iteration cap */
    int theta_mode; /* 0: exact second variation for MP (factor 1/2), 1: literal */
    int accel;      /* 1: PAGD (Algorithm 2), 0: PGD (Algorithm 1) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static long npts(const orc_params *p) {
    long t = 1;
    for (int d = 0; d < p->dim; d++) t *= p->n[d];
    return t;
}

static double cellvol(const orc_params *p) {
    double h = 1.0;
    for (int d = 0; d < p->dim; d++) h *= p->L[d] / p->n[d];
    return h;
}

/* kappa = |k|^2 at linear spectral index idx (same layout as the grid) */
static double kappa_at(const orc_params *p, long idx) {
    double kap = 0.0;
    for (int d = p->dim - 1; d >= 0; d--) {
        int i = (int)(idx % p->n[d]);
        idx /= p->n[d];
        int r = (i <= p->n[d] / 2) ? i : i - p->n[d];
        double k = 2.0 * 3.14159265358979323846 * (double)r / p->L[d];
        kap += k * k;
    }
    return kap;
}

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 on one line, then axis by axis (Sec. 3.2)          */
/* ------------------------------------------------------------------------ */

static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

/* in-place complex DFT of length n (power of two), sign -1 forward, +1 inverse,
 * unnormalised.  Twiddles exp(sign 2 pi i m / n) from long double libm. */
static void fft_line(cplx *a, int n, int sign) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)(n / 2 > 0 ? n / 2 : 1));
    for (int m = 0; m < n / 2; m++) {
        long double ang = (long double)sign * 2.0L * 3.141592653589793238462643383279502884L *
                          (long double)m / (long double)n;
        w[m] = (double)cosl(ang) + I * (double)sinl(ang);
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int st = 0; st < n; st += len) {
            for (int k = 0; k < half; k++) {
                cplx u = a[st + k];
                cplx v = a[st + k + half] * w[k * step];
                a[st + k] = u + v;
                a[st + k + half] = u - v;
            }
        }
    }
    free(w);
}

/* multi-dimensional complex FFT over a row-major grid, in place, unnormalised */
/* Threads for the line transforms of fft_nd (default 1; OpenMP builds only).
 * The lines of one axis are independent and each is transformed exactly as
 * with one thread, so no result depends on the count. */
static int orc_nthreads = 1;

int orc_set_threads(int t) {
    orc_nthreads = t < 1 ? 1 : t;
    return ORC_OK;
}

static int fft_nd(int dim, const int *n, cplx *a, int sign) {
    long tot = 1;
    int maxn = 1;
    for (int d = 0; d < dim; d++) {
        if (!is_pow2(n[d])) return ORC_EINVAL;
        tot *= n[d];
        if (n[d] > maxn) maxn = n[d];
    }
    for (int d = 0; d < dim; d++) {
        long stride = 1;
        for (int e = d + 1; e < dim; e++) stride *= n[e];
        long nlines = tot / n[d];
#ifdef _OPENMP
#pragma omp parallel num_threads(orc_nthreads) if (orc_nthreads > 1)
#endif
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)maxn);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (long l = 0; l < nlines; l++) {
                long inner = l % stride, outer = l / stride;
                long base = outer * stride * n[d] + inner;
                for (int i = 0; i < n[d]; i++) line[i] = a[base + (long)i * stride];
                fft_line(line, n[d], sign);
                for (int i = 0; i < n[d]; i++) a[base + (long)i * stride] = line[i];
            }
            free(line);
        }
    }
    return ORC_OK;
}

/* Exported for the FFT pins: interleaved (re, im) doubles, in place. */
int orc_fft(int dim, const int *n, double *data, int sign) {
    return fft_nd(dim, n, (cplx *)data, sign);
}

/* Brute-force DFT, O(n_pts^2): out(k) = sum_m in(m) exp(sign 2 pi i k.m / n). */
int orc_dft_brute(int dim, const int *n, const double *in, double *out, int sign) {
    long tot = 1;
    for (int d = 0; d < dim; d++) tot *= n[d];
    const cplx *x = (const cplx *)in;
    cplx *y = (cplx *)out;
    int ki[3], mi[3];
    for (long k = 0; k < tot; k++) {
        long t = k;
        for (int d = dim - 1; d >= 0; d--) { ki[d] = (int)(t % n[d]); t /= n[d]; }
        cplx acc = 0.0;
        for (long m = 0; m < tot; m++) {
            long u = m;
            for (int d = dim - 1; d >= 0; d--) { mi[d] = (int)(u % n[d]); u /= n[d]; }
            long double ph = 0.0L;
            for (int d = 0; d < dim; d++)
                ph += (long double)((long)ki[d] * mi[d] % n[d]) / (long double)n[d];
            ph *= (long double)sign * 2.0L * 3.141592653589793238462643383279502884L;
            acc += x[m] * ((double)cosl(ph) + I * (double)sinl(ph));
        }
        y[k] = acc;
    }
    return ORC_OK;
}

/* real field -> full complex spectrum */
static void fwd_real(const orc_params *p, const double *u, cplx *uh) {
    long N = npts(p);
    for (long i = 0; i < N; i++) uh[i] = u[i];
    fft_nd(p->dim, p->n, uh, -1);
}

/* full complex spectrum -> real field (real part of the normalised inverse) */
static void inv_real(const orc_params *p, const cplx *uh, double *u) {
    long N = npts(p);
    cplx *t = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    memcpy(t, uh, sizeof(cplx) * (size_t)N);
    fft_nd(p->dim, p->n, t, +1);
    for (long i = 0; i < N; i++) u[i] = creal(t[i]) / (double)N;
    free(t);
}

/* (-Delta_N)^alpha w for alpha in {-1, 1, 2} (Eq. def:frac-Lap); for alpha=-1
 * the zero mode is left out of the sum. */
int orc_frac_lap(const orc_params *p, const double *w, double *out, int alpha) {
    long N = npts(p);
    cplx *wh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    fwd_real(p, w, wh);
    for (long k = 0; k < N; k++) {
        double kap = kappa_at(p, k);
        double m;
        if (alpha == -1) m = (k == 0) ? 0.0 : 1.0 / kap;
        else if (alpha == 1) m = kap;
        else if (alpha == 2) m = kap * kap;
        else { free(wh); return ORC_EINVAL; }
        wh[k] *= m;
    }
    inv_real(p, wh, out);
    free(wh);
    return ORC_OK;
}

/* Delta_N w = -(-Delta_N) w */
static void lap(const orc_params *p, const double *w, double *out) {
    orc_frac_lap(p, w, out, 1);
    long N = npts(p);
    for (long i = 0; i < N; i++) out[i] = -out[i];
}

/* discrete inner product (u, v)_N = h^d sum u v (trapezoid, Sec. 3.2) */
static double ip(const orc_params *p, const double *u, const double *v) {
    long N = npts(p);
    long double acc = 0.0L;
    for (long i = 0; i < N; i++) acc += (long double)u[i] * v[i];
    return (double)acc * cellvol(p);
}

static double mean(const orc_params *p, const double *u) {
    long N = npts(p);
    long double acc = 0.0L;
    for (long i = 0; i < N; i++) acc += u[i];
    return (double)(acc / (long double)N);
}

/* Pi_0: mean-zero projection (Remark on discrete mass conservation, Sec. 3.4) */
static void pi0(const orc_params *p, double *u) {
    long N = npts(p);
    double m = mean(p, u);
    for (long i = 0; i < N; i++) u[i] -= m;
}

/* mass (u, 1)_N */
double orc_mass(const orc_params *p, const double *u) {
    long N = npts(p);
    long double acc = 0.0L;
    for (long i = 0; i < N; i++) acc += u[i];
    return (double)acc * cellvol(p);
}

/* ------------------------------------------------------------------------ */
/* models (Sec. 2)                                                           */
/* ------------------------------------------------------------------------ */

/* double well F(z) = 1/2 (z+1)^2 (1/2 (z-1)^2 + 2/3 tau (z-2))  (Sec. 2.2),
 * and its derivatives by the product rule with g = 1/2 (z-1)^2 + 2/3 tau (z-2). */
static double Fw(double z, double tau) {
    double g = 0.5 * (z - 1) * (z - 1) + (2.0 / 3.0) * tau * (z - 2);
    return 0.5 * (z + 1) * (z + 1) * g;
}
static double Fw1(double z, double tau) {
    double g = 0.5 * (z - 1) * (z - 1) + (2.0 / 3.0) * tau * (z - 2);
    double g1 = (z - 1) + (2.0 / 3.0) * tau;
    return (z + 1) * g + 0.5 * (z + 1) * (z + 1) * g1;
}
static double Fw2(double z, double tau) {
    double g = 0.5 * (z - 1) * (z - 1) + (2.0 / 3.0) * tau * (z - 2);
    double g1 = (z - 1) + (2.0 / 3.0) * tau;
    return g + 2.0 * (z + 1) * g1 + 0.5 * (z + 1) * (z + 1);
}
static double Fw3(double z, double tau) {
    double g1 = (z - 1) + (2.0 / 3.0) * tau;
    return 3.0 * g1 + 3.0 * (z + 1);
}

/* chemical potential mu = dE/du.
 * PFC (eqn:PFCsystem): mu = u^3 + (1-eps) u + 2 Lap u + Lap^2 u.
 * FCH (eqn:FCHsystem, read with omega = eps^2 Lap u - F'(u) and the product as
 * the operator (eps^2 Lap - F''(u) + eta1) applied to omega):
 *   mu = eps^2 Lap omega - (F''(u) - eta1) omega + (eta1 - eta2) F'(u). */
int orc_mu(const orc_params *p, const double *u, double *mu) {
    long N = npts(p);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)N);
    if (p->model == ORC_PFC) {
        lap(p, u, t1);      /* Lap u */
        lap(p, t1, t2);     /* Lap^2 u */
        for (long i = 0; i < N; i++)
            mu[i] = u[i] * u[i] * u[i] + (1.0 - p->eps) * u[i] + 2.0 * t1[i] + t2[i];
    } else {
        double e2 = p->eps * p->eps;
        lap(p, u, t1);                                   /* Lap u */
        for (long i = 0; i < N; i++) t1[i] = e2 * t1[i] - Fw1(u[i], p->tau); /* omega */
        lap(p, t1, t2);                                  /* Lap omega */
        for (long i = 0; i < N; i++)
            mu[i] = e2 * t2[i] - (Fw2(u[i], p->tau) - p->eta1) * t1[i] +
                    (p->eta1 - p->eta2) * Fw1(u[i], p->tau);
    }
    free(t1);
    free(t2);
    return ORC_OK;
}

/* discrete energy E_N: the integrand with Fourier differentiation and the
 * trapezoidal rule; |grad u|^2 enters as (-Lap_N u, u)_N. */
int orc_energy(const orc_params *p, const double *u, double *E) {
    long N = npts(p);
    double *lu = (double *)malloc(sizeof(double) * (size_t)N);
    double *nl = (double *)malloc(sizeof(double) * (size_t)N);
    double *f = (double *)malloc(sizeof(double) * (size_t)N);
    lap(p, u, lu);
    for (long i = 0; i < N; i++) nl[i] = -lu[i];
    double grad2 = ip(p, nl, u); /* (grad u, grad u)_N */
    if (p->model == ORC_PFC) {
        /* obj:PFC-egy */
        for (long i = 0; i < N; i++)
            f[i] = 0.25 * u[i] * u[i] * u[i] * u[i] + 0.5 * (1.0 - p->eps) * u[i] * u[i] +
                   0.5 * lu[i] * lu[i];
        long double acc = 0.0L;
        for (long i = 0; i < N; i++) acc += f[i];
        *E = (double)acc * cellvol(p) - grad2;
    } else {
        /* obj:FCHegy */
        double e2 = p->eps * p->eps;
        for (long i = 0; i < N; i++) {
            double w = e2 * lu[i] - Fw1(u[i], p->tau);
            f[i] = 0.5 * w * w - p->eta2 * Fw(u[i], p->tau);
        }
        long double acc = 0.0L;
        for (long i = 0; i < N; i++) acc += f[i];
        *E = (double)acc * cellvol(p) - 0.5 * e2 * p->eta1 * grad2;
    }
    free(lu);
    free(nl);
    free(f);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* schemes (Sec. 3.1.1)                                                      */
/* ------------------------------------------------------------------------ */

/* coefficients a_n, b_n, c_n (obj:BDF2 / obj:MP; backward Euler for the first
 * BDF2 / LBDF2 step, Algorithm 3 caption).  step = n, dt = dt_{n+1},
 * dt_prev = dt_n. */
int orc_coeffs(int scheme, int step, double dt, double dt_prev, double *abc) {
    if (scheme == ORC_BDF2 || scheme == ORC_LBDF2) {
        if (step == 0) {
            abc[0] = 1.0 / dt; abc[1] = -1.0 / dt; abc[2] = 0.0;
        } else {
            abc[0] = 1.0 / dt + 1.0 / (dt + dt_prev);
            abc[1] = -1.0 / dt - 1.0 / dt_prev;
            abc[2] = 1.0 / dt_prev - 1.0 / (dt + dt_prev);
        }
    } else if (scheme == ORC_MP || scheme == ORC_LMP) {
        abc[0] = 1.0 / dt; abc[1] = -1.0 / dt; abc[2] = 0.0;
    } else {
        return ORC_EINVAL;
    }
    return ORC_OK;
}

/* the scheme argument breve v (BDF2: v; MP: (v + u^n)/2) */
static void breve(const orc_params *p, const double *v, const double *un, double *out) {
    long N = npts(p);
    if (p->scheme == ORC_MP)
        for (long i = 0; i < N; i++) out[i] = 0.5 * (v[i] + un[i]);
    else
        for (long i = 0; i < N; i++) out[i] = v[i];
}

/* objective G_N(v) of the Proposition (obj:FCH-mini-objv):
 *   1/(2 M a) ||a v + b u^n + c u^{n-1}||_{-1,N}^2 + Etilde_N(breve v),
 * Etilde = E_N(v) for BDF2 and 2 E_N((v+u^n)/2) for MP. */
int orc_objective(const orc_params *p, const double *abc, const double *un, const double *unm1,
                  const double *v, double *G) {
    long N = npts(p);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *iw = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; i++) w[i] = abc[0] * v[i] + abc[1] * un[i] + abc[2] * unm1[i];
    orc_frac_lap(p, w, iw, -1);
    double nrm2 = ip(p, iw, w); /* Eq. def:neg-norm */
    breve(p, v, un, w);
    double E;
    orc_energy(p, w, &E);
    if (p->scheme == ORC_MP) E *= 2.0;
    *G = nrm2 / (2.0 * p->M * abc[0]) + E;
    free(w);
    free(iw);
    return ORC_OK;
}

/* projected gradient G'_N(v) (obj:G'):
 *   1/M (-Lap)^{-1} Pi0 (a v + b u^n + c u^{n-1}) + Pi0 mu(breve v).
 * (For MP, Etilde = 2 E((v+u^n)/2) and the chain rule gives exactly mu(breve v).) */
int orc_gradient(const orc_params *p, const double *abc, const double *un, const double *unm1,
                 const double *v, double *g) {
    long N = npts(p);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *t = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; i++) w[i] = abc[0] * v[i] + abc[1] * un[i] + abc[2] * unm1[i];
    pi0(p, w);
    orc_frac_lap(p, w, t, -1);
    breve(p, v, un, w);
    double *mu = (double *)malloc(sizeof(double) * (size_t)N);
    orc_mu(p, w, mu);
    pi0(p, mu);
    for (long i = 0; i < N; i++) g[i] = t[i] / p->M + mu[i];
    free(w);
    free(t);
    free(mu);
    return ORC_OK;
}

/* averaged Newton preconditioner constants (Sec. 3.4.1), evaluated at the
 * scheme argument of the initial guess vb0.  out = {beta_-2, beta_0, beta_2,
 * beta_4}.
 *   PFC G'' = a/M (-Lap)^-1 + (3u^2 + 1 - eps) - 2 (-Lap) + Lap^2: beta_0 is the
 *     absolute grid average of 3 vb0^2 + 1 - eps; beta_2 = -2 and beta_4 = 1 are
 *     constants and kept with their values.
 *   FCH: beta_0 = |avg(F''^2 - eta2 F'' + F''' F')| (the eps^2-Laplacian terms
 *     dropped as stated), beta_2 = |avg(eps^2 (F'' - eta1))|, beta_4 = eps^4.
 *   For MP the energy part is scaled by 1/2 (the second variation of
 *   2 E((v+u^n)/2)) unless theta_mode = 1. */
int orc_betas(const orc_params *p, double a, const double *vb0, double *beta) {
    long N = npts(p);
    double th = (p->scheme == ORC_MP && p->theta_mode == 0) ? 0.5 : 1.0;
    beta[0] = a / p->M;
    if (p->model == ORC_PFC) {
        long double acc = 0.0L;
        for (long i = 0; i < N; i++) acc += 3.0 * vb0[i] * vb0[i] + 1.0 - p->eps;
        beta[1] = th * fabs((double)(acc / (long double)N));
        beta[2] = -2.0 * th;
        beta[3] = th;
    } else {
        double e2 = p->eps * p->eps;
        long double a0 = 0.0L, a2 = 0.0L;
        for (long i = 0; i < N; i++) {
            double f1 = Fw1(vb0[i], p->tau), f2 = Fw2(vb0[i], p->tau), f3 = Fw3(vb0[i], p->tau);
            a0 += f2 * f2 - p->eta2 * f2 + f3 * f1;
            a2 += e2 * (f2 - p->eta1);
        }
        beta[1] = th * fabs((double)(a0 / (long double)N));
        beta[2] = th * fabs((double)(a2 / (long double)N));
        beta[3] = th * e2 * e2;
    }
    return ORC_OK;
}

/* d = Lcal^{-1} r, Lcal = beta_-2 (-Lap)^-1 + beta_0 + beta_2 (-Lap) + beta_4 Lap^2,
 * applied per wavenumber; the zero mode of d is zero.  Returns EPRECOND if the
 * symbol is not positive on some nonzero wavenumber. */
static int precond_solve(const orc_params *p, const double *beta, const double *r, double *d) {
    long N = npts(p);
    cplx *rh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    fwd_real(p, r, rh);
    int st = ORC_OK;
    for (long k = 0; k < N; k++) {
        if (k == 0) { rh[k] = 0.0; continue; }
        double kap = kappa_at(p, k);
        double Lk = beta[0] / kap + beta[1] + beta[2] * kap + beta[3] * kap * kap;
        if (!(Lk > 0.0)) st = ORC_EPRECOND;
        rh[k] /= Lk;
    }
    inv_real(p, rh, d);
    free(rh);
    return st;
}

/* One fully implicit step (Algorithm 3 body at a fixed step size) solved with
 * PAGD (Algorithm 2) or PGD (Algorithm 1).
 *   step = n (0 for the first step), un = u^n, unm1 = u^{n-1} (u^{-1} := u^0),
 *   dt = dt_{n+1}, dt_prev = dt_n, guess = optional initial iterate (its mean is
 *   replaced by that of u^n), otherwise the extrapolation of the previous two
 *   solutions (Sec. 3.4.2).  Writes u^{n+1}, the iteration count and, if hist
 *   is not NULL, ||d_i||_inf for every iteration taken. */
int orc_pagd_step(const orc_params *p, int step, const double *un, const double *unm1, double dt,
                  double dt_prev, double tol, const double *guess, double *unp1, int *iters,
                  double *hist, double *beta_out) {
    long N = npts(p);
    if (p->scheme != ORC_BDF2 && p->scheme != ORC_MP) return ORC_EINVAL;
    double abc[3];
    orc_coeffs(p->scheme, step, dt, dt_prev, abc);
    double *x = (double *)malloc(sizeof(double) * (size_t)N);
    double *xp = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)malloc(sizeof(double) * (size_t)N);
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    /* initial guess */
    if (guess) {
        double shift = mean(p, un) - mean(p, guess);
        for (long i = 0; i < N; i++) x[i] = guess[i] + shift;
    } else {
        double rho = (step == 0) ? 0.0 : dt / dt_prev;
        for (long i = 0; i < N; i++) x[i] = un[i] + rho * (un[i] - unm1[i]);
    }
    memcpy(xp, x, sizeof(double) * (size_t)N); /* x_{-1} := x_0 */
    /* preconditioner from the initial guess */
    double beta[4];
    breve(p, x, un, y);
    orc_betas(p, abc[0], y, beta);
    if (beta_out) memcpy(beta_out, beta, sizeof(beta));
    int st = ORC_ENOCONV;
    int it = 0;
    double sq = sqrt(p->s);
    for (int i = 0; i < p->max_iter; i++) {
        double lam = 0.0;
        if (p->accel) {
            double eta = p->eta[i % p->n_eta];
            lam = (1.0 - eta * sq) / (1.0 + eta * sq);
        }
        for (long q = 0; q < N; q++) y[q] = x[q] + lam * (x[q] - xp[q]);
        orc_gradient(p, abc, un, unm1, y, r);
        for (long q = 0; q < N; q++) r[q] = -r[q];
        int pst = precond_solve(p, beta, r, d);
        if (pst != ORC_OK) { st = pst; it = i; break; }
        double dn = 0.0;
        for (long q = 0; q < N; q++) {
            xp[q] = x[q];
            x[q] = y[q] + p->s * d[q];
            double ad = fabs(d[q]);
            if (ad > dn || ad != ad) dn = ad;
        }
        if (hist) hist[i] = dn;
        it = i + 1;
        if (!(dn == dn) || isinf(dn)) { st = ORC_ENAN; break; }
        if (dn <= tol) { st = ORC_OK; break; }
    }
    memcpy(unp1, x, sizeof(double) * (size_t)N);
    *iters = it;
    free(x); free(xp); free(y); free(r); free(d);
    return st;
}

/* Linear IMEX step (eqn:FCH-semidis-simplicit, Sec. 3.3): mu = L(u) + N(u) with
 *   PFC: L = (1 + Lap)^2, N = u^3 - eps u;
 *   FCH: L = eps^4 Lap^2 + kappa2 (-Lap) + kappa0, kappa0 = 1 - 2 tau^2 + eta2,
 *        kappa2 = 1, N = -kappa0 u - eps^2 Lap F'(u) - (eps^2 (F'' - eta1) - kappa2) Lap u
 *                        + (F'' - eta2) F'.
 * LBDF2: Lbar = u^{n+1}, breve u = u^n + rho (u^n - u^{n-1});
 * LMP:   Lbar = (u^n + u^{n+1})/2, breve u = ((2 + rho) u^n - rho u^{n-1}) / 2.
 * The linear system is diagonal in Fourier space and solved per wavenumber. */
int orc_imex_step(const orc_params *p, int step, const double *un, const double *unm1, double dt,
                  double dt_prev, double *unp1) {
    long N = npts(p);
    if (p->scheme != ORC_LBDF2 && p->scheme != ORC_LMP) return ORC_EINVAL;
    double abc[3];
    orc_coeffs(p->scheme, step, dt, dt_prev, abc);
    double rho = (step == 0) ? 0.0 : dt / dt_prev;
    double *ub = (double *)malloc(sizeof(double) * (size_t)N);
    double *nl = (double *)malloc(sizeof(double) * (size_t)N);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)N);
    if (p->scheme == ORC_LBDF2)
        for (long i = 0; i < N; i++) ub[i] = un[i] + rho * (un[i] - unm1[i]);
    else
        for (long i = 0; i < N; i++) ub[i] = 0.5 * ((2.0 + rho) * un[i] - rho * unm1[i]);
    double kap0 = 1.0 - 2.0 * p->tau * p->tau + p->eta2, kap2 = 1.0;
    if (p->model == ORC_PFC) {
        for (long i = 0; i < N; i++) nl[i] = ub[i] * ub[i] * ub[i] - p->eps * ub[i];
    } else {
        double e2 = p->eps * p->eps;
        for (long i = 0; i < N; i++) t1[i] = Fw1(ub[i], p->tau);
        lap(p, t1, t2);  /* Lap F'(u) */
        lap(p, ub, t1);  /* Lap u */
        for (long i = 0; i < N; i++) {
            double f1 = Fw1(ub[i], p->tau), f2 = Fw2(ub[i], p->tau);
            nl[i] = -kap0 * ub[i] - e2 * t2[i] - (e2 * (f2 - p->eta1) - kap2) * t1[i] +
                    (f2 - p->eta2) * f1;
        }
    }
    cplx *nh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *unh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *umh = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    fwd_real(p, nl, nh);
    fwd_real(p, un, unh);
    fwd_real(p, unm1, umh);
    double half = (p->scheme == ORC_LMP) ? 0.5 : 1.0;
    for (long k = 0; k < N; k++) {
        double kap = kappa_at(p, k);
        double Lh;
        if (p->model == ORC_PFC) Lh = (1.0 - kap) * (1.0 - kap);
        else Lh = p->eps * p->eps * p->eps * p->eps * kap * kap + kap2 * kap + kap0;
        /* a u^{n+1} + b u^n + c u^{n-1} = M Lap (L(ubar) + N(breve u)), Lap -> -kappa */
        cplx rhs = -abc[1] * unh[k] - abc[2] * umh[k] - p->M * kap * nh[k];
        if (p->scheme == ORC_LMP) rhs -= p->M * kap * 0.5 * Lh * unh[k];
        nh[k] = rhs / (abc[0] + p->M * kap * half * Lh);
    }
    inv_real(p, nh, unp1);
    free(ub); free(nl); free(t1); free(t2); free(nh); free(unh); free(umh);
    return ORC_OK;
}

/* Residual of the discrete scheme (eqn:FCH-fulldis-implicit) at a candidate
 * u^{n+1}: a u + b u^n + c u^{n-1} - M Lap_N mu(breve u).  Used by the tests
 * to check a converged step by a route other than the solver's own. */
int orc_scheme_residual(const orc_params *p, int step, const double *un, const double *unm1,
                        double dt, double dt_prev, const double *u, double *res) {
    long N = npts(p);
    double abc[3];
    orc_coeffs(p->scheme, step, dt, dt_prev, abc);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *mu = (double *)malloc(sizeof(double) * (size_t)N);
    double *lm = (double *)malloc(sizeof(double) * (size_t)N);
    breve(p, u, un, w);
    orc_mu(p, w, mu);
    lap(p, mu, lm);
    for (long i = 0; i < N; i++)
        res[i] = abc[0] * u[i] + abc[1] * un[i] + abc[2] * unm1[i] - p->M * lm[i];
    free(w); free(mu); free(lm);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* adaptive time stepping (Sec. 3.1.2, Algorithm 3)                          */
/* ------------------------------------------------------------------------ */

/* R(v) = M Lap_N (delta E / delta u)(v), the right-hand side of the gradient
 * flow (Eqs. eqn:PFCsystem / eqn:FCHPDE) that the AM3 estimator samples. */
int orc_rhs(const orc_params *p, const double *v, double *out) {
    long N = npts(p);
    double *mu = (double *)malloc(sizeof(double) * (size_t)N);
    orc_mu(p, v, mu);
    lap(p, mu, out);
    for (long i = 0; i < N; i++) out[i] *= p->M;
    free(mu);
    return ORC_OK;
}

static double l2(const orc_params *p, const double *u) { return sqrt(ip(p, u, u)); }

/* AM3 stepping: the explicit variant of the third-order Adams-Moulton formula
 * with the tentative solution ut in place of the implicit value,
 *   uh = un + dt/6 [ (3 + 2 rho)/(1 + rho) R(ut) + (3 + rho) R(un) - rho^2/(1 + rho) R(unm1) ],
 * rho = dt / dt_prev; returns ERR = ||ut - uh|| / ||uh|| (discrete L2) and
 * writes uh. */
double orc_am3_err(const orc_params *p, const double *un, const double *ut, const double *Rt, const double *Rn,
                   const double *Rnm1, double dt, double dt_prev, double *uh) {
    long N = npts(p);
    double rho = dt / dt_prev;
    double ct = (3.0 + 2.0 * rho) / (1.0 + rho), cn = 3.0 + rho, cm = -rho * rho / (1.0 + rho);
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; i++) {
        uh[i] = un[i] + dt / 6.0 * (ct * Rt[i] + cn * Rn[i] + cm * Rnm1[i]);
        d[i] = ut[i] - uh[i];
    }
    double e = l2(p, d) / l2(p, uh);
    free(d);
    return e;
}

/* midAB2 stepping (used with MP): the quadratic extrapolation through
 * (t_{n-2}, t_{n-1}, t_n) evaluated at t_n + dt,
 *   uh = a un - b unm1 + c unm2 with the Lagrange weights of the paper,
 * and ERR = ||ut - uh|| / ||uh|| / (1 - 1 / (24 R_n)),
 * R_n = 1/24 + 1/8 (1 + dtn/dt)(1 + 2 dtn/dt + dtnm1/dt). */
double orc_midab2_err(const orc_params *p, const double *un, const double *unm1, const double *unm2,
                      const double *ut, double dt, double dtn, double dtnm1, double *uh) {
    long N = npts(p);
    double a = (dt + dtn) * (dt + dtn + dtnm1) / (dtn * (dtn + dtnm1));
    double b = dt * (dt + dtn + dtnm1) / (dtn * dtnm1);
    double c = dt * (dt + dtn) / (dtnm1 * (dtn + dtnm1));
    double Rn = 1.0 / 24.0 + 0.125 * (1.0 + dtn / dt) * (1.0 + 2.0 * dtn / dt + dtnm1 / dt);
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; i++) {
        uh[i] = a * un[i] - b * unm1[i] + c * unm2[i];
        d[i] = ut[i] - uh[i];
    }
    double e = l2(p, d) / l2(p, uh) / (1.0 - 1.0 / (24.0 * Rn));
    free(d);
    return e;
}

/* Sizes of the structs for the ctypes side to check its layout against. */
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
