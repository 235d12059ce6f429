// pagd.cu -- C ABI of the PAGD library (include/pagd.h): solver objects,
// workspace layout, launch planning and the persistent cooperative kernel.
//
// Built by nvcc for sm_103a into libpagd.so.  The same file also compiles as
// host C++ with -DPAGD_EMU into a test-only emulation library in which device
// memory is host memory and a "launch" runs the kernel's phases block by block
// on the calling thread.
#include "solver.cuh"
#include "cluster.cuh"
#include "../../include/pagd.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace pagd;

#ifndef PAGD_EMU
namespace pagd {
template <class T, int NF>
cudaError_t pagd_launch(const Params& P, int grid, int threads, size_t smem, void* stream, int* grid_used);
template <class T>
cudaError_t pagd_batch_launch(const BatchParams& B, int grid, int threads, size_t smem, void* stream,
                              int* grid_used);
}
#else
thread_local EmuDim3 threadIdx{0, 0, 0}, blockIdx{0, 0, 0}, blockDim{1, 1, 1}, gridDim{1, 1, 1};
#endif

// ------------------------------------------------------------ solver object

constexpr int kMaxChunk = 4096;
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA on sm_103a
constexpr int kMaxBatch = 4096;
constexpr int kTraceCap = 8192;  // phase records kept per launch when tracing
// FP32-mixed: steps between exact FP64 recomputations of the reference spectra
constexpr int kRefreshSteps = 32;

struct pagd_solver {
    int model, dim, n[3];
    double L[3];
    double eps, eta1, eta2, tau, M;
    int scheme, precision;
    pagd_opts opts;
    void* stream;
    // layout
    long long npts;
    int h1, nslots, tsize;
    size_t off[48];  // workspace offsets, indexed by the O_* enum
    size_t ws_bytes;
    char* ws;
    // launch plan (grid_used: the grid of the last launch)
    int grid, logtw, threads, coop, cl, stage, coop32, grid_used;
    size_t smem, warp_bytes;
    // state
    int have_state, step, cur, trace, ref_valid;
    double dt_prev;
    std::string err;
};

enum {
    O_SC, O_NORMS, O_SUMS, O_STATS, O_TW64, O_TW32, O_U0, O_U1, O_VB, O_G64, O_VBT, O_LBT, O_DD0,
    O_DD1, O_SS0, O_SS1, O_C0, O_NB, O_DB, O_CL64, O_NB64, O_DB64, O_MASS, O_TRACE, O_VR64, O_NR64, O_WR64, O_LB64, O_YB, O_X, O_X64, O_GH64, O_LCTL, O_END
};

static pagd_status fail(pagd_solver* s, pagd_status st, const char* msg) {
    if (s) s->err = msg;
    return st;
}

static bool pow2_ok(int v) { return v >= 8 && v <= 512 && (v & (v - 1)) == 0; }

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// rows of the row passes (all points but the last axis) and the half-spectrum
// size of one field
static long long rows_of(const pagd_solver* s) { return s->npts / s->n[s->dim - 1]; }

static double cell_volume(const pagd_solver* s) {
    double h = 1.0;
    for (int d = 0; d < s->dim; d++) h *= s->L[d] / s->n[d];
    return h;
}

static void plan_layout(pagd_solver* s) {
    const long long N = s->npts;
    const long long H = (long long)s->h1 * rows_of(s);
    const int T = s->tsize;
    size_t sz[O_END];
    sz[O_SC] = sizeof(Scal);
    sz[O_NORMS] = sizeof(unsigned long long) * 2 * s->nslots;
    sz[O_SUMS] = sizeof(double) * 2 * s->nslots;
    sz[O_STATS] = sizeof(StepStat) * kMaxChunk;
    sz[O_TW64] = sizeof(double2) * kNMax;
    sz[O_TW32] = sizeof(float2) * kNMax;
    sz[O_U0] = sz[O_U1] = sz[O_VB] = sz[O_G64] = sizeof(double) * N;
    sz[O_VBT] = sz[O_LBT] = sz[O_DD0] = sz[O_DD1] = (size_t)T * N;
    sz[O_SS0] = sz[O_SS1] = sz[O_C0] = (size_t)2 * T * H;
    sz[O_NB] = (size_t)2 * T * H * 3;
    sz[O_DB] = (size_t)2 * T * H * 2;
    sz[O_CL64] = sizeof(double2) * H * 3;
    sz[O_NB64] = sizeof(double2) * H * 3;
    sz[O_DB64] = sizeof(double2) * H * 2;
    sz[O_MASS] = sizeof(double) * 4;
    sz[O_TRACE] = sizeof(unsigned long long) * 2 * kTraceCap;
    sz[O_VR64] = sizeof(double2) * H;
    sz[O_NR64] = sizeof(double2) * H * 2;
    sz[O_WR64] = sizeof(double2) * H;
    sz[O_LB64] = sizeof(double) * N;
    sz[O_YB] = (size_t)T * N;
    sz[O_X] = s->dim == 3 ? (size_t)2 * T * H * 3 : 0;
    sz[O_X64] = s->dim == 3 ? sizeof(double2) * H * 3 : 0;
    sz[O_GH64] = sizeof(double2) * H;
    sz[O_LCTL] = sizeof(Ctl);
    static_assert(O_END <= (int)(sizeof(((pagd_solver*)nullptr)->off) / sizeof(size_t)), "offset table too small");
    size_t o = 0;
    for (int i = 0; i < O_END; i++) {
        s->off[i] = o;
        o += (sz[i] + 255) & ~(size_t)255;
    }
    s->ws_bytes = o;
}

static Params params_for(const pagd_solver* s, char* w) {
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.model = s->model;
    P.scheme = s->scheme;
    P.precision = s->precision;
    const int last = s->dim - 1;
    P.n0 = s->n[0];
    P.n1 = s->n[last];
    P.nm = s->dim == 3 ? s->n[1] : 1;
    P.logn0 = ilog2(P.n0);
    P.logn1 = ilog2(P.n1);
    P.logm = ilog2(P.nm);
    P.h1 = s->h1;
    P.rows = (int)rows_of(s);
    P.ncols = s->h1 * P.nm;
    P.H = (long long)s->h1 * P.rows;
    P.logtw = s->logtw;
    P.npts = s->npts;
    P.inv_npts = 1.0 / (double)s->npts;
    P.warp_bytes = (long long)s->warp_bytes;
    P.coop = s->coop;
    P.stage = s->stage;
    P.coop32 = s->coop32;
    const double twopi = 6.283185307179586476925286766559;
    P.k0sq = (twopi / s->L[0]) * (twopi / s->L[0]);
    P.k1sq = (twopi / s->L[last]) * (twopi / s->L[last]);
    P.kmsq = s->dim == 3 ? (twopi / s->L[1]) * (twopi / s->L[1]) : 0.0;
    P.cellvol = 1.0;
    for (int d = 0; d < s->dim; d++) P.cellvol *= s->L[d] / s->n[d];
    P.eps = s->eps;
    P.eta1 = s->eta1;
    P.eta2 = s->eta2;
    P.tau = s->tau;
    P.M = s->M;
    P.s = s->opts.s;
    P.n_eta = s->opts.n_eta;
    P.accel = s->opts.accel;
    P.max_iter = s->opts.max_iter;
    P.max_recheck = 16;
    P.theta_mode = s->opts.theta_mode;
    const double sq = std::sqrt(s->opts.s);
    for (int j = 0; j < s->opts.n_eta; j++) P.lam[j] = (1.0 - s->opts.eta[j] * sq) / (1.0 + s->opts.eta[j] * sq);
    P.nslots = s->nslots;
    P.cur0 = s->cur;
    P.step0 = s->step;
    P.sc = (Scal*)(w + s->off[O_SC]);
    P.norms = (unsigned long long*)(w + s->off[O_NORMS]);
    P.sums = (double*)(w + s->off[O_SUMS]);
    P.stats = (StepStat*)(w + s->off[O_STATS]);
    P.tw64 = (const double2*)(w + s->off[O_TW64]);
    P.tw32 = (const float2*)(w + s->off[O_TW32]);
    P.U[0] = (double*)(w + s->off[O_U0]);
    P.U[1] = (double*)(w + s->off[O_U1]);
    P.VB = (double*)(w + s->off[O_VB]);
    P.G64 = (double*)(w + s->off[O_G64]);
    P.VBt = w + s->off[O_VBT];
    P.LBt = w + s->off[O_LBT];
    P.DD[0] = w + s->off[O_DD0];
    P.DD[1] = w + s->off[O_DD1];
    P.SS[0] = w + s->off[O_SS0];
    P.SS[1] = w + s->off[O_SS1];
    P.C0 = w + s->off[O_C0];
    P.NB = w + s->off[O_NB];
    P.DB = w + s->off[O_DB];
    P.CL64 = (double2*)(w + s->off[O_CL64]);
    P.NB64 = (double2*)(w + s->off[O_NB64]);
    P.DB64 = (double2*)(w + s->off[O_DB64]);
    P.mass = (double*)(w + s->off[O_MASS]);
    P.trace = s->trace ? (unsigned long long*)(w + s->off[O_TRACE]) : nullptr;
    P.trace_cap = kTraceCap;
    P.VR64 = (double2*)(w + s->off[O_VR64]);
    P.NR64 = (double2*)(w + s->off[O_NR64]);
    P.WR64 = (double2*)(w + s->off[O_WR64]);
    P.GH64 = (double2*)(w + s->off[O_GH64]);
    P.LB64 = (double*)(w + s->off[O_LB64]);
    P.YB = w + s->off[O_YB];
    P.X = s->dim == 3 ? (void*)(w + s->off[O_X]) : nullptr;
    P.X64 = s->dim == 3 ? (double2*)(w + s->off[O_X64]) : nullptr;
    P.ref_valid = s->ref_valid;
    P.refresh = kRefreshSteps;
    P.cl = s->cl;
    P.lctl = w + s->off[O_LCTL];
    return P;
}

static Params base_params(const pagd_solver* s) { return params_for(s, s->ws); }

// ------------------------------------------------------- device plumbing

#ifdef PAGD_EMU
static pagd_status dcopy(pagd_solver*, void* dst, const void* src, size_t n) {
    std::memmove(dst, src, n);
    return PAGD_OK;
}
static pagd_status dzero(pagd_solver*, void* dst, size_t n) {
    std::memset(dst, 0, n);
    return PAGD_OK;
}
static pagd_status dsync(pagd_solver*) { return PAGD_OK; }
static int num_sms() {
    const char* e = std::getenv("PAGD_EMU_SMS");  // tile plan of an n-SM device
    const int v = e ? std::atoi(e) : 4;
    return v > 0 ? v : 4;
}
template <class T> static pagd_status launch(pagd_solver* s, const Params& P) {
    std::vector<char> sm(s->smem + 64);
    char* base = (char*)(((uintptr_t)sm.data() + 15) & ~(uintptr_t)15);
    double red[32];
    gridDim.x = (unsigned)s->grid;
    blockDim.x = 1;
    threadIdx.x = 0;
    const int ntw = 1 << P.logtw;
    double2* t64 = (double2*)base;
    float2* t32 = (float2*)(base + (size_t)ntw * sizeof(double2));
    for (int m = 0; m < ntw; m++) {
        t64[m] = P.tw64[m * (kNMax >> P.logtw)];
        t32[m] = P.tw32[m * (kNMax >> P.logtw)];
    }
    Tw tw{t64, t32, P.logtw, 0, s->grid, 0, -1};
    char* wsm = base + tw_smem_bytes(P.logtw);
    Ctl c = ctl_init(P);
    const int nf = fixed_len(P.n0, P.n1);
    while (c.ph != PH_DONE) {
        if (P.cl && c.ph == PH_CI) {
            switch (nf) {
                case 64: cluster_iterate_emu<T, 64>(P, c, tw); break;
                case 128: cluster_iterate_emu<T, 128>(P, c, tw); break;
                case 256: cluster_iterate_emu<T, 256>(P, c, tw); break;
                default: break;
            }
            c = *(const Ctl*)P.lctl;  // resume after the loop's last row pass (phase RI)
            ctl_advance<T>(P, c);
            continue;
        }
        for (int b = 0; b < s->grid; b++) {
            blockIdx.x = (unsigned)b;
            tw.wr = b;
            switch (nf) {
                case 64: exec_phase<T, 64>(P, c, tw, wsm, red); break;
                case 128: exec_phase<T, 128>(P, c, tw, wsm, red); break;
                case 256: exec_phase<T, 256>(P, c, tw, wsm, red); break;
                case 512: exec_phase<T, 512>(P, c, tw, wsm, red); break;
                default: exec_phase<T, 0>(P, c, tw, wsm, red); break;
            }
        }
        ctl_advance<T>(P, c);
    }
    s->grid_used = s->grid;
    return PAGD_OK;
}
#else
static pagd_status cuda_fail(pagd_solver* s, cudaError_t e, const char* what) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fail(s, PAGD_ECUDA, buf);
}
static pagd_status dcopy(pagd_solver* s, void* dst, const void* src, size_t n) {
    cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, (cudaStream_t)s->stream);
    return e == cudaSuccess ? PAGD_OK : cuda_fail(s, e, "cudaMemcpyAsync");
}
static pagd_status dzero(pagd_solver* s, void* dst, size_t n) {
    cudaError_t e = cudaMemsetAsync(dst, 0, n, (cudaStream_t)s->stream);
    return e == cudaSuccess ? PAGD_OK : cuda_fail(s, e, "cudaMemsetAsync");
}
static pagd_status dsync(pagd_solver* s) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)s->stream);
    return e == cudaSuccess ? PAGD_OK : cuda_fail(s, e, "cudaStreamSynchronize");
}
static int num_sms() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return v > 0 ? v : 1;
}
template <class T> static pagd_status launch(pagd_solver* s, const Params& P) {
    cudaError_t e;
    int used = 0;
    switch (fixed_len(P.n0, P.n1)) {
        case 64: e = pagd_launch<T, 64>(P, s->grid, s->threads, s->smem, s->stream, &used); break;
        case 128: e = pagd_launch<T, 128>(P, s->grid, s->threads, s->smem, s->stream, &used); break;
        case 256: e = pagd_launch<T, 256>(P, s->grid, s->threads, s->smem, s->stream, &used); break;
        case 512: e = pagd_launch<T, 512>(P, s->grid, s->threads, s->smem, s->stream, &used); break;
        default: e = pagd_launch<T, 0>(P, s->grid, s->threads, s->smem, s->stream, &used); break;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "cooperative launch of pagd_kernel");
    s->grid_used = used;
    return PAGD_OK;
}
#endif

static pagd_status run_program(pagd_solver* s, Params& P) {
    pagd_status st = dzero(s, P.sc, sizeof(Scal));
    if (st != PAGD_OK) return st;
    if (s->tsize == 8) st = launch<double>(s, P);
    else st = launch<float>(s, P);
    return st;
}

// The FP32 iteration passes stage their inputs through shared memory
// (row_pass_staged / col_pass_staged) when a warp slice of warp_bytes holds
// the staging slots (PFC two, FCH one); fixed line lengths only.  PAGD_STAGED=0 keeps the
// register-staged passes (the same arithmetic, for comparison).
static bool stage_fits(const pagd_solver* s, size_t warp_bytes) {
    const int last = s->dim - 1;
    const int nf = fixed_len(s->n[0], s->n[last]);
    if (nf == 0 || s->tsize != 4) return false;
    if (const char* e = std::getenv("PAGD_STAGED"))
        if (e[0] == '0' && e[1] == 0) return false;
    const int k = k_iter(s->model);
    // the middle passes of a cubic grid stage too (mid_pass_staged)
    if (s->dim == 3 && s->n[1] == nf && mid_staged_smem(nf) > warp_bytes) return false;
    const int sl = staged_slots(s->model);
    return row_staged_smem(nf, k, staged_row_state(s->model), sl) <= warp_bytes &&
           col_staged_smem(nf, k, 3, sl) <= warp_bytes;
}

// One warp per row unit / column / middle unit.  A CTA has as many warps (at
// most 8) as their shared-memory slices allow (one in the emulation).  The
// grid covers the largest unit count and is capped at the co-resident CTA
// count when launched.
static void make_plan(pagd_solver* s) {
    const int last = s->dim - 1, nm = s->dim == 3 ? s->n[1] : 1;
    s->logtw = 0;
    for (int d = 0; d < s->dim; d++) s->logtw = std::max(s->logtw, ilog2(s->n[d]));
    s->warp_bytes = warp_smem_bytes(s->n[0], s->n[last], s->model, s->tsize, fixed_len(s->n[0], s->n[last]), nm);
#ifdef PAGD_EMU
    const int wpb = 1;
#else
    const size_t room = kMaxSmem - tw_smem_bytes(s->logtw);
    int wpb = (int)std::min<size_t>((size_t)(kMaxThreads / 32), room / s->warp_bytes);
    if (wpb < 1) wpb = 1;
#endif
    s->threads = wpb * 32;
    const long long rows = rows_of(s);
    long long units = rows / 2;
    if ((long long)s->h1 * nm > units) units = (long long)s->h1 * nm;
    const int sms = num_sms();
    s->grid = units < sms ? (int)units : sms;
    if ((long long)s->grid < (units + wpb - 1) / wpb) {
        const long long g = (units + wpb - 1) / wpb;
        s->grid = (int)(g < 65536 ? g : 65536);  // capped at the co-resident CTAs when launched
    }
    if (s->grid < 1) s->grid = 1;
    s->smem = tw_smem_bytes(s->logtw) + (size_t)wpb * s->warp_bytes;
    // CTA-cooperative units for the passes with FP64 lines when a phase has
    // fewer units than half the warps (most warps would otherwise idle and an
    // FP64 line would run on one SM sub-partition); fixed line lengths only.
    // PAGD_COOP=0 / 1 overrides the choice.
    s->coop = (fixed_len(s->n[0], s->n[last]) != 0 && 2 * units <= (long long)s->grid * wpb) ? 1 : 0;
    if (const char* e = std::getenv("PAGD_COOP")) {
        if ((e[0] == '0' || e[0] == '1') && e[1] == 0) s->coop = fixed_len(s->n[0], s->n[last]) != 0 ? e[0] - '0' : 0;
    }
    // Cluster-resident iterations (cluster.cuh) on square 2D grids of 64, 128
    // or 256 points per axis, when the cluster buffers fit a CTA's shared
    // memory.  Off by default (measured slower than the device-wide phases so
    // far); PAGD_CLUSTER=1 turns it on, 0 off.  A launch with 16-CTA clusters
    // co-schedules fewer CTAs than a 256^2 grid has columns, so there the
    // device-wide phases run warp-owned.
    s->cl = 0;
    const int nf = fixed_len(s->n[0], s->n[last]);
    bool want_cl = false;
    if (const char* e = std::getenv("PAGD_CLUSTER")) want_cl = e[0] == '1' && e[1] == 0;
    if (want_cl && s->dim == 2 && cl_size_for(nf) > 0) {
        const ClOff co = cl_offsets(nf, k_iter(s->model), s->tsize);
        const size_t need = tw_smem_bytes(s->logtw) + co.end;
        bool on = need <= kMaxSmem;
#ifndef PAGD_EMU
        on = on && wpb == kMaxThreads / 32;
#endif
        if (on) {
            s->cl = cl_size_for(nf);
            if (need > s->smem) s->smem = need;
            if (nf == 256) s->coop = 0;
        }
    }
    s->stage = (!s->cl && stage_fits(s, s->warp_bytes)) ? 1 : 0;
    // FP32 iteration passes with CTA-cooperative units (unstaged FP32 passes
    // of fixed line length): opt-in with PAGD_COOP32=1.  Measured slower on
    // FCH 256^2 (128 row pairs on 152 SMs), where the FP64 passes gain from
    // them: 382.7 against 359.3 us per step, the column pass 13.4 against
    // 10.3 us.
    s->coop32 = 0;
    if (const char* e = std::getenv("PAGD_COOP32")) {
        if (e[0] == '1' && e[1] == 0)
            s->coop32 = (fixed_len(s->n[0], s->n[last]) != 0 && s->tsize == 4 && !s->stage && !s->cl) ? 1 : 0;
    }
}

// ----------------------------------------------------------------- C ABI

extern "C" {

pagd_status pagd_default_opts(pagd_opts* o) {
    if (!o) return PAGD_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->s = 0.9;
    o->n_eta = 5;
    for (int j = 0; j < 5; j++) o->eta[j] = std::sqrt(0.1 + 0.475 * j);
    o->max_iter = 1000;
    o->theta_mode = 0;
    o->accel = 1;
    return PAGD_OK;
}

static pagd_status init_common(pagd_solver** out, int model, int dim, const int* n, const double* L,
                               double eps, double eta1, double eta2, double tau, double M, int scheme,
                               int precision, const pagd_opts* opts, void* stream) {
    if (!out) return PAGD_EINVAL;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !n || !L) return PAGD_EINVAL;
    for (int d = 0; d < dim; d++) {
        if (!pow2_ok(n[d]) || !(L[d] > 0.0) || !std::isfinite(L[d])) return PAGD_EINVAL;
    }
    if (!(M > 0.0) || !std::isfinite(eps)) return PAGD_EINVAL;
    if (scheme < PAGD_BDF2 || scheme > PAGD_LMP) return PAGD_EINVAL;
    if (precision != PAGD_FP64 && precision != PAGD_FP32_MIXED) return PAGD_EINVAL;
    pagd_opts o;
    if (opts) o = *opts;
    else pagd_default_opts(&o);
    if (!(o.s > 0.0) || o.n_eta < 1 || o.n_eta > 16 || o.max_iter < 1 || o.max_iter > 100000 ||
        (o.theta_mode != 0 && o.theta_mode != 1) || (o.accel != 0 && o.accel != 1))
        return PAGD_EINVAL;
    for (int j = 0; j < o.n_eta; j++)
        if (!(o.eta[j] > 0.0)) return PAGD_EINVAL;
    pagd_solver* s = new (std::nothrow) pagd_solver();
    if (!s) return PAGD_ENOMEM;
    s->model = model;
    s->dim = dim;
    for (int d = 0; d < 3; d++) {
        s->n[d] = d < dim ? n[d] : 1;
        s->L[d] = d < dim ? L[d] : 1.0;
    }
    s->eps = eps;
    s->eta1 = eta1;
    s->eta2 = eta2;
    s->tau = tau;
    s->M = M;
    s->scheme = scheme;
    s->precision = precision;
    s->opts = o;
    s->stream = stream;
    s->npts = (long long)s->n[0] * s->n[1] * s->n[2];
    s->h1 = s->n[dim - 1] / 2 + 1;
    s->nslots = o.max_iter + 16 * 9 + 16;
    s->tsize = precision == PAGD_FP64 ? 8 : 4;
    s->ws = nullptr;
    s->have_state = 0;
    s->step = 0;
    s->cur = 0;
    s->trace = 0;
    s->ref_valid = 0;
    s->dt_prev = 0.0;
    plan_layout(s);
    make_plan(s);
    *out = s;
    return PAGD_OK;
}

pagd_status pfc_init(pagd_solver** out, int dim, const int* n, const double* L, double eps, double M,
                     int scheme, int precision, const pagd_opts* opts, void* stream) {
    return init_common(out, PAGD_PFC, dim, n, L, eps, 0.0, 0.0, 0.0, M, scheme, precision, opts, stream);
}

pagd_status fch_init(pagd_solver** out, int dim, const int* n, const double* L, double eps, double eta1,
                     double eta2, double tau, double M, int scheme, int precision, const pagd_opts* opts,
                     void* stream) {
    if (!std::isfinite(eta1) || !std::isfinite(eta2) || !std::isfinite(tau)) return PAGD_EINVAL;
    return init_common(out, PAGD_FCH, dim, n, L, eps, eta1, eta2, tau, M, scheme, precision, opts, stream);
}

pagd_status pagd_workspace_size(const pagd_solver* s, size_t* bytes) {
    if (!s || !bytes) return PAGD_EINVAL;
    *bytes = s->ws_bytes;
    return PAGD_OK;
}

pagd_status pagd_set_workspace(pagd_solver* s, void* dev_ptr, size_t bytes) {
    if (!s) return PAGD_EINVAL;
    if (!dev_ptr || ((uintptr_t)dev_ptr & 255)) return fail(s, PAGD_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < s->ws_bytes) return fail(s, PAGD_ENOMEM, "workspace smaller than pagd_workspace_size");
    s->ws = (char*)dev_ptr;
    s->have_state = 0;
    // twiddles exp(-2 pi i m / kNMax) from the host libm in long double
    std::vector<double2> t64(kNMax);
    std::vector<float2> t32(kNMax);
    for (int m = 0; m < kNMax; m++) {
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)m / (long double)kNMax;
        t64[m].x = (double)cosl(ang);
        t64[m].y = (double)sinl(ang);
        t32[m].x = (float)t64[m].x;
        t32[m].y = (float)t64[m].y;
    }
    pagd_status st = dcopy(s, s->ws + s->off[O_TW64], t64.data(), sizeof(double2) * kNMax);
    if (st == PAGD_OK) st = dcopy(s, s->ws + s->off[O_TW32], t32.data(), sizeof(float2) * kNMax);
    if (st == PAGD_OK) st = dsync(s);
    return st;
}

pagd_status pagd_set_state(pagd_solver* s, const double* u0_dev) {
    if (!s || !u0_dev) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    const size_t b = sizeof(double) * s->npts;
    s->cur = 0;
    pagd_status st = dcopy(s, s->ws + s->off[O_U0], u0_dev, b);
    if (st == PAGD_OK) st = dcopy(s, s->ws + s->off[O_U1], u0_dev, b);
    if (st == PAGD_OK) st = dzero(s, s->ws + s->off[O_MASS], 4 * sizeof(double));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    s->have_state = 1;
    s->step = 0;
    s->dt_prev = 0.0;
    s->ref_valid = 0;
    return PAGD_OK;
}

static pagd_status status_from(int st) {
    switch (st) {
        case ST_OK: return PAGD_OK;
        case ST_ENOCONV: return PAGD_ENOCONV;
        case ST_EPRECOND: return PAGD_EPRECOND;
        case ST_ENAN: return PAGD_ENAN;
        default: return PAGD_ECUDA;
    }
}

// Parameters of a run of nsteps steps of size dt on s (one launch).
static Params run_params(const pagd_solver* s, double* u_out, double dt, int nsteps, double tol) {
    Params P = base_params(s);
    const bool imex = s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP;
    P.prog = imex ? PROG_IMEX : PROG_RUN;
    P.tol = tol;
    P.dt = dt;
    P.dt_prev0 = (s->step == 0) ? dt : s->dt_prev;
    P.nsteps = nsteps;
    P.out_real = u_out;
    fill_step_table(P);
    return P;
}

// Reads back the outcome of a run launched with P (the stream must be idle):
// per-step results, the solver's step count and history slot.  bar_error: the
// launch's device barrier gave up.
static pagd_status run_finish(pagd_solver* s, const Params& P, double dt, int nsteps, int* iters, double* resid,
                              bool bar_error, int* used_guess = nullptr) {
    const bool imex = s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP;
    Scal sc;
    pagd_status st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    bar_error = bar_error || sc.bar_error;
    std::vector<StepStat> stats(nsteps > 0 ? nsteps : 1);
    const int ndone = sc.steps_done;
    const int nrec = (sc.status != ST_OK) ? ndone + 1 : ndone;
    if (nrec > 0) {
        st = dcopy(s, stats.data(), P.stats, sizeof(StepStat) * (size_t)(nrec < nsteps ? nrec : nsteps));
        if (st == PAGD_OK) st = dsync(s);
        if (st != PAGD_OK) return st;
    }
    for (int i = 0; i < nrec && i < nsteps; i++) {
        if (iters) iters[i] = stats[i].iters;
        if (resid) resid[i] = stats[i].resid;
        if (used_guess) used_guess[i] = stats[i].used_guess;
    }
    if (ndone > 0) {
        s->step += ndone;
        s->cur ^= (ndone & 1);
        s->dt_prev = dt;
    }
    // the reference spectra of the incremental base evaluation stay valid only
    // after a run that ended on an accepted step
    s->ref_valid = (!imex && sc.status == ST_OK && !bar_error && ndone == nsteps && nsteps > 0) ? 1 : 0;
    if (bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    if (sc.status != ST_OK) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "step %d (global %d) failed with status %d after %d evaluations",
                      sc.fail_step, s->step, sc.status, nrec > 0 ? stats[nrec - 1].iters : 0);
        return fail(s, status_from(sc.status), buf);
    }
    if (ndone != nsteps) return fail(s, PAGD_ECUDA, "kernel ended early");
    return PAGD_OK;
}

static pagd_status run_chunk(pagd_solver* s, double* u_out, double dt, int nsteps, double tol, int* iters,
                             double* resid) {
    Params P = run_params(s, u_out, dt, nsteps, tol);
    pagd_status st = run_program(s, P);
    if (st != PAGD_OK) return st;
    return run_finish(s, P, dt, nsteps, iters, resid, false);
}

pagd_status pagd_run(pagd_solver* s, double* u_dev, double dt, int nsteps, double tol, int* iters_out,
                     double* resid_out) {
    if (!s) return PAGD_EINVAL;
    if (!s->ws || !s->have_state) return fail(s, PAGD_ESTATE, "workspace and state must be set first");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0 || !(tol >= 0.0))
        return fail(s, PAGD_EINVAL, "bad dt / nsteps / tol");
    int done = 0;
    while (done < nsteps) {
        const int c = (nsteps - done > kMaxChunk) ? kMaxChunk : nsteps - done;
        const bool last = done + c == nsteps;
        pagd_status st = run_chunk(s, last ? u_dev : nullptr, dt, c, tol, iters_out ? iters_out + done : nullptr,
                                   resid_out ? resid_out + done : nullptr);
        if (st != PAGD_OK) return st;
        done += c;
    }
    return PAGD_OK;
}

// one step from the caller's initial iterate, the new state kept in the solver
// (u_dev nullable)
static pagd_status run_with_guess(pagd_solver* s, const double* guess_dev, double dt, double tol, int* iters_out,
                                  double* resid_out, int* used_guess_out, double* u_dev = nullptr) {
    Params P = run_params(s, u_dev, dt, 1, tol);
    P.guess = guess_dev;
    pagd_status st = run_program(s, P);
    if (st != PAGD_OK) return st;
    return run_finish(s, P, dt, 1, iters_out, resid_out, false, used_guess_out);
}

pagd_status pagd_step_with_guess(pagd_solver* s, double* u_dev, const double* guess_dev, double dt, double tol,
                                 int* iters_out, double* resid_out, int* used_guess_out) {
    if (!s) return PAGD_EINVAL;
    if (!u_dev || !guess_dev) return fail(s, PAGD_EINVAL, "null output or guess");
    if (!s->ws || !s->have_state) return fail(s, PAGD_ESTATE, "workspace and state must be set first");
    if (s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP)
        return fail(s, PAGD_EINVAL, "an initial iterate applies to the implicit schemes only");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(tol >= 0.0)) return fail(s, PAGD_EINVAL, "bad dt / tol");
    return run_with_guess(s, guess_dev, dt, tol, iters_out, resid_out, used_guess_out, u_dev);
}

pagd_status pagd_step(pagd_solver* s, double* u_dev, double dt, double tol, int* iters_out, double* resid_out) {
    if (!u_dev) return fail(s, PAGD_EINVAL, "null output");
    return pagd_run(s, u_dev, dt, 1, tol, iters_out, resid_out);
}

pagd_status pagd_run_host(pagd_solver* s, const double* u0_host, double* u_host_out, double dt, int nsteps,
                          double tol, int* iters_out, double* resid_out) {
    if (!s || !u0_host || !u_host_out) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    const size_t b = sizeof(double) * s->npts;
    s->cur = 0;
    pagd_status st = dcopy(s, s->ws + s->off[O_U0], u0_host, b);
    if (st == PAGD_OK) st = dcopy(s, s->ws + s->off[O_U1], u0_host, b);
    if (st == PAGD_OK) st = dzero(s, s->ws + s->off[O_MASS], 4 * sizeof(double));
    if (st != PAGD_OK) return st;
    s->have_state = 1;
    s->step = 0;
    s->dt_prev = 0.0;
    s->ref_valid = 0;
    st = pagd_run(s, nullptr, dt, nsteps, tol, iters_out, resid_out);
    if (st != PAGD_OK) return st;
    st = dcopy(s, u_host_out, s->ws + (s->cur ? s->off[O_U1] : s->off[O_U0]), b);
    if (st == PAGD_OK) st = dsync(s);
    return st;
}

pagd_status pagd_get_state(pagd_solver* s, double* un_dev, double* unm1_dev, int* step) {
    if (!s) return PAGD_EINVAL;
    if (!s->ws || !s->have_state) return fail(s, PAGD_ESTATE, "no state");
    const size_t b = sizeof(double) * s->npts;
    const size_t oc = s->cur ? s->off[O_U1] : s->off[O_U0];
    const size_t op = s->cur ? s->off[O_U0] : s->off[O_U1];
    pagd_status st = PAGD_OK;
    if (un_dev) st = dcopy(s, un_dev, s->ws + oc, b);
    if (st == PAGD_OK && unm1_dev) st = dcopy(s, unm1_dev, s->ws + op, b);
    if (st == PAGD_OK) st = dsync(s);
    if (step) *step = s->step;
    return st;
}

static pagd_status reduce_program(pagd_solver* s, int prog, const double* u_dev, double* red2) {
    Params P = base_params(s);
    P.prog = prog;
    P.in_real = u_dev;
    pagd_status st = run_program(s, P);
    if (st != PAGD_OK) return st;
    Scal sc;
    st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    if (sc.bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    red2[0] = sc.red[0];
    red2[1] = sc.red[1];
    return PAGD_OK;
}

pagd_status pagd_energy(pagd_solver* s, const double* u_dev, double* E) {
    if (!s || !u_dev || !E) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    double r[2];
    pagd_status st = reduce_program(s, PROG_ENERGY, u_dev, r);
    if (st != PAGD_OK) return st;
    const double h = cell_volume(s);
    const double N = (double)s->npts;
    if (s->model == PAGD_PFC) *E = h * (r[0] + r[1] / N);
    else *E = h * r[0] - 0.5 * s->eps * s->eps * s->eta1 * h * r[1] / N;
    return PAGD_OK;
}

pagd_status pagd_mass(pagd_solver* s, const double* u_dev, double* m) {
    if (!s || !u_dev || !m) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    double r[2];
    pagd_status st = reduce_program(s, PROG_MASS, u_dev, r);
    if (st != PAGD_OK) return st;
    *m = r[0] * cell_volume(s);
    return PAGD_OK;
}

pagd_status pagd_rhs(pagd_solver* s, const double* v_dev, double* r_dev) {
    if (!s || !v_dev || !r_dev) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    Params P = base_params(s);
    P.prog = PROG_RHS;
    P.in_real = v_dev;
    P.out_real = r_dev;
    pagd_status st = run_program(s, P);
    if (st != PAGD_OK) return st;
    Scal sc;
    st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    if (sc.bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    return PAGD_OK;
}

// ERR of adaptive stepping: sqrt(sum (ut - uh)^2 / sum uh^2), uh = sum c_j in_j
static pagd_status est_program(pagd_solver* s, const double* ut, const double* const in[4], const double c[4],
                               double* err) {
    Params P = base_params(s);
    P.prog = PROG_EST;
    P.in_real = ut;
    for (int j = 0; j < 4; j++) {
        P.est_in[j] = in[j];
        P.est_c[j] = c[j];
    }
    pagd_status st = run_program(s, P);
    if (st != PAGD_OK) return st;
    Scal sc;
    st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    if (sc.bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    *err = sc.red[1] > 0.0 ? std::sqrt(sc.red[0] / sc.red[1]) : 0.0;
    return PAGD_OK;
}

pagd_status pagd_run_adaptive(pagd_solver* s, double T, double dt_min, double dt_max, double step_tol, double tol,
                              int max_steps, double* scratch_dev, double* u_dev, double* t_out, double* dt_out,
                              int* iters_out, int* nsteps_out, int* rejected_out) {
    if (!s || !scratch_dev) return PAGD_EINVAL;
    if (!s->ws || !s->have_state) return fail(s, PAGD_ESTATE, "workspace and state must be set first");
    if (!(T > 0.0) || !(dt_min > 0.0) || !(dt_max >= dt_min) || !(step_tol > 0.0) || !(tol >= 0.0) ||
        max_steps < 1 || !std::isfinite(T) || !std::isfinite(dt_max))
        return fail(s, PAGD_EINVAL, "bad T / dt_min / dt_max / step_tol / tol / max_steps");
    const size_t nb = sizeof(double) * (size_t)s->npts;
    const long long N = s->npts;
    // scratch: R(u^n), R(u^{n-1}), R(ut), ut, u^{n-2}, saved u^{n-1}
    double* Rn = scratch_dev;
    double* Rm = scratch_dev + N;
    double* Rt = scratch_dev + 2 * N;
    double* ut = scratch_dev + 3 * N;
    double* um2 = scratch_dev + 4 * N;
    double* save = scratch_dev + 5 * N;
    const bool mp = s->scheme == PAGD_MP;
    auto slot = [&](int c) { return (double*)(s->ws + (c ? s->off[O_U1] : s->off[O_U0])); };
    double* mass = (double*)(s->ws + s->off[O_MASS]);
    double mass_save[2];
    pagd_status st = pagd_rhs(s, slot(s->cur), Rn);
    if (st == PAGD_OK) st = dcopy(s, Rm, Rn, nb);
    if (st != PAGD_OK) return st;
    double t = 0.0, dtt = dt_min, dt_prev = s->step > 0 ? s->dt_prev : dt_min;
    double dtn = 0.0, dtnm1 = 0.0;  // the last two accepted steps (midAB2)
    int n = 0, rej = 0;
    if (t_out) t_out[0] = 0.0;
    while (t < T && n < max_steps) {
        // tentative step from (u^n, u^{n-1}); its writes are undone on rejection
        const int cur0 = s->cur, step0 = s->step;
        const double dtp0 = s->dt_prev;
        st = dcopy(s, save, slot(cur0 ^ 1), nb);
        if (st == PAGD_OK) st = dcopy(s, mass_save, mass, sizeof(mass_save));
        if (st == PAGD_OK) st = dsync(s);
        if (st != PAGD_OK) return st;
        s->dt_prev = dt_prev;
        int it = 0;
        double res = 0.0;
        st = run_chunk(s, ut, dtt, 1, tol, &it, &res);
        if (st != PAGD_OK) return st;
        st = pagd_rhs(s, ut, Rt);
        if (st != PAGD_OK) return st;
        double err = 0.0;
        if (mp && n >= 2) {
            const double a = (dtt + dtn) * (dtt + dtn + dtnm1) / (dtn * (dtn + dtnm1));
            const double b = dtt * (dtt + dtn + dtnm1) / (dtn * dtnm1);
            const double c = dtt * (dtt + dtn) / (dtnm1 * (dtn + dtnm1));
            const double* in[4] = {slot(cur0), save, um2, nullptr};
            const double cf[4] = {a, -b, c, 0.0};
            st = est_program(s, ut, in, cf, &err);
            const double Rn_ = 1.0 / 24.0 + 0.125 * (1.0 + dtn / dtt) * (1.0 + 2.0 * dtn / dtt + dtnm1 / dtt);
            err /= (1.0 - 1.0 / (24.0 * Rn_));
        } else {
            const double rho = dtt / (n > 0 ? dt_prev : dtt);
            const double* in[4] = {slot(cur0), Rt, Rn, Rm};
            const double cf[4] = {1.0, dtt / 6.0 * (3.0 + 2.0 * rho) / (1.0 + rho), dtt / 6.0 * (3.0 + rho),
                                  -dtt / 6.0 * rho * rho / (1.0 + rho)};
            st = est_program(s, ut, in, cf, &err);
        }
        if (st != PAGD_OK) return st;
        const double tmp = dtt;
        if (err <= step_tol || dtt <= dt_min) {
            // accept: the solver already holds u^{n+1} = ut and u^n
            st = dcopy(s, um2, save, nb);
            if (st == PAGD_OK) st = dcopy(s, Rm, Rn, nb);
            if (st == PAGD_OK) st = dcopy(s, Rn, Rt, nb);
            if (st != PAGD_OK) return st;
            dtnm1 = dtn;
            dtn = dtt;
            dt_prev = dtt;
            t += dtt;
            if (t_out) t_out[n + 1] = t;
            if (dt_out) dt_out[n] = dtt;
            if (iters_out) iters_out[n] = it;
            n++;
        } else {
            // reject: put back u^{n-1}, the mass accumulators and the counters
            st = dcopy(s, slot(cur0 ^ 1), save, nb);
            if (st == PAGD_OK) st = dcopy(s, mass, mass_save, sizeof(mass_save));
            if (st == PAGD_OK) st = dsync(s);
            if (st != PAGD_OK) return st;
            s->cur = cur0;
            s->step = step0;
            s->dt_prev = dtp0;
            s->ref_valid = 0;  // the reference spectra moved with the rejected step
            rej++;
        }
        dtt = 0.9 * std::cbrt(step_tol / (err > 1e-300 ? err : 1e-300)) * tmp;
        dtt = std::max(dt_min, std::min(dtt, dt_max));
    }
    if (nsteps_out) *nsteps_out = n;
    if (rejected_out) *rejected_out = rej;
    if (u_dev) {
        st = dcopy(s, u_dev, slot(s->cur), nb);
        if (st == PAGD_OK) st = dsync(s);
    }
    return st;
}

pagd_status pagd_fft_r2c(pagd_solver* s, const double* u_dev, double* spec_dev) {
    if (!s || !u_dev || !spec_dev) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    Params P = base_params(s);
    P.prog = PROG_FFT_FWD;
    P.in_real = u_dev;
    P.out_spec = (double2*)spec_dev;
    pagd_status st = run_program(s, P);
    if (st == PAGD_OK) st = dsync(s);
    return st;
}

pagd_status pagd_fft_c2r(pagd_solver* s, const double* spec_dev, double* u_dev) {
    if (!s || !u_dev || !spec_dev) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    Params P = base_params(s);
    P.prog = PROG_FFT_INV;
    P.in_spec = (const double2*)spec_dev;
    P.out_real = u_dev;
    pagd_status st = run_program(s, P);
    if (st == PAGD_OK) st = dsync(s);
    return st;
}

// ------------------------------------------------------------------------
// Allocation-free single step.
//
// Some callers cannot allocate device memory at the point where they need a
// step: runtimes that own the device allocator and forbid allocations by the
// libraries they host, and programs that fix their device-memory budget up
// front and must not grow it later.  pagd_step_static gives them one time step
// that uses a file-scope static device array as its scratch instead of a
// caller-provided workspace.  The array has a fixed size (kStaticScratchBytes,
// 8 MiB) and every GPU that loads this library holds it until the process
// exits.  Its head holds the twiddle tables, written once per device at
// set-up; the rest holds one solver workspace (pagd_workspace_size at most
// kStaticWorkspaceBytes: every 2D grid up to 128 x 128 points and every 3D grid
// up to 16 x 16 x 16 in either precision).  All calls share the one array and
// it keeps the last call's contents; everything that must start at zero is
// cleared by each call.  Calls whose work overlaps on the GPU (on different
// streams, or from different host threads) race on the array and must be
// serialised by the caller.
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
constexpr size_t kStaticTwBytes = ((sizeof(double2) + sizeof(float2)) * kNMax + 255) & ~(size_t)255;
constexpr size_t kStaticWorkspaceBytes = kStaticScratchBytes - kStaticTwBytes;  // 8,364,032
static_assert(kStaticWorkspaceBytes == 8364032, "the limit stated in include/pagd.h");
#ifndef PAGD_EMU
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
#else
alignas(256) static unsigned char g_static_scratch[kStaticScratchBytes];
#endif
constexpr int kMaxDevices = 64;
static void* g_static_ptr[kMaxDevices];
static std::mutex g_static_mu;  // guards g_static_ptr and the one-time set-up

// Device address of the static scratch for the current device, with the
// twiddle tables at its head.  In host code the array's name is only a
// host-side stand-in, so the address is obtained with cudaGetSymbolAddress,
// once per device, with that device current, and the tables are copied there
// with a synchronous cudaMemcpy.  This happens on the first call on each device
// (make that first call before any stream capture); the lock makes concurrent
// first calls from several host threads do it once.
static pagd_status static_scratch(pagd_solver* s, char** out) {
#ifdef PAGD_EMU
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[0]) {
        std::vector<double2> t64(kNMax);
        std::vector<float2> t32(kNMax);
        for (int m = 0; m < kNMax; m++) {
            const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)m / (long double)kNMax;
            t64[m] = double2{(double)cosl(ang), (double)sinl(ang)};
            t32[m] = float2{(float)t64[m].x, (float)t64[m].y};
        }
        std::memcpy(g_static_scratch, t64.data(), sizeof(double2) * kNMax);
        std::memcpy(g_static_scratch + sizeof(double2) * kNMax, t32.data(), sizeof(float2) * kNMax);
        g_static_ptr[0] = g_static_scratch;
    }
    (void)s;
    *out = (char*)g_static_ptr[0];
    return PAGD_OK;
#else
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(s, PAGD_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetSymbolAddress of the static scratch");
        // twiddles exp(-2 pi i m / kNMax) from the host libm in long double
        std::vector<double2> t64(kNMax);
        std::vector<float2> t32(kNMax);
        for (int m = 0; m < kNMax; m++) {
            const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)m / (long double)kNMax;
            t64[m].x = (double)cosl(ang);
            t64[m].y = (double)sinl(ang);
            t32[m].x = (float)t64[m].x;
            t32[m].y = (float)t64[m].y;
        }
        e = cudaMemcpy(ptr, t64.data(), sizeof(double2) * kNMax, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy((char*)ptr + sizeof(double2) * kNMax, t32.data(), sizeof(float2) * kNMax,
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(s, e, "cudaMemcpy of the static twiddle tables");
        g_static_ptr[dev] = ptr;
    }
    *out = (char*)g_static_ptr[dev];
    return PAGD_OK;
#endif
}

pagd_status pagd_step_static(pagd_solver* s, const double* un_dev, const double* unm1_dev, int step_index,
                             double dt, double dt_prev, double tol, double* unp1_dev, int* iters_out,
                             double* resid_out) {
    if (!s || !un_dev || !unm1_dev || !unp1_dev) return PAGD_EINVAL;
    if (step_index < 0 || !(dt > 0.0) || !std::isfinite(dt) || !(tol >= 0.0) ||
        (step_index > 0 && !(dt_prev > 0.0)))
        return fail(s, PAGD_EINVAL, "bad step index / dt / dt_prev / tol");
    if (s->ws_bytes > kStaticWorkspaceBytes) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "grid too large for the static scratch: needs %zu bytes, the maximum is %zu "
                      "(use pagd_set_workspace and pagd_step)",
                      s->ws_bytes, kStaticWorkspaceBytes);
        return fail(s, PAGD_EINVAL, buf);
    }
    char* head = nullptr;
    pagd_status st = static_scratch(s, &head);
    if (st != PAGD_OK) return st;
    char* w = head + kStaticTwBytes;
    const size_t b = sizeof(double) * s->npts;
    st = dcopy(s, w + s->off[O_U0], un_dev, b);
    if (st == PAGD_OK) st = dcopy(s, w + s->off[O_U1], unm1_dev, b);
    if (st == PAGD_OK) st = dzero(s, w + s->off[O_MASS], 4 * sizeof(double));
    if (st != PAGD_OK) return st;
    Params P = params_for(s, w);
    P.tw64 = (const double2*)head;
    P.tw32 = (const float2*)(head + sizeof(double2) * kNMax);
    P.trace = nullptr;  // no phase trace: pagd_get_trace reads the solver's own workspace
    const bool imex = s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP;
    P.prog = imex ? PROG_IMEX : PROG_RUN;
    P.ref_valid = 0;  // the static scratch holds no reference spectra
    P.cur0 = 0;
    P.step0 = step_index;
    P.tol = tol;
    P.dt = dt;
    P.dt_prev0 = step_index == 0 ? dt : dt_prev;
    P.nsteps = 1;
    P.out_real = unp1_dev;
    fill_step_table(P);
    st = run_program(s, P);
    if (st != PAGD_OK) return st;
    Scal sc;
    StepStat stat;
    st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dcopy(s, &stat, P.stats, sizeof(StepStat));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    if (iters_out) *iters_out = stat.iters;
    if (resid_out) *resid_out = stat.resid;
    if (sc.bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    if (sc.status != ST_OK) return fail(s, status_from(sc.status), "static-scratch step failed");
    if (sc.steps_done != 1) return fail(s, PAGD_ECUDA, "kernel ended early");
    return PAGD_OK;
}

// Device barrier probe (instrumentation, not in the paper): one launch of the
// solver's persistent kernel with its launch plan that runs `count` empty
// phases, each ended by the device-wide barrier; *us_per_phase receives the
// launch's device time / count (CUDA events on the solver's stream).
// Device time per phase of one launch of a probe program (P.nsteps phases).
static pagd_status timed_probe(pagd_solver* s, Params& P, double* us_per_phase) {
#ifdef PAGD_EMU
    pagd_status st = run_program(s, P);
    *us_per_phase = 0.0;
    return st;
#else
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaEventCreate");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(s, e, "cudaEventCreate");
    }
    pagd_status st = PAGD_OK;
    e = cudaEventRecord(e0, (cudaStream_t)s->stream);
    if (e == cudaSuccess) {
        st = run_program(s, P);
        e = cudaEventRecord(e1, (cudaStream_t)s->stream);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PAGD_OK) return st;
    if (e != cudaSuccess) return cuda_fail(s, e, "probe timing");
    Scal sc;
    st = dcopy(s, &sc, P.sc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    if (sc.bar_error) return fail(s, PAGD_ETIMEOUT, "device barrier timed out");
    *us_per_phase = 1000.0 * (double)ms / (double)P.nsteps;
    return PAGD_OK;
#endif
}

pagd_status pagd_barrier_probe(pagd_solver* s, int count, double* us_per_phase) {
    if (!s || count < 1 || count > 1000000 || !us_per_phase) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    Params P = base_params(s);
    P.prog = PROG_BARRIER;
    P.nsteps = count;
    P.trace = nullptr;
    return timed_probe(s, P, us_per_phase);
}

pagd_status pagd_pass_probe(pagd_solver* s, int pass, int count, double* us_per_pass) {
    if (!s || pass < 0 || pass > 3 || count < 1 || count > 1000000 || !us_per_pass) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    if (pass >= 2 && s->dim != 3) return fail(s, PAGD_EINVAL, "middle passes exist in 3D only");
    if (s->step < 1 || s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP)
        return fail(s, PAGD_ESTATE, "the pass probe needs a completed step of an implicit scheme");
    static const int kPass[4] = {PH_RI, PH_CI, PH_MF, PH_MI};
    Params P = run_params(s, nullptr, s->dt_prev, count, 0.0);
    P.prog = PROG_PASS;
    P.pass = kPass[pass];
    P.cl = 0;
    P.trace = nullptr;
    return timed_probe(s, P, us_per_pass);
}

// Launch plan of the solver's persistent kernel (instrumentation): CTAs of
// the last launch (0 before the first), threads per CTA, cluster size of the
// cluster-resident iterations (0: device-wide phases only), whether the
// passes with FP64 lines run CTA-cooperative units, dynamic shared memory.
pagd_status pagd_launch_info(const pagd_solver* s, int* grid, int* threads, int* cluster, int* coop,
                             size_t* smem, int* staged) {
    if (!s) return PAGD_EINVAL;
    if (staged) *staged = s->stage;
    if (grid) *grid = s->grid_used;
    if (threads) *threads = s->threads;
    if (cluster) *cluster = s->cl;
    if (coop) *coop = s->coop;
    if (smem) *smem = s->smem;
    return PAGD_OK;
}

pagd_status pagd_set_trace(pagd_solver* s, int enable) {
    if (!s) return PAGD_EINVAL;
    s->trace = enable ? 1 : 0;
    return PAGD_OK;
}

pagd_status pagd_get_trace(pagd_solver* s, int* phase, double* t_us, int cap, int* count) {
    if (!s || !count || cap < 0 || (cap > 0 && (!phase || !t_us))) return PAGD_EINVAL;
    if (!s->ws) return fail(s, PAGD_ESTATE, "no workspace");
    Scal sc;
    pagd_status st = dcopy(s, &sc, s->ws + s->off[O_SC], sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s);
    if (st != PAGD_OK) return st;
    const int n = sc.ntrace < kTraceCap ? sc.ntrace : kTraceCap;
    *count = n;
    unsigned long long rec[2 * 256];
    unsigned long long t0 = 0;
    for (int base = 0; base < n && base < cap; base += 256) {
        const int m = (n - base < 256) ? n - base : 256;
        st = dcopy(s, rec, s->ws + s->off[O_TRACE] + sizeof(unsigned long long) * 2 * base,
                   sizeof(unsigned long long) * 2 * m);
        if (st == PAGD_OK) st = dsync(s);
        if (st != PAGD_OK) return st;
        for (int i = 0; i < m && base + i < cap; i++) {
            if (base + i == 0) t0 = rec[1];
            phase[base + i] = (int)rec[2 * i];
            t_us[base + i] = (double)(rec[2 * i + 1] - t0) * 1e-3;
        }
    }
    return PAGD_OK;
}

// ------------------------------------------------------------ batches

}  // extern "C"

struct pagd_batch {
    std::vector<pagd_solver*> m;
    int tsize, logtw, grid, threads, wpb, grid_used;
    int sequential;  // the last run went member after member (batch_members_fill_the_device)
    size_t warp_bytes, smem, ws_bytes;
    char* ws;
    void* stream;
    std::string err;
};

static pagd_status bfail(pagd_batch* b, pagd_status st, const char* msg) {
    if (b) b->err = msg;
    return st;
}

static size_t batch_off_params() { return (sizeof(Scal) + 255) & ~(size_t)255; }

#ifdef PAGD_EMU
constexpr int kEmuBatchWarps = 3;  // warps per emulated CTA in batched launches
#endif

#ifdef PAGD_EMU
template <class T> static void batch_exec_host(const Params& P, const Ctl& c, const Tw& t, char* wsm, double* red) {
    switch (batch_nf(P.n0, P.n1)) {
        case 128: exec_phase<T, 128>(P, c, t, wsm, red); break;
        case 256: exec_phase<T, 256>(P, c, t, wsm, red); break;
        case 512: exec_phase<T, 512>(P, c, t, wsm, red); break;
        default: exec_phase<T, 0>(P, c, t, wsm, red); break;
    }
}
// the batched kernel's schedule, one CTA after the other and within a CTA one
// warp (of one thread) after the other, kEmuBatchWarps warps per CTA
template <class T> static pagd_status batch_launch(pagd_batch* b, const BatchParams& B) {
    std::vector<char> sm(b->smem + 64);
    char* base = (char*)(((uintptr_t)sm.data() + 15) & ~(uintptr_t)15);
    double red[32];
    gridDim.x = (unsigned)b->grid;
    blockDim.x = (unsigned)b->wpb;
    threadIdx.x = 0;
    const int ntw = 1 << B.logtw;
    double2* t64 = (double2*)base;
    float2* t32 = (float2*)(base + (size_t)ntw * sizeof(double2));
    for (int m = 0; m < ntw; m++) {
        t64[m] = B.tw64[m * (kNMax >> B.logtw)];
        t32[m] = B.tw32[m * (kNMax >> B.logtw)];
    }
    char* wsm = base + tw_smem_bytes(B.logtw) + batch_ctl_bytes(B.count);
    std::vector<Ctl> ctl(B.count);
    std::vector<long long> G(B.count + 1);
    for (int i = 0; i < B.count; i++) ctl[i] = ctl_init(B.PI[i]);
    const int wpb = b->wpb;
    const long long nw = (long long)b->grid * wpb;
    for (;;) {
        G[0] = 0;
        for (int i = 0; i < B.count; i++)
            G[i + 1] = G[i] + (ctl[i].ph == PH_DONE ? 0
                                                    : (long long)phase_units(B.PI[i], ctl[i].ph) *
                                                          weighted_unit_cost(B.PI[i], ctl[i]));
        const long long total = G[B.count];
        if (total == 0) break;
        for (int blk = 0; blk < b->grid; blk++) {
            blockIdx.x = (unsigned)blk;
            for (int wi = 0; wi < wpb; wi++) {
                threadIdx.x = (unsigned)wi;
                const long long gw = (long long)blk * wpb + wi;
                const long long clo = cost_start(gw, total, nw), chi = cost_start(gw + 1, total, nw);
                for (int i = 0; i < B.count; i++) {
                    if (G[i + 1] <= clo || G[i] >= chi || G[i + 1] == G[i]) continue;
                    const Params& P = B.PI[i];
                    Tw t{t64, t32, B.logtw, 0, 0, 0, 0};
                    batch_split(t, gw, nw, total, G[i], G[i + 1] - G[i], phase_units(P, ctl[i].ph),
                                (int)weighted_unit_cost(P, ctl[i]));
                    batch_exec_host<T>(P, ctl[i], t, wsm, red);
                }
            }
            threadIdx.x = 0;
        }
        for (int i = 0; i < B.count; i++)
            if (ctl[i].ph != PH_DONE) ctl_advance<T>(B.PI[i], ctl[i]);
    }
    return PAGD_OK;
}
#else
template <class T> static pagd_status batch_launch(pagd_batch* b, const BatchParams& B) {
    int used = 0;
    cudaError_t e = pagd_batch_launch<T>(B, b->grid, b->threads, b->smem, b->stream, &used);
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "cooperative launch of pagd_batch_kernel: %s", cudaGetErrorString(e));
        return bfail(b, PAGD_ECUDA, buf);
    }
    b->grid_used = used;
    return PAGD_OK;
}
#endif

extern "C" {

pagd_status pagd_batch_create(pagd_batch** out, pagd_solver* const* members, int count) {
    if (!out) return PAGD_EINVAL;
    *out = nullptr;
    if (!members || count < 1 || count > kMaxBatch) return PAGD_EINVAL;
    for (int i = 0; i < count; i++) {
        if (!members[i]) return PAGD_EINVAL;
        if (members[i]->tsize != members[0]->tsize) return PAGD_EINVAL;  // one precision per batch
        for (int j = 0; j < i; j++)
            if (members[j] == members[i]) return PAGD_EINVAL;
    }
    pagd_batch* b = new (std::nothrow) pagd_batch();
    if (!b) return PAGD_ENOMEM;
    b->m.assign(members, members + count);
    b->tsize = members[0]->tsize;
    b->stream = members[0]->stream;
    b->logtw = 0;
    b->warp_bytes = 0;
    for (pagd_solver* s : b->m) {
        const int last = s->dim - 1, nm = s->dim == 3 ? s->n[1] : 1;
        for (int d = 0; d < s->dim; d++) b->logtw = std::max(b->logtw, ilog2(s->n[d]));
        b->warp_bytes = std::max(b->warp_bytes, warp_smem_bytes(s->n[0], s->n[last], s->model, s->tsize,
                                                                batch_nf(s->n[0], s->n[last]), nm));
    }
#ifdef PAGD_EMU
    const int wpb = kEmuBatchWarps;
#else
    const size_t fixed = tw_smem_bytes(b->logtw) + batch_ctl_bytes(count);
    int wpb = fixed < kMaxSmem ? (int)std::min<size_t>((size_t)(kMaxThreads / 32), (kMaxSmem - fixed) / b->warp_bytes) : 0;
    if (wpb < 1) wpb = 1;
#endif
    b->wpb = wpb;
    b->threads = wpb * 32;
    b->smem = tw_smem_bytes(b->logtw) + batch_ctl_bytes(count) + (size_t)wpb * b->warp_bytes;
    if (b->smem > kMaxSmem) {
        delete b;
        return PAGD_EINVAL;
    }
    b->grid = num_sms();
    b->ws_bytes = batch_off_params() + sizeof(Params) * (size_t)count;
    b->ws = nullptr;
    *out = b;
    return PAGD_OK;
}

// Launch shape of the batched kernel: warps per CTA (each with its slice of
// shared memory for one unit's lines) and CTAs per SM (the grid is that many
// per SM, capped at the co-resident count when launched).  Together they fix
// how the units of every global phase are tiled over the machine; an
// autotuner times the candidates and keeps the fastest.
pagd_status pagd_batch_set_shape(pagd_batch* b, int warps_per_cta, int ctas_per_sm) {
    if (!b || warps_per_cta < 1 || warps_per_cta > kMaxThreads / 32 || ctas_per_sm < 1 || ctas_per_sm > 8)
        return PAGD_EINVAL;
    const size_t smem = tw_smem_bytes(b->logtw) + batch_ctl_bytes((int)b->m.size()) + (size_t)warps_per_cta * b->warp_bytes;
    if (smem > kMaxSmem) return bfail(b, PAGD_EINVAL, "the warps' shared-memory slices do not fit one CTA");
#ifndef PAGD_EMU
    int dev = 0, cap = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return bfail(b, PAGD_ECUDA, cudaGetErrorString(e));
    if ((size_t)ctas_per_sm * (smem + 1024) > (size_t)cap)
        return bfail(b, PAGD_EINVAL, "that many CTAs per SM do not fit the SM's shared memory");
    if (ctas_per_sm * warps_per_cta * 32 > 2048) return bfail(b, PAGD_EINVAL, "too many threads per SM");
#endif
    b->wpb = warps_per_cta;
    b->threads = warps_per_cta * 32;
    b->smem = smem;
    b->grid = ctas_per_sm * num_sms();
    return PAGD_OK;
}

// The batched kernel's launch plan: CTAs of the last launch (the planned grid
// before the first), warps per CTA, dynamic shared memory per CTA, and whether
// the last run went member after member.
pagd_status pagd_batch_launch_info(const pagd_batch* b, int* grid, int* warps_per_cta, size_t* smem,
                                   int* sequential, int* staged) {
    if (!b) return PAGD_EINVAL;
    if (staged) {
        *staged = 0;
        for (const pagd_solver* m : b->m) *staged += stage_fits(m, b->warp_bytes) ? 1 : 0;
    }
    if (sequential) *sequential = b->sequential;
    if (grid) *grid = b->grid_used > 0 ? b->grid_used : b->grid;
    if (warps_per_cta) *warps_per_cta = b->wpb;
    if (smem) *smem = b->smem;
    return PAGD_OK;
}

pagd_status pagd_batch_workspace_size(const pagd_batch* b, size_t* bytes) {
    if (!b || !bytes) return PAGD_EINVAL;
    *bytes = b->ws_bytes;
    return PAGD_OK;
}

pagd_status pagd_batch_set_workspace(pagd_batch* b, void* dev_ptr, size_t bytes) {
    if (!b || !dev_ptr) return PAGD_EINVAL;
    if (bytes < b->ws_bytes) return bfail(b, PAGD_ENOMEM, "batch workspace too small");
    if (((uintptr_t)dev_ptr & 255) != 0) return bfail(b, PAGD_EINVAL, "batch workspace not 256-byte aligned");
    b->ws = (char*)dev_ptr;
    return PAGD_OK;
}

static pagd_status batch_chunk(pagd_batch* b, double dt, int nsteps, double tol, std::vector<int>& live,
                               int done, int total_steps, int* iters_out, double* resid_out, int* status_out,
                               const double* const* guesses = nullptr, int* used_out = nullptr) {
    const int count = (int)b->m.size();
    std::vector<Params> PI(count);
    pagd_status st = PAGD_OK;
    for (int i = 0; i < count; i++) {
        pagd_solver* s = b->m[i];
        PI[i] = run_params(s, nullptr, dt, live[i] ? nsteps : 0, tol);
        PI[i].trace = nullptr;
        PI[i].warp_bytes = (long long)b->warp_bytes;
        PI[i].coop = 0;  // batch warps own their units: no CTA-wide barriers
        PI[i].coop32 = 0;
        PI[i].cl = 0;    // and every phase of a batch is device-wide
        PI[i].stage = stage_fits(s, b->warp_bytes) ? 1 : 0;
        PI[i].logtw = b->logtw;
        PI[i].guess = guesses ? guesses[i] : nullptr;  // the first step's initial iterate (nullable)
        st = dzero(s, PI[i].sc, sizeof(Scal));
        if (st != PAGD_OK) return bfail(b, st, s->err.c_str());
    }
    pagd_solver* s0 = b->m[0];
    Scal* bsc = (Scal*)b->ws;
    Params* dPI = (Params*)(b->ws + batch_off_params());
    st = dzero(s0, bsc, sizeof(Scal));
    if (st == PAGD_OK) st = dcopy(s0, dPI, PI.data(), sizeof(Params) * (size_t)count);
    if (st != PAGD_OK) return bfail(b, st, s0->err.c_str());
    BatchParams B;
    B.PI = dPI;
    B.count = count;
    B.logtw = b->logtw;
    B.sc = bsc;
    B.tw64 = PI[0].tw64;
    B.tw32 = PI[0].tw32;
    // tracing on the first member records the launch's global phases there
    B.trace = s0->trace ? (unsigned long long*)(s0->ws + s0->off[O_TRACE]) : nullptr;
    B.trace_cap = kTraceCap;
    B.ntrace = &PI[0].sc->ntrace;
    st = (b->tsize == 8) ? batch_launch<double>(b, B) : batch_launch<float>(b, B);
    if (st != PAGD_OK) return st;
    Scal bs;
    st = dcopy(s0, &bs, bsc, sizeof(Scal));
    if (st == PAGD_OK) st = dsync(s0);
    if (st != PAGD_OK) return bfail(b, st, s0->err.c_str());
    pagd_status first = PAGD_OK;
    for (int i = 0; i < count; i++) {
        if (!live[i]) continue;
        pagd_solver* s = b->m[i];
        const pagd_status si =
            run_finish(s, PI[i], dt, nsteps, iters_out ? iters_out + (size_t)i * total_steps + done : nullptr,
                       resid_out ? resid_out + (size_t)i * total_steps + done : nullptr, bs.bar_error != 0,
                       used_out ? used_out + (size_t)i * total_steps + done : nullptr);
        if (si != PAGD_OK) {
            live[i] = 0;
            if (status_out) status_out[i] = si;
            if (first == PAGD_OK) {
                first = si;
                char buf[256];
                std::snprintf(buf, sizeof(buf), "member %d: %s", i, s->err.c_str());
                b->err = buf;
            }
        }
    }
    return first;
}

// Whether every member alone fills every warp of the batched launch in every
// phase (row pairs, columns, middle-axis groups): a single launch then adds no
// concurrency, and members that drift apart in their phases make every global
// phase as slow as its slowest part, so such batches run member after member
// through the single-instance kernel.
static bool batch_members_fill_the_device(const pagd_batch* b) {
    // PAGD_BATCH_SEQ=0 / 1 forces the batched launch / member after member
    if (const char* e = std::getenv("PAGD_BATCH_SEQ")) {
        if ((e[0] == '0' || e[0] == '1') && e[1] == 0) return e[0] == '1';
    }
#ifdef PAGD_EMU
    return false;  // the emulation exists to exercise the batched kernel
#endif
    const long long warps = (long long)b->grid * b->wpb;
    for (const pagd_solver* s : b->m) {
        const long long rows = rows_of(s), nm = s->dim == 3 ? s->n[1] : 1;
        long long units = rows / 2;
        units = std::min(units, (long long)s->h1 * nm);
        if (s->dim == 3) units = std::min(units, (long long)s->h1 * (s->n[0] / kMidG));
        if (units < warps) return false;
    }
    return b->m.size() > 1;
}

pagd_status pagd_batch_run(pagd_batch* b, double dt, int nsteps, double tol, int* iters_out, double* resid_out,
                           int* status_out) {
    if (!b) return PAGD_EINVAL;
    if (!b->ws) return bfail(b, PAGD_ESTATE, "no batch workspace");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0 || !(tol >= 0.0))
        return bfail(b, PAGD_EINVAL, "bad dt / nsteps / tol");
    const int count = (int)b->m.size();
    for (int i = 0; i < count; i++) {
        pagd_solver* s = b->m[i];
        if (!s->ws || !s->have_state) return bfail(b, PAGD_ESTATE, "every member needs a workspace and a state");
        if (s->stream != b->stream) return bfail(b, PAGD_EINVAL, "members must share one stream");
    }
    std::vector<int> live(count, 1);
    if (status_out)
        for (int i = 0; i < count; i++) status_out[i] = PAGD_OK;
    pagd_status first = PAGD_OK;
    b->sequential = batch_members_fill_the_device(b) ? 1 : 0;
    if (b->sequential) {
        for (int i = 0; i < count; i++) {
            pagd_solver* s = b->m[i];
            const pagd_status si = pagd_run(s, nullptr, dt, nsteps, tol, iters_out ? iters_out + (size_t)i * nsteps : nullptr,
                                            resid_out ? resid_out + (size_t)i * nsteps : nullptr);
            if (si == PAGD_ECUDA || si == PAGD_ETIMEOUT) return bfail(b, si, s->err.c_str());
            if (si != PAGD_OK) {
                if (status_out) status_out[i] = si;
                if (first == PAGD_OK) {
                    first = si;
                    b->err = s->err;
                }
            }
        }
        return first;
    }
    int done = 0;
    while (done < nsteps) {
        const int c = (nsteps - done > kMaxChunk) ? kMaxChunk : nsteps - done;
        const pagd_status st = batch_chunk(b, dt, c, tol, live, done, nsteps, iters_out, resid_out, status_out);
        if (st != PAGD_OK && first == PAGD_OK) first = st;
        if (st == PAGD_ECUDA || st == PAGD_ETIMEOUT || st == PAGD_ENOMEM) return st;
        done += c;
    }
    return first;
}

pagd_status pagd_batch_step_with_guess(pagd_batch* b, const double* const* guesses, double dt, double tol,
                                       int* iters_out, double* resid_out, int* status_out, int* used_guess_out) {
    if (!b) return PAGD_EINVAL;
    if (!b->ws) return bfail(b, PAGD_ESTATE, "no batch workspace");
    if (!guesses) return bfail(b, PAGD_EINVAL, "null guess array");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(tol >= 0.0)) return bfail(b, PAGD_EINVAL, "bad dt / tol");
    const int count = (int)b->m.size();
    for (int i = 0; i < count; i++) {
        pagd_solver* s = b->m[i];
        if (!s->ws || !s->have_state) return bfail(b, PAGD_ESTATE, "every member needs a workspace and a state");
        if (s->stream != b->stream) return bfail(b, PAGD_EINVAL, "members must share one stream");
        if (guesses[i] && (s->scheme == PAGD_LBDF2 || s->scheme == PAGD_LMP))
            return bfail(b, PAGD_EINVAL, "an initial iterate applies to the implicit schemes only");
    }
    std::vector<int> live(count, 1);
    if (status_out)
        for (int i = 0; i < count; i++) status_out[i] = PAGD_OK;
    if (used_guess_out)
        for (int i = 0; i < count; i++) used_guess_out[i] = 0;
    b->sequential = batch_members_fill_the_device(b) ? 1 : 0;
    if (b->sequential) {
        pagd_status first = PAGD_OK;
        for (int i = 0; i < count; i++) {
            pagd_solver* s = b->m[i];
            pagd_status si;
            if (guesses[i]) {
                si = run_with_guess(s, guesses[i], dt, tol, iters_out ? iters_out + i : nullptr,
                                    resid_out ? resid_out + i : nullptr, used_guess_out ? used_guess_out + i : nullptr);
            } else {
                si = pagd_run(s, nullptr, dt, 1, tol, iters_out ? iters_out + i : nullptr, resid_out ? resid_out + i : nullptr);
            }
            if (si == PAGD_ECUDA || si == PAGD_ETIMEOUT) return bfail(b, si, s->err.c_str());
            if (si != PAGD_OK) {
                if (status_out) status_out[i] = si;
                if (first == PAGD_OK) {
                    first = si;
                    b->err = s->err;
                }
            }
        }
        return first;
    }
    return batch_chunk(b, dt, 1, tol, live, 0, 1, iters_out, resid_out, status_out, guesses, used_guess_out);
}

const char* pagd_batch_last_error(const pagd_batch* b) { return b ? b->err.c_str() : "null batch"; }

void pagd_batch_destroy(pagd_batch* b) { delete b; }

const char* pagd_last_error(const pagd_solver* s) { return s ? s->err.c_str() : "null solver"; }

void pagd_destroy(pagd_solver* s) { delete s; }

}  // extern "C"
