// kernels.cuh -- the persistent cooperative kernel and its launcher.
//
// Included by one translation unit per fixed line length and iteration type
// (pagd_k<NF>_f32.cu / _f64.cu), each instantiating one pagd_launch<T, NF>; the
// units compile in parallel and link into libpagd.so.
#pragma once
#include "solver.cuh"
#include "cluster.cuh"

namespace pagd {


constexpr unsigned long long kBarrierTimeoutNs = 5000000000ull;  // 5 s per wait

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Device-wide barrier for a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows: barrier number g (from 1) is complete once it
// reaches g * gridDim.x.  Thread 0 publishes the CTA's writes with a release
// add (ordered after the CTA's other threads by __syncthreads) and waits with
// acquire loads.  The wait is bounded: after kBarrierTimeoutNs, or once another
// CTA has flagged an error, the CTA records the error and returns false
// instead of spinning on.
static __device__ bool grid_barrier(Scal* sc, unsigned& gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x;
        red_release_add(&sc->bar_count, 1ull);
        if (ld_acquire(&sc->bar_count) < target) {
            const unsigned long long t0 = gtimer();
            volatile int* ve = &sc->bar_error;
            while (ld_acquire(&sc->bar_count) < target) {
                if (*ve) { ok = 0; break; }
                if (gtimer() - t0 > kBarrierTimeoutNs) {
                    atomicOr(&sc->bar_error, 1);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    gen++;
    __syncthreads();
    return s_ok != 0;
}

template <class T, int NF>
__global__ void __launch_bounds__(kMaxThreads, 1) pagd_kernel(const __grid_constant__ Params P) {
    extern __shared__ __align__(16) char smem[];
    __shared__ double red[32];
    // twiddles exp(-2 pi i m / 2^logtw) staged from the global table
    const int ntw = 1 << P.logtw;
    double2* t64 = (double2*)smem;
    float2* t32 = (float2*)(smem + (size_t)ntw * sizeof(double2));
    const int stride = kNMax >> P.logtw;
    for (int m = threadIdx.x; m < ntw; m += blockDim.x) {
        t64[m] = P.tw64[m * stride];
        t32[m] = P.tw32[m * stride];
    }
    __syncthreads();
    const int wpb = blockDim.x / kWarp;
    const Tw tw{t64, t32, P.logtw, (int)(threadIdx.x / kWarp) * (int)gridDim.x + (int)blockIdx.x,
                (int)gridDim.x * wpb, 0, -1};
    char* wsm = smem + tw_smem_bytes(P.logtw);
    // The control state is the same in every thread: it lives in shared memory
    // and thread 0 advances it between two CTA barriers, which keeps its ~40
    // values out of the registers of the phase code.
    __shared__ Ctl c;
    unsigned gen = 0;
    int ntr = 0;
    if (threadIdx.x == 0) {
        c = ctl_init(P);
        if (P.trace && blockIdx.x == 0) {
            P.trace[0] = (unsigned long long)PH_DONE;  // start marker
            P.trace[1] = gtimer();
            ntr = 1;
        }
    }
    __syncthreads();
    while (c.ph != PH_DONE) {
        // the iterations of a base point run cluster-resident where the plan
        // chose it: cluster 0 loops until a decision other than "iterate on"
        // and hands its control state back through P.lctl
        const bool cl_phase = P.cl && c.ph == PH_CI;
        if (cl_phase) cluster_iterate<T, NF>(P, c, tw, wsm, &ntr);
        else exec_phase<T, NF>(P, c, tw, wsm, red);
        if (!grid_barrier(P.sc, gen)) break;
        if (threadIdx.x == 0) {
            if (P.trace && blockIdx.x == 0 && ntr < P.trace_cap && !cl_phase) {
                // bit 16: a phase of an incremental (T-transform) base evaluation
                const bool incb = c.inc && (c.ph == PH_B || c.ph == PH_C || c.ph == PH_D || c.ph == PH_E);
                P.trace[2 * ntr] = (unsigned long long)c.ph | (incb ? (1ull << 16) : 0ull);
                P.trace[2 * ntr + 1] = gtimer();
                ntr++;
            }
            if (cl_phase) {
                // resume after the loop's last row pass (phase RI)
                const unsigned* src = (const unsigned*)P.lctl;
                unsigned* dst = (unsigned*)&c;
                for (int i = 0; i < (int)(sizeof(Ctl) / sizeof(unsigned)); i++) dst[i] = __ldcg(src + i);
            }
            ctl_advance<T>(P, c);
        }
        __syncthreads();
    }
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0) P.sc->ntrace = ntr;
}


// Launch pagd_kernel<T, NF> cooperatively: the grid is capped at the number of
// co-resident CTAs so that the device-wide barrier is safe.
template <class T, int NF>
cudaError_t pagd_launch(const Params& P, int grid, int threads, size_t smem, void* stream, int* grid_used) {
    void (*kern)(const Params) = pagd_kernel<T, NF>;
    cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 1;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int cap = per_sm * sms;
    if (grid > cap) grid = cap;
    Params Pc = P;
    if (P.cl > 0) {
        // cluster launch: cluster 0 runs the iterations (cluster.cuh); the grid
        // is a whole number of clusters that the device co-schedules
        e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)P.cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cfg.gridDim = dim3((unsigned)P.cl);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = (cudaStream_t)stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (ncl < 1) return cudaErrorInvalidConfiguration;
        int nc = (grid + P.cl - 1) / P.cl;
        if (nc > ncl) nc = ncl;
        grid = nc * P.cl;
        if (grid_used) *grid_used = grid;
        cfg.gridDim = dim3((unsigned)grid);
        cfg.numAttrs = 2;
        return cudaLaunchKernelEx(&cfg, kern, Pc);
    }
    if (grid_used) *grid_used = grid;
    void* args[] = {(void*)&Pc};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, smem,
                                       (cudaStream_t)stream);
}

}  // namespace pagd

#define PAGD_INSTANTIATE(T, NF) \
    template cudaError_t pagd::pagd_launch<T, NF>(const pagd::Params&, int, int, size_t, void*, int*);
