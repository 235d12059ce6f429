// batch.cuh -- one persistent cooperative kernel advancing many independent
// instances (own grid size, model parameters, scheme and initial data) through
// their PAGD time steps (Algorithm 2 per step).
//
// Every CTA keeps the control state of all instances in shared memory and runs
// the same control machine as the single-instance kernel for each of them, so
// instances move through their phases independently: one may be in an
// iteration column pass while another accepts a step.  A global phase is one
// work item per instance (its current phase), separated from the next by the
// device-wide barrier.  The work of a global phase is laid out on a cost axis:
// instance i covers [G_i, G_i + units_i * q_i), q_i the points a unit touches
// (2 n1 for a row unit of two rows, n0 for a column) times the relative cost
// per point of the instance's current phase (phase_weight: an FP64 base pass
// costs several FP32 iteration passes), and warp w of the grid takes the
// slice [C_w, C_{w+1}), C_w = floor(total * w / NW), so every warp gets about
// the same time of work whatever the mix of sizes and phases.  Each warp
// runs the members on its own slice; reductions are per warp (lane 0 publishes
// with an atomic), so warps never wait for each other inside a global phase.
#pragma once
#include "kernels.cuh"

namespace pagd {

template <class T, int NF>
__device__ __forceinline__ void batch_exec_nf(const Params& P, const Ctl& c, const Tw& t, char* wsm, double* red) {
    exec_phase<T, NF | kNoCoop>(P, c, t, wsm, red);
}

template <class T>
__device__ void batch_exec(const Params& P, const Ctl& c, const Tw& t, char* wsm, double* red) {
    switch (batch_nf(P.n0, P.n1)) {
        case 128: batch_exec_nf<T, 128>(P, c, t, wsm, red); break;
        case 256: batch_exec_nf<T, 256>(P, c, t, wsm, red); break;
        case 512: batch_exec_nf<T, 512>(P, c, t, wsm, red); break;
        default: batch_exec_nf<T, 0>(P, c, t, wsm, red); break;
    }
}

template <class T>
__global__ void __launch_bounds__(kMaxThreads, 1) pagd_batch_kernel(BatchParams B) {
    extern __shared__ __align__(16) char smem[];
    __shared__ double red[32];
    const int ntw = 1 << B.logtw;
    double2* t64 = (double2*)smem;
    float2* t32 = (float2*)(smem + (size_t)ntw * sizeof(double2));
    const int stride = kNMax >> B.logtw;
    for (int m = threadIdx.x; m < ntw; m += blockDim.x) {
        t64[m] = B.tw64[m * stride];
        t32[m] = B.tw32[m * stride];
    }
    Ctl* ctl = (Ctl*)(smem + tw_smem_bytes(B.logtw));
    long long* G = (long long*)(ctl + B.count);  // cost prefix, count + 1 entries
    char* wsm = smem + tw_smem_bytes(B.logtw) + batch_ctl_bytes(B.count);
    for (int i = threadIdx.x; i < B.count; i += blockDim.x) ctl[i] = ctl_init(B.PI[i]);
    const int wpb = blockDim.x / kWarp;
    const long long nw = (long long)gridDim.x * wpb;
    const long long gw = (long long)blockIdx.x * wpb + threadIdx.x / kWarp;
    unsigned gen = 0;
    __shared__ unsigned s_mask;
    int ntr = 0;
    const bool tr = B.trace && blockIdx.x == 0 && threadIdx.x == 0;
    if (tr) {
        B.trace[0] = 1ull << PH_DONE;  // start marker
        B.trace[1] = gtimer();
        ntr = 1;
    }
    for (;;) {
        __syncthreads();
        // cost prefix over the instances' current phases (warp 0, 32 at a time)
        if (threadIdx.x < 32) {
            long long base = 0;
            unsigned mask = 0;
            for (int i0 = 0; i0 < B.count; i0 += 32) {
                const int i = i0 + (int)threadIdx.x;
                long long v = 0;
                if (i < B.count && ctl[i].ph != PH_DONE) {
                    v = (long long)phase_units(B.PI[i], ctl[i].ph) * weighted_unit_cost(B.PI[i], ctl[i]);
                    mask |= 1u << ctl[i].ph;
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long u = __shfl_up_sync(0xffffffffu, v, o);
                    if ((int)threadIdx.x >= o) v += u;
                }
                if (i < B.count) G[i + 1] = base + v;
                base += __shfl_sync(0xffffffffu, v, 31);
            }
            mask = __reduce_or_sync(0xffffffffu, mask);
            if (threadIdx.x == 0) {
                G[0] = 0;
                s_mask = mask;
            }
        }
        __syncthreads();
        const long long total = G[B.count];
        if (total == 0) break;
        // the members on this warp's slice [C_gw, C_{gw+1}) of the cost axis; the
        // warps of a CTA need not agree (phases hold no CTA-wide barrier)
        const long long clo = cost_start(gw, total, nw), chi = cost_start(gw + 1, total, nw);
        int lo = 0, hi = B.count;  // first member with G[i+1] > clo
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (G[mid + 1] > clo) hi = mid;
            else lo = mid + 1;
        }
        for (int i = lo; i < B.count && G[i] < chi; i++) {
            const long long cost = G[i + 1] - G[i];
            if (cost == 0) continue;
            const Params& P = B.PI[i];
            Tw t{t64, t32, B.logtw, 0, 0, 0, 0};
            batch_split(t, gw, nw, total, G[i], cost, phase_units(P, ctl[i].ph), (int)weighted_unit_cost(P, ctl[i]));
            batch_exec<T>(P, ctl[i], t, wsm, red);
        }
        if (!grid_barrier(B.sc, gen)) break;
        if (tr && ntr < B.trace_cap) {
            B.trace[2 * ntr] = s_mask;
            B.trace[2 * ntr + 1] = gtimer();
            ntr++;
        }
        for (int i = threadIdx.x; i < B.count; i += blockDim.x)
            if (ctl[i].ph != PH_DONE) ctl_advance<T>(B.PI[i], ctl[i]);
    }
    if (tr) *B.ntrace = ntr;
}

template <class T>
cudaError_t pagd_batch_launch(const BatchParams& B, int grid, int threads, size_t smem, void* stream,
                              int* grid_used) {
    void (*kern)(BatchParams) = pagd_batch_kernel<T>;
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
    if (grid_used) *grid_used = grid;
    BatchParams Bc = B;
    void* args[] = {(void*)&Bc};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, smem,
                                       (cudaStream_t)stream);
}

}  // namespace pagd

#define PAGD_INSTANTIATE_BATCH(T) \
    template cudaError_t pagd::pagd_batch_launch<T>(const pagd::BatchParams&, int, int, size_t, void*, int*);
