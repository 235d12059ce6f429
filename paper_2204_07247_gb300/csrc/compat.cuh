// compat.cuh -- lets the device code of this library also compile as plain
// host C++ (PAGD_EMU) so that its index arithmetic and control flow can be
// checked on a machine without a GPU.  The emulation runs one thread per CTA
// and executes the phases of the persistent kernel block by block; it is a
// test harness, never a code path of the shipped library.
#pragma once

#ifdef PAGD_EMU
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __noinline__
#define __launch_bounds__(...)

struct EmuDim3 { unsigned x, y, z; };
extern thread_local EmuDim3 threadIdx, blockIdx, blockDim, gridDim;

struct alignas(8) float2 { float x, y; };
struct alignas(16) double2 { double x, y; };
struct alignas(16) float4 { float x, y, z, w; };

inline void __syncthreads() {}
inline void __threadfence() {}
inline double atomicAdd(double* p, double v) { double o = *p; *p = o + v; return o; }
inline unsigned atomicAdd(unsigned* p, unsigned v) { unsigned o = *p; *p = o + v; return o; }
inline int atomicOr(int* p, int v) { int o = *p; *p = o | v; return o; }
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
    unsigned long long o = *p;
    if (v > o) *p = v;
    return o;
}
template <class T> inline T ldcg(const T* p) { return *p; }
template <class T> inline T ldg(const T* p) { return *p; }
inline unsigned long long dbl_bits(double d) { unsigned long long u; std::memcpy(&u, &d, 8); return u; }
inline double bits_dbl(unsigned long long u) { double d; std::memcpy(&d, &u, 8); return d; }
#define PAGD_WARP 1
template <class T> inline T warp_max(T v) { return v; }
template <class T> inline T warp_sum(T v) { return v; }
// asynchronous 16-byte global -> shared copies (the emulation copies at once)
inline void cp_async16(void* dst, const void* src) { std::memcpy(dst, src, 16); }
inline void cp_async_commit() {}
template <int N> inline void cp_async_wait() {}

#else  // CUDA
#include <cuda_runtime.h>
#include <stdint.h>
template <class T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <class T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
__device__ __forceinline__ unsigned long long dbl_bits(double d) { return (unsigned long long)__double_as_longlong(d); }
__device__ __forceinline__ double bits_dbl(unsigned long long u) { return __longlong_as_double((long long)u); }
#define PAGD_WARP 32
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v || w != w) ? w : v;
    }
    return v;
}
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Asynchronous 16-byte copy global -> shared (cp.async, cached in L2 only):
// both addresses 16-byte aligned.  Completion per thread in commit groups:
// cp_async_wait<N>() returns once at most N of this thread's most recent
// groups are still in flight; other threads' copies are visible after a
// barrier that follows their waits.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
#endif
