// common.cuh -- shared device helpers of librandutv: status flags, the bounded
// grid barrier used by the cooperative panel/SVD kernels, warp reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rutv {

// Bits OR-ed into the device status word; translated to randutv_status on the host.
enum : int {
    ST_NONFINITE = 1,
    ST_NOCONV = 2,
    ST_TIMEOUT = 4,
};

// A bounded wait gives up after this many polls (each poll sleeps ~64-256 ns),
// i.e. after roughly a second, records ST_TIMEOUT and lets the kernel return.
// This is the default; the host may lower it for the whole process
// (wait_limit() in internal.h), and every launcher of a kernel with a grid
// barrier passes the current value.
constexpr long long kSpinLimit = 1LL << 23;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch.  *count starts at 0 for the
// launch; the k-th barrier waits until count reaches k * gridDim.x.  Returns
// false (on every thread of the block) when the wait ran out after
// spin_limit polls; the caller then returns without touching more memory.
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned& target, int* status, long long spin_limit) {
    __shared__ int s_fail;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        s_fail = 0;
        __threadfence();
        atomicAdd(count, 1u);
        long long spins = 0;
        unsigned ns = 64;
        while (ld_acquire_u32(count) < target) {
            if (++spins > spin_limit) {
                atomicOr(status, ST_TIMEOUT);
                s_fail = 1;
                break;
            }
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
        }
        __threadfence();
    }
    __syncthreads();
    return s_fail == 0;
}

// A launch gate: a kernel launched under it runs only when the device int
// *flag is at least `need`, and otherwise returns at once on every thread.
// It lets a choice made on the device (the number of power iterations of a
// block step) skip launches the host has already queued, with no host
// synchronisation.  flag == nullptr: always open.
struct DevGate {
    const int* flag;
    int need;
};

__device__ __forceinline__ bool gate_closed(const DevGate g) {
    return g.flag != nullptr && *(const volatile int*)g.flag < g.need;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace rutv
