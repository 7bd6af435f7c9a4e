// Device-wide synchronisation shared by the persistent kernels (cooperative launches only).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace rafem {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// An error (a wait that gave up) is recorded in bar->err and also poisons the barrier counter with kBarrierPoison,
// so that every block learns of it from the count its barrier wait reads anyway: a count at least
// kBarrierPoison / 2 past a block's target can only come from an error (a launch passes fewer than 2^29 barrier
// arrivals). The counter and the error word are cleared together before each launch.
constexpr unsigned kBarrierPoison = 1u << 30;
__device__ __forceinline__ void raise_barrier_error(GridBarrier* bar, int code) {
    atomicExch(&bar->err, code);
    __threadfence();
    atomicAdd(&bar->count, kBarrierPoison);
}

// Grid barrier on a counter that only grows during a launch: every block adds 1 and waits until the counter
// reaches its own running target (gridDim.x per barrier). No block has a special role, so the release is one
// atomic plus one poll latency. The wait is bounded (wall clock spin_limit_ns): on expiry RAFEM_ERR_TIMEOUT is
// recorded. Returns true when the kernel must stop because an error was recorded.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, long long spin_limit_ns, unsigned& target) {
    __shared__ int s_err;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&bar->count, 1u);
        const unsigned long long t0 = globaltimer();
        long long spins = 0;
        unsigned c;
        int err = 0;
        while ((int)((c = ld_acquire_u32(&bar->count)) - target) < 0) {
            ++spins;
            if ((spins & 255) == 0 && ((long long)(globaltimer() - t0) > spin_limit_ns || spins > (1LL << 40))) {
                raise_barrier_error(bar, RAFEM_ERR_TIMEOUT);
                err = 1;
                break;
            }
        }
        __threadfence();
        s_err = err || c - target >= kBarrierPoison / 2;
    }
    __syncthreads();
    return s_err != 0;
}

}  // namespace rafem
