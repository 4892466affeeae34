// Shared helpers for the GB300 (sm_103a) dense Kohn-Sham solver kernels.
// Storage convention everywhere: column-major, element (i, j) of a matrix with leading
// dimension ld at a[i + j * ld].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>

#include "elsi_gb.h"

namespace egb {

// Host-side count of the kernels this library has launched (reported through
// elsi_gb_launch_count for benchmarking).
extern std::atomic<long long> g_launches;
#define EGB_COUNT_LAUNCH() (::egb::g_launches.fetch_add(1, std::memory_order_relaxed))

// Device status word layout (one int array per handle, zeroed before each call):
//   [0] first error code seen by any kernel (ELSI_ERR_*), 0 = none
//   [1] auxiliary value (e.g. failing Cholesky pivot, 0-based)
enum { ST_CODE = 0, ST_AUX = 1, ST_WORDS = 8 };

__device__ __forceinline__ void report_error(int *status, int code, int aux)
{
    if (atomicCAS(status + ST_CODE, 0, code) == 0) status[ST_AUX] = aux;
}

// Default iteration limit of the SIMT spin waits of this library (the grid barrier of the
// cooperative kernels and the progress flags of the bulge chase). Each iteration backs off
// for 32-64 ns and reads a word from L2, so the limit is reached after seconds, far longer
// than any legitimate wait; on expiry the waiting kernel records ELSI_ERR_TIMEOUT and
// returns. The limit in force is read on the host at each launch (spin_limit()) and passed
// to the kernel, so that a test can make a wait run out (elsi_gb_set_spin_limit).
constexpr long long kSpinLimit = 1ll << 26;
long long spin_limit();

// Grid-wide barrier for cooperative launches (all CTAs co-resident by construction).
// *count lives in global memory, is zero before the launch and only grows: every CTA
// adds one at each barrier, so barrier number k (k = 1, 2, ...) is passed once the count
// reaches k * nblocks. Nobody resets the count, which saves the round trips of a
// generation word. A CTA that has polled the count more than `limit` times records
// ELSI_ERR_TIMEOUT. Returns false if the wait timed out or another CTA reported an error;
// the caller must then return.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target, int *status,
                                             long long limit)
{
    __shared__ int ok_flag;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        volatile unsigned *vc = count;
        volatile int *vst = status;
        long long it = 0;
        while (*vc < target) {
            if (++it > limit) { report_error(status, ELSI_ERR_TIMEOUT, 0); ok = 0; break; }
            if ((it & 255) == 0 && vst[ST_CODE] != 0) { ok = 0; break; }
            __nanosleep(32);
        }
        __threadfence();
        ok_flag = ok;
    }
    __syncthreads();
    return ok_flag != 0;
}

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

// Block-wide sum of one value per thread (blockDim.x multiple of 32, <= 1024). Every warp
// reduces the per-warp partials with the same shuffle tree, so all threads get the same
// bits without a second round through shared memory; the leading barrier keeps a
// previous call's readers of red ahead of this call's writers.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red /* >= 32 entries of shared */)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    T s = (lane < nw) ? red[lane] : T(0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// One-time set-up per device (cudaFuncSetAttribute and similar): such a setting applies to
// the device that is current when it is made, so a process that uses several GPUs has to
// make it once on each. fn() returns cudaError_t; it runs until it has succeeded once on
// the current device (two threads may both run it, which is harmless for these settings).
constexpr int kMaxDevices = 64;
struct PerDeviceOnce {
    std::atomic<bool> done[kMaxDevices];
};
template <typename F>
inline cudaError_t once_per_device(PerDeviceOnce &o, F &&fn)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return fn();
    if (o.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = fn();
    if (e == cudaSuccess) o.done[dev].store(true, std::memory_order_release);
    return e;
}

}  // namespace egb
